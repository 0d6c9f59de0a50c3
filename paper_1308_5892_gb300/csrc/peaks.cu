// peaks.cu -- FP32 and FP64 fused multiply-add throughput of the device, the
// ALU denominators of the rooflines (the FP64 path is bound by GB300's FP64
// pipe, not by HBM).
//
// Every thread runs 8 independent FMA chains x <- x * a + b (|a| < 1, so the
// values stay bounded), enough independent work per warp to fill the pipe at
// full occupancy: 8 blocks of 256 threads per SM.  Each FMA counts as 2 flops.
// The loop body is unrolled 8 times, so loop overhead is small next to the 64
// FMAs per iteration.
#include <cuda_runtime.h>

#include "pic.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T *sink, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = T(threadIdx.x + u) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = fma(x[u], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int u = 0; u < 8; ++u) s += x[u];
    if (s == T(-1)) sink[blockIdx.x] = s;   // never true; keeps the chains alive
}

template <typename T>
pic_status run_peak(int iters, double *tflops, double *ms_out) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PIC_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PIC_ECUDA;
    const int blocks = sms * 8, threads = 256;
    T *sink = nullptr;
    if (cudaMalloc(&sink, sizeof(T) * blocks) != cudaSuccess) return PIC_ENOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    pic_status st = PIC_OK;
    float ms = 0.f;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = PIC_ECUDA;
    if (st == PIC_OK) {
        k_fma_peak<T><<<blocks, threads>>>(sink, iters / 8 + 1, T(0.999999), T(1e-7));   // warm-up
        cudaEventRecord(e0);
        k_fma_peak<T><<<blocks, threads>>>(sink, iters, T(0.999999), T(1e-7));
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            st = PIC_ECUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (st != PIC_OK) return st;
    const double flops = 2.0 * 64.0 * (double)iters * blocks * threads;
    if (tflops) *tflops = flops / ((double)ms * 1e-3) / 1e12;
    if (ms_out) *ms_out = ms;
    return PIC_OK;
}

}  // namespace

extern "C" pic_status pic_alu_peak(int kind, double *tflops, double *ms) {
    if (!tflops) return PIC_EINVAL;
    if (kind == PIC_PEAK_FP32_FMA) return run_peak<float>(1 << 15, tflops, ms);
    if (kind == PIC_PEAK_FP64_FMA) return run_peak<double>(1 << 9, tflops, ms);
    return PIC_EINVAL;
}
