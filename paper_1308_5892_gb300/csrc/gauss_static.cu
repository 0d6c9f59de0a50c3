// gauss_static.cu -- Gauss-law residual of a caller-owned FP64 state that
// allocates no device memory.
//
// The FP64 diagnostics of a context (pic_diagnostics) deposit the charge
// density into a scratch grid that pic_init obtains from the allocator.  Some
// callers cannot allocate device memory at the point where they want this
// check: code that runs between the stages of a pipeline whose memory pool is
// fixed up front, hosts whose allocator is owned by another framework, or
// loops that must not enter the CUDA allocator (and its implicit
// synchronisation) at all.  pic_gauss_residual_static serves them: its only
// scratch is the file-scope device array below, which every GPU that loads
// the library holds, whole, until the process exits.
#include <cstdio>
#include <mutex>

#include "../../include/pic.h"
#include "pic_internal.cuh"

namespace pic {

namespace {

constexpr long long kStaticCells = 1LL << 20;   // largest nx*ny*nz accepted (8 MiB of doubles)

// Charge density of the nodes, shared by every call on this device.
static __device__ __align__(256) double g_rho_static[kStaticCells];

// Device address of g_rho_static per device, resolved once with that device
// current; the mutex makes the first resolution safe when several host threads
// call at once.  The cache lives as long as the process: after cudaDeviceReset
// the runtime reloads the module at another address, so the entry point must
// not be used after a reset.
double *g_rho_addr[64] = {nullptr};
std::mutex g_rho_mutex;

__global__ void k_zero_d(double *a, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a[i] = 0.0;
}

__device__ inline void max_nonneg(double *addr, double v) {
    atomicMax(reinterpret_cast<long long *>(addr), __double_as_longlong(v));
}

// max over nodes of |div e - rho|; e in the plain (unpadded) layout.
__global__ void k_div_minus_rho_max(Geom g, const double *ex, const double *ey, const double *ez, const double *rho,
                                    double *out) {
    const long long n = (long long)g.nx * g.ny * g.nz;
    double m = 0.0;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % g.nx);
        const long long r = q / g.nx;
        const int j = (int)(r % g.ny), k = (int)(r / g.ny);
        const double div = (ex[q] - ex[g.widx(i - 1, j, k)]) + (ey[q] - ey[g.widx(i, j - 1, k)]) +
                           (ez[q] - ez[g.widx(i, j, k - 1)]);
        m = fmax(m, fabs(div - rho[q]));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) max_nonneg(out, m);
}

inline int blocks(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : (b < 152LL * 16 ? b : 152LL * 16));
}

}  // namespace

}  // namespace pic

using namespace pic;

extern "C" pic_status pic_gauss_residual_static(int ndim, int nx, int ny, int nz, const double *e, int nspecies,
                                                const int64_t *counts, const double *const *pos,
                                                const double *alpha, double *out, void *stream) {
    if (ndim != 2 && ndim != 3) return PIC_EINVAL;
    if (ndim == 2 && nz != 1) return PIC_EINVAL;
    if (nx < 2 || ny < 2 || (ndim == 3 && nz < 2)) return PIC_EINVAL;
    const long long ncell = (long long)nx * ny * nz;
    if (ncell > kStaticCells) {
        fprintf(stderr, "pic_gauss_residual_static: %lld cells exceed the static limit of %lld\n", ncell,
                kStaticCells);
        return PIC_EINVAL;
    }
    if (!e || !out || nspecies < 0 || nspecies > PIC_MAX_SPECIES || (nspecies > 0 && (!counts || !pos || !alpha)))
        return PIC_EINVAL;
    for (int s = 0; s < nspecies; ++s)
        if (counts[s] < 0 || (counts[s] > 0 && !pos[s])) return PIC_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return PIC_ECUDA;
    double *rho = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_rho_mutex);
        if (!g_rho_addr[dev]) {
            // the symbol's device address, resolved on the current device (first call only)
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_rho_static) != cudaSuccess || !ptr) return PIC_ECUDA;
            g_rho_addr[dev] = (double *)ptr;
        }
        rho = g_rho_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    Geom g{};
    g.ndim = ndim; g.nx = nx; g.ny = ny; g.nz = nz;
    g.G = 0; g.Gz = 0;
    g.px = nx; g.py = ny; g.pz = nz;
    g.pcells = ncell;
    g.set_divisors();
    g.bcx = 0;
    // out[0] = max |div e - rho~|, out[1] = max over species of max |rho~_s|
    k_zero_d<<<1, 32, 0, s>>>(out, 2);
    for (int sp = 0; sp < nspecies; ++sp) {
        Species64 P{};
        for (int a = 0; a < 3; ++a) P.x[a] = const_cast<double *>(pos[sp] + (size_t)a * counts[sp]);
        k_zero_d<<<blocks(ncell), 256, 0, s>>>(rho, ncell);
        launch_rho64(g, P, counts[sp], alpha[sp], rho, s);
        launch_max_abs_diff(rho, nullptr, ncell, out + 1, s);
    }
    k_zero_d<<<blocks(ncell), 256, 0, s>>>(rho, ncell);
    for (int sp = 0; sp < nspecies; ++sp) {
        Species64 P{};
        for (int a = 0; a < 3; ++a) P.x[a] = const_cast<double *>(pos[sp] + (size_t)a * counts[sp]);
        launch_rho64(g, P, counts[sp], alpha[sp], rho, s);
    }
    k_div_minus_rho_max<<<blocks(ncell), 256, 0, s>>>(g, e, e + ncell, e + 2 * ncell, rho, out);
    return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}
