// push_mixed.cu -- launches of the mixed-precision tile body (push_tile.cuh):
// one CTA per tile of one run, a persistent form for a batch of runs, and the
// initial half step back of the momenta (App. A.3.1).
#include <algorithm>

#include "push_tile.cuh"

namespace pic {

namespace {

// One CTA per tile of one run; WALLS: conducting walls in x (a separate
// instantiation keeps their register cost out of the periodic kernel); CT: the
// fixed tile geometry code (fixed_tile), 0 for the run-time geometry.
template <int NDIM, int THREADS, int MINB, bool WALLS, bool HIST, int CT>
__global__ void __launch_bounds__(THREADS, MINB) k_push_mixed(const __grid_constant__ MixedStepArgs a) {
    push_tile<NDIM, THREADS, WALLS, HIST, CT>(a, blockIdx.x, &a);
}

// Persistent form for a batch of independent runs of uneven size: resident
// CTAs take (run, tile) work items from one counter until all tiles of all
// runs are done, so small runs do not leave most of the GPU idle.
// tile_prefix[r] is the number of tiles of runs 0..r-1.
template <int NDIM, int THREADS, int MINB, bool WALLS, bool HIST, int CT>
__global__ void __launch_bounds__(THREADS, MINB) k_push_mixed_multi(const MixedStepArgs *runs, const int *tile_prefix,
                                                                    int nruns, int *counter) {
    __shared__ int item_sh;
    __shared__ __align__(128) MixedStepArgs args_sh;
    const int total = tile_prefix[nruns];
    for (;;) {
        if (threadIdx.x == 0) item_sh = atomicAdd(counter, 1);
        __syncthreads();
        const int item = item_sh;
        if (item >= total) break;
        int lo = 0, hi = nruns;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (tile_prefix[mid] <= item) lo = mid; else hi = mid;
        }
        const int *src = reinterpret_cast<const int *>(runs + lo);
        int *dst = reinterpret_cast<int *>(&args_sh);
        for (int q = threadIdx.x; q < (int)(sizeof(MixedStepArgs) / sizeof(int)); q += THREADS) dst[q] = src[q];
        __syncthreads();
        push_tile<NDIM, THREADS, WALLS, HIST, CT>(args_sh, item - tile_prefix[lo], runs + lo);
    }
}

// Initial staggering (App. A.3.1): u^0 -> u^{-dt/2} by one Boris step of
// -dt/2 with the node fields gathered from global memory; no move, no deposit.
template <int NDIM>
__global__ void k_half_back_mixed(Geom g, const float4 *nfA, const float2 *nfB, SpeciesMixed P, long long n,
                                  float h, float dt) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        int ci, cj, ck;
        unpack_cell(NDIM, P.cell[p], ci, cj, ck);
        const float d[3] = {P.off[0][p], P.off[1][p], NDIM == 3 ? P.off[2][p] : 0.f};
        float u[3] = {P.u[0][p], P.u[1][p], P.u[2][p]};
        float E[3], B[3];
        gather_global<NDIM>(g, nfA, nfB, ci, cj, ck, d, E, B);
        boris<float>(u, E, B, h, -0.5f * dt);
        P.u[0][p] = u[0]; P.u[1][p] = u[1]; P.u[2][p] = u[2];
    }
}

// The kernel instance for a tile geometry code: the fixed form where one exists
// for NDIM (periodic runs), else the run-time one.
template <int NDIM, int THREADS, int MINB, bool WALLS, bool HIST>
auto push_kernel(int ct) {
    auto k = k_push_mixed<NDIM, THREADS, MINB, WALLS, HIST, 0>;
    if constexpr (!WALLS && NDIM == 3) {
        if (ct == 1) k = k_push_mixed<NDIM, THREADS, MINB, WALLS, HIST, 1>;
    } else if constexpr (!WALLS) {
        if (ct == 2) k = k_push_mixed<NDIM, THREADS, MINB, WALLS, HIST, 2>;
    }
    return k;
}
template <int NDIM, int THREADS, int MINB, bool WALLS, bool HIST>
auto push_multi_kernel(int ct) {
    auto k = k_push_mixed_multi<NDIM, THREADS, MINB, WALLS, HIST, 0>;
    // (the 3D fixed form spills a few registers in this kernel: the run-time one is kept)
    if constexpr (!WALLS && NDIM == 2) {
        if (ct == 2) k = k_push_mixed_multi<NDIM, THREADS, MINB, WALLS, HIST, 2>;
    }
    return k;
}

template <int NDIM, int THREADS, int MINB, bool WALLS, bool HIST>
void launch_t(const MixedStepArgs &a, size_t smem, cudaStream_t s) {
    auto k = push_kernel<NDIM, THREADS, MINB, WALLS, HIST>(fixed_tile_code(a.t, NDIM));
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<a.t.ntiles, THREADS, smem, s>>>(a);
}

}  // namespace

size_t mixed_smem_bytes(const TileGeom &t, int ndim) {
    const size_t nodes = (size_t)t.R[0] * t.R[1] * (ndim == 3 ? t.R[2] : 1);
    const int warps = (ndim == 3 ? 512 : 256) / 32;
    const size_t wwords = ndim == 3 ? warp_smem_words<3>() : warp_smem_words<2>();
    return node_b_offset((int)nodes) + nodes * (sizeof(float2) + 6 * sizeof(int)) + (size_t)warps * wwords * sizeof(int);
}

void launch_half_back_mixed(const Geom &g, const float4 *nfA, const float2 *nfB, SpeciesMixed sp, long long n,
                            float h, float dt, cudaStream_t s) {
    if (n <= 0) return;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 152LL * 16);
    if (g.ndim == 3) k_half_back_mixed<3><<<blocks, 256, 0, s>>>(g, nfA, nfB, sp, n, h, dt);
    else k_half_back_mixed<2><<<blocks, 256, 0, s>>>(g, nfA, nfB, sp, n, h, dt);
}

template <int NDIM, int THREADS, int MINB, bool WALLS, bool HIST>
void launch_multi_t(const MixedStepArgs *runs, const int *tile_prefix, int nruns, int *counter, size_t smem, int ct,
                    cudaStream_t s) {
    auto k = push_multi_kernel<NDIM, THREADS, MINB, WALLS, HIST>(ct);
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, THREADS, smem);
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k<<<std::max(1, per_sm) * sms, THREADS, smem, s>>>(runs, tile_prefix, nruns, counter);
}

template <int NDIM, int THREADS, int MINB>
void launch_multi_dim(const MixedStepArgs *runs, const int *tile_prefix, int nruns, int *counter, size_t smem,
                      bool walls, bool count, int ct, cudaStream_t s) {
    if (walls) {
        if (count) launch_multi_t<NDIM, THREADS, MINB, true, true>(runs, tile_prefix, nruns, counter, smem, ct, s);
        else launch_multi_t<NDIM, THREADS, MINB, true, false>(runs, tile_prefix, nruns, counter, smem, ct, s);
    } else {
        if (count) launch_multi_t<NDIM, THREADS, MINB, false, true>(runs, tile_prefix, nruns, counter, smem, ct, s);
        else launch_multi_t<NDIM, THREADS, MINB, false, false>(runs, tile_prefix, nruns, counter, smem, ct, s);
    }
}

void launch_push_mixed_multi(const MixedStepArgs *runs_dev, const int *tile_prefix_dev, int nruns, int ndim,
                             const TileGeom &t, bool walls, bool count, int *counter, cudaStream_t s) {
    const size_t smem = mixed_smem_bytes(t, ndim);
    const int ct = fixed_tile_code(t, ndim);
    if (ndim == 3) launch_multi_dim<3, 512, 1>(runs_dev, tile_prefix_dev, nruns, counter, smem, walls, count, ct, s);
    else launch_multi_dim<2, 256, 2>(runs_dev, tile_prefix_dev, nruns, counter, smem, walls, count, ct, s);
}

template <int NDIM, int THREADS, int MINB>
void launch_dim(const MixedStepArgs &a, size_t smem, cudaStream_t s) {
    const bool walls = a.g.bcx == 1, count = a.key_counts[0] != nullptr;
    if (walls) {
        if (count) launch_t<NDIM, THREADS, MINB, true, true>(a, smem, s);
        else launch_t<NDIM, THREADS, MINB, true, false>(a, smem, s);
    } else {
        if (count) launch_t<NDIM, THREADS, MINB, false, true>(a, smem, s);
        else launch_t<NDIM, THREADS, MINB, false, false>(a, smem, s);
    }
}

void launch_push_mixed(const MixedStepArgs &a, cudaStream_t s) {
    const size_t smem = mixed_smem_bytes(a.t, a.g.ndim);
    if (a.g.ndim == 3) launch_dim<3, 512, 1>(a, smem, s);
    else launch_dim<2, 256, 2>(a, smem, s);
}

}  // namespace pic
