// walk.cu -- the persistent step of a mixed ensemble: one launch runs every
// phase of one step of every run: on the steps that re-sort a run, the phases
// of the counting sort of each species (key histogram unless the previous push
// counted it, block scans, rank, gather), then the main loop of App. A.3.1:
// b half advance with the energy record, node-averaged fields,
// gather-push-deposit, the optional current smoothing (step 10), b half
// advance, e advance with the folded current.
//
// Work queue.  The items of phase ph of run r are the tiles of the run (push,
// and parts of the old layout's tiles for the sort's histogram and rank),
// chunks of cells_per_item cells or keys (field, smoothing, zeroing and
// scan-finish phases), scan blocks of 4096 keys, or gather chunks of 4096
// particles.  The queue order is phase-major; inside a phase the runs with the
// most particles per tile come first, so the longest items do not start last.
// Resident CTAs take items from one counter.  Before an item of phase ph of
// run r starts, every item of run r in the phases before ph must be done:
// thread 0 waits until the run's done counter reaches that count
// (base[r][ph]).  Every item it waits on lies earlier in the queue and was
// taken by a CTA that is running, so the earliest unfinished item never waits
// and the walk progresses whatever the number of resident CTAs.  Runs never
// wait on each other: while the tiles of a large run are being pushed, the
// field phases of runs that are done go on, so no phase ends with the GPU idle
// behind its slowest run.
//
// Bounded waits.  A wait that runs out (wait_ns of the device's global timer)
// sets ERR_TIMEOUT and the abort flag; every later item then skips its work and
// no wait blocks, so the launch ends promptly and pic_step reports
// PIC_ETIMEOUT.  The state of the step is then undefined.
//
// Ordering.  A finished item is published by a fence and an atomic add on the
// run's counter (thread 0, after the CTA barrier); the waiter reads the
// counter with acquire semantics and fences before the CTA barrier that
// releases its threads.  Items read arrays that other CTAs of the same launch
// wrote (b, the node fields, the current, the sort's counts, offsets and
// permutation), so this translation unit compiles the bodies with plain loads
// (PIC_COHERENT_LOADS) instead of the read-only data path, and the push stages
// the node fields with coalesced loads instead of TMA (they were written
// through the generic proxy).
//
// Every item runs the same per-cell and per-tile bodies as the phase launches
// (field_cells.cuh, smooth_cells.cuh, sort_cells.cuh, push_tile.cuh), so the
// fields, currents and particles are bitwise those of one launch per phase.
#include <algorithm>

#define PIC_COHERENT_LOADS 1
#include "field_cells.cuh"
#include "push_tile.cuh"
#include "smooth_cells.cuh"
#include "sort_cells.cuh"

namespace pic {

namespace {

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

// Thread 0: wait until run r has `target` items done.  False when the walk was
// aborted or this wait ran out (then the walk is aborted).
__device__ bool wait_run(const WalkArgs &w, int r, int target) {
    if (ld_acquire(w.abort) != 0) return false;
    if (ld_acquire(w.done + r) >= target) return true;
    const unsigned long long t0 = global_ns();
    for (int it = 0;; ++it) {
        __nanosleep(256);
        if (ld_acquire(w.done + r) >= target) return true;
        if (ld_acquire(w.abort) != 0) return false;
        // the timer bounds the wait; the poll count bounds it too, should the timer not advance
        if (global_ns() - t0 > (unsigned long long)w.wait_ns || it >= (1 << 26)) {
            atomicOr(w.err, ERR_TIMEOUT);
            atomicExch(w.abort, 1);
            return false;
        }
    }
}

// One field or smoothing item: cells [p0, p1) of run r.
template <int THREADS>
__device__ void field_item(const WalkArgs &w, int kind, int pass, const FieldRunF &fr, int local) {
    typedef unsigned long long u64;
    const Geom &g = fr.g;
    const long long p0 = (long long)local * w.cells_per_item;
    if (kind == W_B_HALF_E || kind == W_B_HALF) {
        const long long p1 = min(p0 + w.cells_per_item, g.pcells);
        double *slot = fr.hist.slot();
        double *energy_acc = slot ? slot + 2 : nullptr;
        double acc[6] = {0, 0, 0, 0, 0, 0};
        for (long long p = p0 + threadIdx.x; p < p1; p += THREADS)
            b_advance_cell<float>(g, fr.f, w.h, p, energy_acc != nullptr, acc);
        if (energy_acc) block_accumulate<6>(acc, energy_acc);
    } else if (kind == W_NODE) {
        const long long p1 = min(p0 + w.cells_per_item, g.pcells);
        for (long long p = p0 + threadIdx.x; p < p1; p += THREADS) node_cell(g, fr.f, fr.nfA, fr.nfB, p);
    } else if (kind == W_E_FX) {
        const long long p1 = min(p0 + w.cells_per_item, g.pcells);
        if (fr.hist_inc && local == 0 && threadIdx.x == 0) *fr.hist_inc += 1;
        const F2 sc = {(float)fr.scale, (float)(fr.scale - (double)(float)fr.scale)};
        for (long long p = p0 + threadIdx.x; p < p1; p += THREADS) {
            if (fr.smooth > 0)
                e_smoothed_cell<float, u64, long long>(g, fr.f, fr.sbuf[fr.smooth & 1], fr.scale, fr.Z[0], fr.Z[1],
                                                        fr.Z[2], w.dt, p);
            else
                e_fx_cell(g, fr.f, fr.J[0], fr.J[1], fr.J[2], fr.Z[0], fr.Z[1], fr.Z[2], w.dt, sc, p);
        }
    } else {
        // smoothing: compact interior cells (k*ny + j)*nx + i
        const long long ncell = (long long)g.nx * g.ny * g.nz;
        const long long p1 = min(p0 + w.cells_per_item, ncell);
        for (long long c = p0 + threadIdx.x; c < p1; c += THREADS) {
            if (kind == W_SMOOTH_FOLD) {
                int i, j, k;
                compact_coords(g, c, i, j, k);
                for (int q = 0; q < 3; ++q)
                    fr.sbuf[0][q * ncell + c] = (long long)image_sum<u64>(g, fr.J[q], i, j, k, false);
            } else {
                for (int q = 0; q < 3; ++q)
                    smooth_cell<long long>(g, fr.sbuf[pass & 1] + q * ncell, fr.sbuf[(pass + 1) & 1] + q * ncell, c);
            }
        }
    }
}

// Items per old tile of the sort's histogram and rank phases: about 32768
// particles each, at most 8 (a tile holds up to hundreds of thousands of
// particles; shorter items balance the walk, fewer items cost less queueing).
__host__ __device__ inline int walk_tile_parts(const SortArgs &a) {
    const long long per_tile = a.n / (a.t.ntiles > 0 ? a.t.ntiles : 1);
    const long long p = (per_tile + 32767) / 32768;
    return (int)(p < 1 ? 1 : (p > 8 ? 8 : p));
}

// One item of a sort phase: block `local` of the `nitems` blocks of that phase
// of species q's sort (sh: 33 ints of scratch for the scans).
template <int NDIM, int THREADS>
__device__ void sort_item(const SortArgs &a, int kind, int local, int nitems, int *sh) {
    const long long nkeys = nkeys_of(a);
    if (kind == S_ZERO || kind == S_ZERO_AFTER) {
        zero_body(a.counts, nkeys, local, nitems);
    } else if (kind == S_HIST) {
        const SrcWalk sw{a.old_tile_start, a.n, local, nitems, walk_tile_parts(a)};
        histogram_body<NDIM, 8>(a, sw, nkeys);
    } else if (kind == S_SCAN_BLOCKS) {
        scan_blocks_body<THREADS>(a.counts, a.offsets, a.block_sums, nkeys, local, sh);
    } else if (kind == S_SCAN_SUMS) {
        scan_sums_body<THREADS>(a.block_sums, scan_blocks(a), sh);
    } else if (kind == S_SCAN_FINISH) {
        scan_finish_body(a, nkeys, local, nitems);
    } else if (kind == S_RANK) {
        const SrcWalk sw{a.old_tile_start, a.n, local, nitems, walk_tile_parts(a)};
        rank_body<NDIM, 8>(a, sw, nkeys);
    } else {
        // fewer warps per SM than the sort's own gather launch: every array per
        // read of the permutation, more loads in flight per thread
        gather_all_body<NDIM, THREADS, 4>(a.src, a.dst, a.n, a.perm, local);
    }
}

template <int NDIM, int THREADS, int MINB, bool WALLS, bool HIST, int CT>
__global__ void __launch_bounds__(THREADS, MINB) k_walk(const __grid_constant__ WalkArgs w) {
    __shared__ int item_sh, go_sh;
    __shared__ int scan_sh[33];
    __shared__ __align__(16) SortArgs sort_sh;
    __shared__ __align__(128) MixedStepArgs args_sh;
    __shared__ __align__(16) FieldRunF fr_sh;
    const int nslot = w.nphase * w.nruns;
    __shared__ int slot_sh;
    if (threadIdx.x == 0) slot_sh = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            const int item = atomicAdd(w.head, 1);
            item_sh = item;
            // (phase, slot) of the item: the last slot whose first item is <= item.
            // A CTA's items increase, so the previous slot bounds the search.
            int lo = slot_sh;
            if (item < w.total && !(w.prefix[lo] <= item && item < w.prefix[lo + 1])) {
                int hi = nslot;
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (w.prefix[mid] <= item) lo = mid; else hi = mid;
                }
            }
            slot_sh = lo;
        }
        __syncthreads();
        const int item = item_sh;
        if (item >= w.total) break;
        const int lo = slot_sh;
        const int ph = lo / w.nruns, r = w.order[lo - ph * w.nruns];
        const int local = item - w.prefix[lo];
        const int kind = w.kind[ph];
        if (threadIdx.x == 0) {
            go_sh = wait_run(w, r, w.base[r * (w.nphase + 1) + ph]) ? 1 : 0;
            __threadfence();
        }
        __syncthreads();
        if (go_sh) {
            if (kind <= S_GATHER) {
                const int *src = reinterpret_cast<const int *>(w.sort + 4 * r + w.species[ph]);
                int *dst = reinterpret_cast<int *>(&sort_sh);
                for (int q = threadIdx.x; q < (int)(sizeof(SortArgs) / sizeof(int)); q += THREADS) dst[q] = src[q];
                __syncthreads();
                sort_item<NDIM, THREADS>(sort_sh, kind, local, w.prefix[lo + 1] - w.prefix[lo], scan_sh);
            } else if (kind == W_PUSH) {
                const int *src = reinterpret_cast<const int *>(w.push + r);
                int *dst = reinterpret_cast<int *>(&args_sh);
                for (int q = threadIdx.x; q < (int)(sizeof(MixedStepArgs) / sizeof(int)); q += THREADS) dst[q] = src[q];
                __syncthreads();
                if (threadIdx.x == 0) args_sh.use_tma = 0;
                __syncthreads();
                push_tile<NDIM, THREADS, WALLS, HIST, CT>(args_sh, local, w.push + r);
            } else {
                const FieldRunF *fsrc = kind == W_B_HALF_E ? w.fe + r : w.fp + r;
                const int *src = reinterpret_cast<const int *>(fsrc);
                int *dst = reinterpret_cast<int *>(&fr_sh);
                for (int q = threadIdx.x; q < (int)(sizeof(FieldRunF) / sizeof(int)); q += THREADS) dst[q] = src[q];
                __syncthreads();
                field_item<THREADS>(w, kind, w.pass[ph], fr_sh, local);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(w.done + r, 1);
        }
    }
}

// The walker instance for a tile geometry code (fixed_tile): the fixed form where
// one exists for NDIM (periodic runs), else the run-time one.
template <int NDIM, int THREADS, int MINB, bool WALLS, bool HIST>
auto walk_kernel(int ct) {
    auto k = k_walk<NDIM, THREADS, MINB, WALLS, HIST, 0>;
    // (the 3D fixed form spills a few registers in this kernel: the run-time one is kept)
    if constexpr (!WALLS && NDIM == 2) {
        if (ct == 2) k = k_walk<NDIM, THREADS, MINB, WALLS, HIST, 2>;
    }
    return k;
}

template <int NDIM, int THREADS, int MINB, bool WALLS, bool HIST>
bool fits_t(size_t smem) {
    cudaFuncAttributes attr;
    // the fixed-geometry forms hold the same static shared memory
    if (cudaFuncGetAttributes(&attr, k_walk<NDIM, THREADS, MINB, WALLS, HIST, 0>) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return attr.sharedSizeBytes + smem <= (size_t)optin;
}

template <int NDIM, int THREADS, int MINB, bool WALLS, bool HIST>
void launch_t(const WalkArgs &w, size_t smem, int ct, cudaStream_t s) {
    auto k = walk_kernel<NDIM, THREADS, MINB, WALLS, HIST>(ct);
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0, dev = 0, sms = 152;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, THREADS, smem);
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::max(1, std::min(per_sm * sms, w.total));
    k<<<grid, THREADS, smem, s>>>(w);
}

template <int NDIM, int THREADS, int MINB>
void launch_dim(const WalkArgs &w, bool walls, bool count, size_t smem, int ct, cudaStream_t s) {
    if (walls) {
        if (count) launch_t<NDIM, THREADS, MINB, true, true>(w, smem, ct, s);
        else launch_t<NDIM, THREADS, MINB, true, false>(w, smem, ct, s);
    } else {
        if (count) launch_t<NDIM, THREADS, MINB, false, true>(w, smem, ct, s);
        else launch_t<NDIM, THREADS, MINB, false, false>(w, smem, ct, s);
    }
}

template <int NDIM, int THREADS, int MINB>
bool fits_dim(bool walls, bool count, size_t smem) {
    if (walls) return count ? fits_t<NDIM, THREADS, MINB, true, true>(smem) : fits_t<NDIM, THREADS, MINB, true, false>(smem);
    return count ? fits_t<NDIM, THREADS, MINB, false, true>(smem) : fits_t<NDIM, THREADS, MINB, false, false>(smem);
}

}  // namespace

// Field items of 32 cells per thread: 8192 cells (2D, 256 threads), 16384 (3D, 512 threads).
int walk_cells_per_item(int ndim) { return ndim == 3 ? 16384 : 8192; }

int walk_sort_items(const SortArgs &a, int kind, int cpi) {
    const long long nkeys = nkeys_of(a);
    auto chunks = [](long long n, long long per) { return (int)std::max<long long>(1, (n + per - 1) / per); };
    switch (kind) {
    case S_ZERO: return a.counted ? 0 : chunks(nkeys, cpi);
    case S_HIST: return (a.counted || a.n == 0) ? 0 : (a.old_tile_start ? a.t.ntiles * walk_tile_parts(a) : chunks(a.n, cpi));
    case S_SCAN_BLOCKS: return scan_blocks(a);
    case S_SCAN_SUMS: return 1;
    case S_SCAN_FINISH: return chunks(nkeys, cpi);
    case S_RANK: return a.n == 0 ? 0 : (a.old_tile_start ? a.t.ntiles * walk_tile_parts(a) : chunks(a.n, cpi));
    case S_ZERO_AFTER: return chunks(nkeys, cpi);
    case S_GATHER: return a.n == 0 ? 0 : chunks(a.n, kGatherChunk);
    default: return 0;
    }
}

bool walk_fits(int ndim, bool walls, bool count, size_t push_smem) {
    return ndim == 3 ? fits_dim<3, 512, 1>(walls, count, push_smem) : fits_dim<2, 256, 2>(walls, count, push_smem);
}

void launch_walk(const WalkArgs &w, int ndim, bool walls, bool count, size_t push_smem, int tile_code,
                 cudaStream_t s) {
    if (w.total <= 0) return;
    if (ndim == 3) launch_dim<3, 512, 1>(w, walls, count, push_smem, tile_code, s);
    else launch_dim<2, 256, 2>(w, walls, count, push_smem, tile_code, s);
}

}  // namespace pic
