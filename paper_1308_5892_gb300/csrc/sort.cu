// sort.cu -- counting sort of the mixed-path particles by tile-major cell key.
//
// key(cell) = tile_index * cells_per_tile + index of the cell inside its tile,
// so particles end up grouped by tile and, inside a tile, by cell; the cell
// order inside a tile is then stored block-transposed (interleaved_slot).  The sort
// is out of place (src -> dst, the caller swaps the buffers): histogram of the
// keys (unless the preceding push counted it), exclusive scan, a rank pass
// whose per-key cursors are advanced with warp-aggregated atomics (lanes of a
// warp that share a key take consecutive slots with one atomic) and which
// writes only the 4-byte inverse permutation, then a gather pass that writes
// every particle array in destination order (coalesced stores; scattered
// partial-sector stores of the full particle state cost several times its size
// in DRAM traffic).  The tile offsets are read from the scanned counts, and
// the counts are left zeroed for the next push to count into.  Every phase also
// has a batched form that sorts one species of many runs in one launch.
//
// Roofline: HBM bound; per particle 4 B (histogram) + 8 B (rank) +
// 4 + 2 x (24..28 + 4) B (gather) plus per key 3 x 4 B.  Particle counts are
// int32 (at most 2^31 - 1 particles per species).
#include "pic_internal.cuh"
#include "sort_cells.cuh"

namespace pic {

namespace {

// ---- block counts of the phases of one sort ----

inline int blocks_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    const long long cap = 152LL * 32;
    return (int)(b < 1 ? 1 : (b < cap ? b : cap));
}
constexpr int kWalkThreads = 512;
inline int walk_blocks(const SortArgs &a) { return a.old_tile_start ? a.t.ntiles : blocks_for(a.n, kWalkThreads); }
inline int key_blocks(const SortArgs &a) { return blocks_for(nkeys_of(a), 256); }
inline int gather_blocks(const SortArgs &a) { return (int)((a.n + kGatherChunk - 1) / kGatherChunk); }

// ---- one sort: one launch per phase ----

__global__ void k_zero(SortArgs a) { zero_body(a.counts, nkeys_of(a), blockIdx.x, gridDim.x); }

template <int NDIM>
__global__ void k_histogram(SortArgs a) {
    const SrcWalk w{a.old_tile_start, a.n, (int)blockIdx.x, (int)gridDim.x};
    histogram_body<NDIM, 4>(a, w, nkeys_of(a));
}

__global__ void __launch_bounds__(kScanThreads) k_scan_blocks(SortArgs a) {
    __shared__ int sh[33];
    scan_blocks_body<kScanThreads>(a.counts, a.offsets, a.block_sums, nkeys_of(a), blockIdx.x, sh);
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sums(SortArgs a) {
    __shared__ int sh[33];
    scan_sums_body<kScanThreads>(a.block_sums, scan_blocks(a), sh);
}

__global__ void k_scan_finish(SortArgs a) { scan_finish_body(a, nkeys_of(a), blockIdx.x, gridDim.x); }

template <int NDIM>
__global__ void k_rank(SortArgs a) {
    const SrcWalk w{a.old_tile_start, a.n, (int)blockIdx.x, (int)gridDim.x};
    rank_body<NDIM, 4>(a, w, nkeys_of(a));
}

template <int NDIM>
__global__ void __launch_bounds__(kGatherThreads) k_gather(SortArgs a) {
    gather_body<NDIM, kGatherThreads, 4>(a.src, a.dst, a.n, a.perm, blockIdx.x);
}

// ---- many independent sorts (one species of every run of an ensemble): one
// launch per phase; block B belongs to sort s with prefix[s] <= B < prefix[s+1]
// of that phase's block prefix. ----

__device__ inline int find_sort(const int *prefix, int nsort, int B) {
    int lo = 0, hi = nsort;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= B) lo = mid; else hi = mid;
    }
    return lo;
}

// always: zero the counts of every sort (after its rank pass); otherwise skip sorts counted by the push
__global__ void k_zero_multi(const SortArgs *as, const int *prefix, int nsort, int always) {
    const int s = find_sort(prefix, nsort, blockIdx.x);
    const SortArgs &a = as[s];
    if (a.counted && !always) return;
    zero_body(a.counts, nkeys_of(a), blockIdx.x - prefix[s], prefix[s + 1] - prefix[s]);
}

template <int NDIM>
__global__ void k_histogram_multi(const SortArgs *as, const int *prefix, int nsort) {
    const int s = find_sort(prefix, nsort, blockIdx.x);
    const SortArgs &a = as[s];
    if (a.counted) return;
    const SrcWalk w{a.old_tile_start, a.n, (int)blockIdx.x - prefix[s], prefix[s + 1] - prefix[s]};
    histogram_body<NDIM, 4>(a, w, nkeys_of(a));
}

__global__ void __launch_bounds__(kScanThreads) k_scan_blocks_multi(const SortArgs *as, const int *prefix,
                                                                    int nsort) {
    __shared__ int sh[33];
    const int s = find_sort(prefix, nsort, blockIdx.x);
    const SortArgs &a = as[s];
    scan_blocks_body<kScanThreads>(a.counts, a.offsets, a.block_sums, nkeys_of(a), blockIdx.x - prefix[s], sh);
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sums_multi(const SortArgs *as) {
    __shared__ int sh[33];
    const SortArgs &a = as[blockIdx.x];
    scan_sums_body<kScanThreads>(a.block_sums, scan_blocks(a), sh);
}

__global__ void k_scan_finish_multi(const SortArgs *as, const int *prefix, int nsort) {
    const int s = find_sort(prefix, nsort, blockIdx.x);
    scan_finish_body(as[s], nkeys_of(as[s]), blockIdx.x - prefix[s], prefix[s + 1] - prefix[s]);
}

template <int NDIM>
__global__ void k_rank_multi(const SortArgs *as, const int *prefix, int nsort) {
    const int s = find_sort(prefix, nsort, blockIdx.x);
    const SortArgs &a = as[s];
    const SrcWalk w{a.old_tile_start, a.n, (int)blockIdx.x - prefix[s], prefix[s + 1] - prefix[s]};
    rank_body<NDIM, 4>(a, w, nkeys_of(a));
}

template <int NDIM>
__global__ void __launch_bounds__(kGatherThreads) k_gather_multi(const SortArgs *as, const int *prefix, int nsort) {
    const int s = find_sort(prefix, nsort, blockIdx.x);
    const SortArgs &a = as[s];
    gather_body<NDIM, kGatherThreads, 4>(a.src, a.dst, a.n, a.perm, blockIdx.x - prefix[s]);
}

}  // namespace

size_t sort_scan_scratch(long long nkeys) { return (size_t)((nkeys + kScanTile - 1) / kScanTile + 1); }

void launch_sort(const SortArgs &a, cudaStream_t s) {
    if (!a.counted) k_zero<<<key_blocks(a), 256, 0, s>>>(a);
    if (a.n > 0 && !a.counted) {
        if (a.g.ndim == 3) k_histogram<3><<<walk_blocks(a), kWalkThreads, 0, s>>>(a);
        else k_histogram<2><<<walk_blocks(a), kWalkThreads, 0, s>>>(a);
    }
    k_scan_blocks<<<scan_blocks(a), kScanThreads, 0, s>>>(a);
    k_scan_sums<<<1, kScanThreads, 0, s>>>(a);
    k_scan_finish<<<key_blocks(a), 256, 0, s>>>(a);
    if (a.n > 0) {
        if (a.g.ndim == 3) {
            k_rank<3><<<walk_blocks(a), kWalkThreads, 0, s>>>(a);
            k_gather<3><<<gather_blocks(a), kGatherThreads, 0, s>>>(a);
        } else {
            k_rank<2><<<walk_blocks(a), kWalkThreads, 0, s>>>(a);
            k_gather<2><<<gather_blocks(a), kGatherThreads, 0, s>>>(a);
        }
    }
    // the counts end zeroed, ready for a push that counts the next sort's histogram
    k_zero<<<key_blocks(a), 256, 0, s>>>(a);
}

void sort_multi_prefixes(const SortArgs *h_args, int nsort, int *h_prefix) {
    int *pz = h_prefix, *pw = h_prefix + (nsort + 1), *pb = h_prefix + 2 * (nsort + 1),
        *pg = h_prefix + 3 * (nsort + 1);
    pz[0] = pw[0] = pb[0] = pg[0] = 0;
    for (int i = 0; i < nsort; ++i) {
        const SortArgs &a = h_args[i];
        pz[i + 1] = pz[i] + key_blocks(a);
        pw[i + 1] = pw[i] + (a.n > 0 ? walk_blocks(a) : 0);
        pb[i + 1] = pb[i] + scan_blocks(a);
        pg[i + 1] = pg[i] + gather_blocks(a);
    }
}

void launch_sort_multi(const SortArgs *d_args, const int *d_prefix, const int *h_prefix, int nsort, int ndim,
                       cudaStream_t s) {
    if (nsort <= 0) return;
    const int *pz = d_prefix, *pw = d_prefix + (nsort + 1), *pb = d_prefix + 2 * (nsort + 1),
              *pg = d_prefix + 3 * (nsort + 1);
    const int nz = h_prefix[nsort], nw = h_prefix[2 * (nsort + 1) - 1], nb = h_prefix[3 * (nsort + 1) - 1],
              ng = h_prefix[4 * (nsort + 1) - 1];
    k_zero_multi<<<nz, 256, 0, s>>>(d_args, pz, nsort, 0);
    if (nw > 0) {
        if (ndim == 3) k_histogram_multi<3><<<nw, kWalkThreads, 0, s>>>(d_args, pw, nsort);
        else k_histogram_multi<2><<<nw, kWalkThreads, 0, s>>>(d_args, pw, nsort);
    }
    k_scan_blocks_multi<<<nb, kScanThreads, 0, s>>>(d_args, pb, nsort);
    k_scan_sums_multi<<<nsort, kScanThreads, 0, s>>>(d_args);
    k_scan_finish_multi<<<nz, 256, 0, s>>>(d_args, pz, nsort);
    if (nw > 0) {
        if (ndim == 3) k_rank_multi<3><<<nw, kWalkThreads, 0, s>>>(d_args, pw, nsort);
        else k_rank_multi<2><<<nw, kWalkThreads, 0, s>>>(d_args, pw, nsort);
    }
    // the counts end zeroed, ready for a push that counts the next sort's histogram
    k_zero_multi<<<nz, 256, 0, s>>>(d_args, pz, nsort, 1);
    if (ng > 0) {
        if (ndim == 3) k_gather_multi<3><<<ng, kGatherThreads, 0, s>>>(d_args, pg, nsort);
        else k_gather_multi<2><<<ng, kGatherThreads, 0, s>>>(d_args, pg, nsort);
    }
}

}  // namespace pic
