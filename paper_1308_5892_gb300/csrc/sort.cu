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

namespace pic {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

template <int NDIM>
__device__ inline int cell_key(const TileGeom &t, uint32_t c) {
    int i, j, k;
    unpack_cell(NDIM, c, i, j, k);
    if (t.lg[0] >= 0) return tile_key_pow2(t, i, j, k);   // shifts instead of divisions
    const int ti = i / t.T[0], tj = j / t.T[1], tk = NDIM == 3 ? k / t.T[2] : 0;
    const int li = i - ti * t.T[0], lj = j - tj * t.T[1], lk = NDIM == 3 ? k - tk * t.T[2] : 0;
    const int tile = (tk * t.ntile[1] + tj) * t.ntile[0] + ti;
    return tile * t.cells_per_tile + (lk * t.T[1] + lj) * t.T[0] + li;
}

// Tile of a key.
__device__ inline int key_tile(const TileGeom &t, int key) {
    return t.lg[0] >= 0 ? key >> (t.lg[0] + t.lg[1] + t.lg[2]) : key / t.cells_per_tile;
}

// Position of cell-sorted rank r inside a tile of n_t particles: every full
// block of 1024 is stored as a 32 x 32 transpose, so that lane a of a warp,
// reading element base + 32k + a for k = 0..31, walks the 32 consecutive
// ranks 32a .. 32a+31 (mostly one cell) while the 32 lanes of one load sit in
// 32 different cells; the tail of the tile (n_t mod 1024) keeps rank order.
__device__ __forceinline__ int interleaved_slot(int r, int n_t) {
    const int nfull = n_t & ~1023;
    if (r >= nfull) return r;
    const int i = r & 1023;
    return (r - i) + ((i & 31) << 5) + (i >> 5);
}

// Source traversal: with a tiled source (sorted before), CTA b walks old tile b
// in its cell-sorted rank order (slot t0 + interleaved_slot(i)), so consecutive
// threads see consecutive ranks of one cell; an untiled source (as uploaded)
// is walked in storage order by a grid-stride loop.
struct SrcWalk {
    const int *old_start;   // old tile offsets, or nullptr when the source is untiled
    long long n;
    int b, nb;              // this block and the block count of the walk
    __device__ __forceinline__ void begin(long long &i, long long &end, int &t0, int &nt) const {
        if (old_start) {
            t0 = old_start[b];
            nt = old_start[b + 1] - t0;
            i = threadIdx.x;
            end = nt;
        } else {
            t0 = 0;
            nt = 0;
            i = (long long)b * blockDim.x + threadIdx.x;
            end = n;
        }
    }
    __device__ __forceinline__ long long step() const {
        return old_start ? (long long)blockDim.x : (long long)nb * blockDim.x;
    }
    __device__ __forceinline__ long long pos(long long i, int t0, int nt) const {
        return old_start ? (long long)t0 + interleaved_slot((int)i, nt) : i;
    }
};

// ---- phase bodies, written for block b of nb blocks working on one sort ----

__device__ inline void zero_body(int *a, long long n, int b, int nb) {
    for (long long i = (long long)b * blockDim.x + threadIdx.x; i < n; i += (long long)nb * blockDim.x) a[i] = 0;
}

// Keys of the four source elements i + v * step (v = 0..3) of a walk, -1 past its end.
template <int NDIM>
__device__ __forceinline__ void walk_keys(const SortArgs &a, const SrcWalk &w, long long i, long long end, int t0,
                                          int nt, long long nkeys, long long (&p)[4], int (&key)[4]) {
    uint32_t c[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const long long iv = i + v * w.step();
        p[v] = iv < end ? w.pos(iv, t0, nt) : -1;
        c[v] = p[v] >= 0 ? __ldg(a.src.cell + p[v]) : 0u;
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        key[v] = p[v] >= 0 ? cell_key<NDIM>(a.t, c[v]) : -1;
        if (p[v] >= 0 && (key[v] < 0 || key[v] >= nkeys)) {
            atomicOr(a.err, ERR_SORT);
            key[v] = -1;
        }
    }
}

template <int NDIM>
__device__ inline void histogram_body(const SortArgs &a, const SrcWalk &w, long long nkeys) {
    long long i, end;
    int t0, nt;
    w.begin(i, end, t0, nt);
    // four independent loads in flight per thread; the loop is warp-uniform
    // (every lane takes part in the warp aggregation)
    const int lane = threadIdx.x & 31;
    for (long long ib = i - lane; ib < end; ib += 4 * w.step()) {
        long long p[4];
        int key[4];
        walk_keys<NDIM>(a, w, ib + lane, end, t0, nt, nkeys, p, key);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            // warp aggregation: lanes with the same key add once
            const unsigned peers = __match_any_sync(0xffffffffu, key[v]);
            const int leader = __ffs(peers) - 1;
            if (key[v] >= 0 && (int)(threadIdx.x & 31) == leader) atomicAdd(a.counts + key[v], __popc(peers));
        }
    }
}

// Block-level exclusive scan of kScanTile ints; returns the block total.
__device__ inline int block_scan(int (&v)[kScanItems], int *sh) {
    int local = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) { const int x = v[q]; v[q] = local; local += x; }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = local;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) sh[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = lane < (kScanThreads / 32) ? sh[lane] : 0;
        int wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        sh[lane] = wi - w;       // exclusive warp offsets
        if (lane == 31) sh[32] = wi;
    }
    __syncthreads();
    const int off = sh[warp] + incl - local;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) v[q] += off;
    const int total = sh[32];
    __syncthreads();
    return total;
}

// Scan of block b's kScanTile counts into offsets; the block total goes to block_sums[b].
__device__ inline void scan_blocks_body(const int *in, int *out, int *block_sums, long long n, int b, int *sh) {
    const long long base = (long long)b * kScanTile + (long long)threadIdx.x * kScanItems;
    int v[kScanItems];
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) v[q] = base + q < n ? in[base + q] : 0;
    const int total = block_scan(v, sh);
#pragma unroll
    for (int q = 0; q < kScanItems; ++q)
        if (base + q < n) out[base + q] = v[q];
    if (threadIdx.x == 0) block_sums[b] = total;
}

// Exclusive scan of the block sums in one block (any count, in chunks).
__device__ inline void scan_sums_body(int *block_sums, int nb, int *sh) {
    int carry = 0;
    for (int base = 0; base < nb; base += kScanTile) {
        int v[kScanItems];
        const int b0 = base + threadIdx.x * kScanItems;
#pragma unroll
        for (int q = 0; q < kScanItems; ++q) v[q] = b0 + q < nb ? block_sums[b0 + q] : 0;
        const int total = block_scan(v, sh);
#pragma unroll
        for (int q = 0; q < kScanItems; ++q)
            if (b0 + q < nb) block_sums[b0 + q] = v[q] + carry;
        carry += total;
    }
}

// Add block offsets; copy to the cursors (counts array); extract tile offsets.
__device__ inline void scan_finish_body(const SortArgs &a, long long nkeys, int b, int nb) {
    for (long long i = (long long)b * blockDim.x + threadIdx.x; i < nkeys; i += (long long)nb * blockDim.x) {
        int v = a.offsets[i] + a.block_sums[i / kScanTile];
        if (v < 0 || v > a.n) {   // counts inconsistent with the particles: flag, keep offsets in range
            atomicOr(a.err, ERR_SORT);
            v = v < 0 ? 0 : (int)a.n;
        }
        a.offsets[i] = v;
        a.counts[i] = v;
        if (i % a.t.cells_per_tile == 0) a.tile_start[i / a.t.cells_per_tile] = v;
    }
    if (b == 0 && threadIdx.x == 0) a.tile_start[a.t.ntiles] = (int)a.n;
}

// Rank pass: the destination slot of every source particle, written as the
// inverse permutation perm[slot] = source index (4-byte scattered writes only).
template <int NDIM>
__device__ inline void rank_body(const SortArgs &a, const SrcWalk &w, long long nkeys) {
    long long i, end;
    int t0s, nts;
    w.begin(i, end, t0s, nts);
    const int lane = threadIdx.x & 31;
    for (long long ib = i - lane; ib < end; ib += 4 * w.step()) {   // warp-uniform loop
        long long p[4];
        int key[4];
        walk_keys<NDIM>(a, w, ib + lane, end, t0s, nts, nkeys, p, key);
        int base[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            // lanes that share a key take consecutive slots with one atomic
            const unsigned peers = __match_any_sync(0xffffffffu, key[v]);
            const int leader = __ffs(peers) - 1;
            int b = 0;
            if (key[v] >= 0 && lane == leader) b = atomicAdd(a.counts + key[v], __popc(peers));
            base[v] = __shfl_sync(0xffffffffu, b, leader) + __popc(peers & ((1u << lane) - 1u));
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            if (key[v] < 0) continue;
            const int tile = key_tile(a.t, key[v]);
            const int t0 = __ldg(a.tile_start + tile), t1 = __ldg(a.tile_start + tile + 1);
            const long long dst = (long long)t0 + interleaved_slot(base[v] - t0, t1 - t0);
            if (base[v] >= t0 && base[v] < t1 && dst < a.n) a.perm[dst] = (int)p[v];
            else atomicOr(a.err, ERR_SORT);   // counts inconsistent with the particles
        }
    }
}

// Gather pass in destination order.  One CTA per chunk of kGatherChunk
// destination slots, one particle array at a time: the sources of a chunk lie
// in the same tile of the previous layout (plus the few particles that changed
// tile), so while the resident CTAs work on one array the source regions they
// read stay in L2 and every source sector comes from DRAM about once.  (A
// grid-stride loop over the whole array spreads the resident threads over all
// of it and fetches each 32-byte sector many times for its 4 used bytes.)
constexpr int kGatherThreads = 256;
constexpr int kGatherChunk = 4096;

template <int NDIM>
__device__ inline void gather_body(const SpeciesMixed &src, const SpeciesMixed &dst, long long n, const int *perm,
                                   int b) {
    constexpr int NA = NDIM + 5;   // cell, offsets, 3 momenta, id
    const long long q0 = (long long)b * kGatherChunk;
    const long long q1 = q0 + kGatherChunk < n ? q0 + kGatherChunk : n;
#pragma unroll 1
    for (int a = 0; a < NA; ++a) {
        const uint32_t *sa;
        uint32_t *da;
        if (a == 0) { sa = src.cell; da = dst.cell; }
        else if (a <= NDIM) { sa = reinterpret_cast<const uint32_t *>(src.off[a - 1]);
                              da = reinterpret_cast<uint32_t *>(dst.off[a - 1]); }
        else if (a < NA - 1) { sa = reinterpret_cast<const uint32_t *>(src.u[a - 1 - NDIM]);
                               da = reinterpret_cast<uint32_t *>(dst.u[a - 1 - NDIM]); }
        else { sa = reinterpret_cast<const uint32_t *>(src.id); da = reinterpret_cast<uint32_t *>(dst.id); }
        // four independent loads in flight per thread
        for (long long q = q0 + threadIdx.x; q < q1; q += 4 * kGatherThreads) {
            int p[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const long long qq = q + v * kGatherThreads;
                p[v] = qq < q1 ? __ldg(perm + qq) : -1;
            }
            uint32_t x[4];
            // an out-of-range entry exists only after a bad key, which the sort has flagged
#pragma unroll
            for (int v = 0; v < 4; ++v) x[v] = (p[v] >= 0 && p[v] < n) ? __ldg(sa + p[v]) : 0u;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const long long qq = q + v * kGatherThreads;
                if (qq < q1) da[qq] = x[v];
            }
        }
    }
}

// ---- block counts of the phases of one sort ----

inline int blocks_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    const long long cap = 152LL * 32;
    return (int)(b < 1 ? 1 : (b < cap ? b : cap));
}
__host__ __device__ inline long long nkeys_of(const SortArgs &a) { return (long long)a.t.ntiles * a.t.cells_per_tile; }
constexpr int kWalkThreads = 512;
inline int walk_blocks(const SortArgs &a) { return a.old_tile_start ? a.t.ntiles : blocks_for(a.n, kWalkThreads); }
__host__ __device__ inline int scan_blocks(const SortArgs &a) { return (int)((nkeys_of(a) + kScanTile - 1) / kScanTile); }
inline int key_blocks(const SortArgs &a) { return blocks_for(nkeys_of(a), 256); }
inline int gather_blocks(const SortArgs &a) { return (int)((a.n + kGatherChunk - 1) / kGatherChunk); }

// ---- one sort: one launch per phase ----

__global__ void k_zero(SortArgs a) { zero_body(a.counts, nkeys_of(a), blockIdx.x, gridDim.x); }

template <int NDIM>
__global__ void k_histogram(SortArgs a) {
    const SrcWalk w{a.old_tile_start, a.n, (int)blockIdx.x, (int)gridDim.x};
    histogram_body<NDIM>(a, w, nkeys_of(a));
}

__global__ void __launch_bounds__(kScanThreads) k_scan_blocks(SortArgs a) {
    __shared__ int sh[33];
    scan_blocks_body(a.counts, a.offsets, a.block_sums, nkeys_of(a), blockIdx.x, sh);
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sums(SortArgs a) {
    __shared__ int sh[33];
    scan_sums_body(a.block_sums, scan_blocks(a), sh);
}

__global__ void k_scan_finish(SortArgs a) { scan_finish_body(a, nkeys_of(a), blockIdx.x, gridDim.x); }

template <int NDIM>
__global__ void k_rank(SortArgs a) {
    const SrcWalk w{a.old_tile_start, a.n, (int)blockIdx.x, (int)gridDim.x};
    rank_body<NDIM>(a, w, nkeys_of(a));
}

template <int NDIM>
__global__ void __launch_bounds__(kGatherThreads) k_gather(SortArgs a) {
    gather_body<NDIM>(a.src, a.dst, a.n, a.perm, blockIdx.x);
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
    histogram_body<NDIM>(a, w, nkeys_of(a));
}

__global__ void __launch_bounds__(kScanThreads) k_scan_blocks_multi(const SortArgs *as, const int *prefix,
                                                                    int nsort) {
    __shared__ int sh[33];
    const int s = find_sort(prefix, nsort, blockIdx.x);
    const SortArgs &a = as[s];
    scan_blocks_body(a.counts, a.offsets, a.block_sums, nkeys_of(a), blockIdx.x - prefix[s], sh);
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sums_multi(const SortArgs *as) {
    __shared__ int sh[33];
    const SortArgs &a = as[blockIdx.x];
    scan_sums_body(a.block_sums, scan_blocks(a), sh);
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
    rank_body<NDIM>(a, w, nkeys_of(a));
}

template <int NDIM>
__global__ void __launch_bounds__(kGatherThreads) k_gather_multi(const SortArgs *as, const int *prefix, int nsort) {
    const int s = find_sort(prefix, nsort, blockIdx.x);
    const SortArgs &a = as[s];
    gather_body<NDIM>(a.src, a.dst, a.n, a.perm, blockIdx.x - prefix[s]);
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
