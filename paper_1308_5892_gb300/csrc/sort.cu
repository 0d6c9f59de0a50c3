// sort.cu -- counting sort of the mixed-path particles by tile-major cell key.
//
// key(cell) = tile_index * cells_per_tile + index of the cell inside its tile,
// so particles end up grouped by tile and, inside a tile, by cell; the cell
// order inside a tile is then stored block-transposed (interleaved_slot).  The sort
// is out of place (src -> dst, the caller swaps the buffers): histogram of the
// keys, exclusive scan, a rank pass whose per-key cursors are advanced with
// warp-aggregated atomics (lanes of a warp that share a key take consecutive
// slots with one atomic) and which writes only the 4-byte inverse permutation,
// then a gather pass that writes every particle array in destination order
// (coalesced stores; scattered partial-sector stores of the full particle
// state cost several times its size in DRAM traffic).  The tile offsets are
// read from the scanned counts.
//
// Roofline: HBM bound; per particle 4 B (histogram) + 8 B (rank) +
// 4 + 2 x (24..28 + 4) B (gather) plus per key 3 x 4 B.
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
    const int ti = i / t.T[0], tj = j / t.T[1], tk = NDIM == 3 ? k / t.T[2] : 0;
    const int li = i - ti * t.T[0], lj = j - tj * t.T[1], lk = NDIM == 3 ? k - tk * t.T[2] : 0;
    const int tile = (tk * t.ntile[1] + tj) * t.ntile[0] + ti;
    return tile * t.cells_per_tile + (lk * t.T[1] + lj) * t.T[0] + li;
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
    __device__ __forceinline__ bool begin(long long &i, long long &end, int &t0, int &nt) const {
        if (old_start) {
            t0 = old_start[blockIdx.x];
            nt = old_start[blockIdx.x + 1] - t0;
            i = threadIdx.x;
            end = nt;
        } else {
            t0 = 0;
            nt = 0;
            i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
            end = n;
        }
        return true;
    }
    __device__ __forceinline__ long long step() const {
        return old_start ? (long long)blockDim.x : (long long)gridDim.x * blockDim.x;
    }
    __device__ __forceinline__ long long pos(long long i, int t0, int nt) const {
        return old_start ? (long long)t0 + interleaved_slot((int)i, nt) : i;
    }
};

__global__ void k_zero(int *a, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a[i] = 0;
}

template <int NDIM>
__global__ void k_histogram(TileGeom t, const uint32_t *cell, SrcWalk w, int *counts, long long nkeys, int *err) {
    long long i, end;
    int t0, nt;
    w.begin(i, end, t0, nt);
    for (; i < end; i += w.step()) {
        const long long p = w.pos(i, t0, nt);
        const int key = cell_key<NDIM>(t, cell[p]);
        if (key < 0 || key >= nkeys) { atomicOr(err, ERR_SORT); continue; }
        // warp aggregation: lanes with the same key add once
        const unsigned act = __activemask();
        const unsigned peers = __match_any_sync(act, key);
        const int leader = __ffs(peers) - 1;
        if ((int)(threadIdx.x & 31) == leader) atomicAdd(counts + key, __popc(peers));
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

__global__ void __launch_bounds__(kScanThreads) k_scan_blocks(const int *in, int *out, int *block_sums, long long n) {
    __shared__ int sh[33];
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    int v[kScanItems];
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) v[q] = base + q < n ? in[base + q] : 0;
    const int total = block_scan(v, sh);
#pragma unroll
    for (int q = 0; q < kScanItems; ++q)
        if (base + q < n) out[base + q] = v[q];
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// Exclusive scan of the block sums in one block (any count, in chunks).
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(int *block_sums, int nb) {
    __shared__ int sh[33];
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

// Add block offsets; copy to cursors; extract tile offsets.
__global__ void k_scan_finish(int *offsets, int *cursors, const int *block_sums, long long nkeys, int cells_per_tile,
                              int ntiles, int *tile_start, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nkeys;
         i += (long long)gridDim.x * blockDim.x) {
        const int v = offsets[i] + block_sums[i / kScanTile];
        offsets[i] = v;
        cursors[i] = v;
        if (i % cells_per_tile == 0) tile_start[i / cells_per_tile] = v;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) tile_start[ntiles] = (int)n;
}

// Rank pass: the destination slot of every source particle, written as the
// inverse permutation perm[slot] = source index (4-byte scattered writes only).
template <int NDIM>
__global__ void k_rank(TileGeom t, const uint32_t *cell, SrcWalk w, int *cursors, long long nkeys,
                       const int *tile_start, int *perm) {
    long long i, end;
    int t0s, nts;
    w.begin(i, end, t0s, nts);
    for (; i < end; i += w.step()) {
        const long long p = w.pos(i, t0s, nts);
        const int key = cell_key<NDIM>(t, cell[p]);
        if (key < 0 || key >= nkeys) continue;
        const unsigned act = __activemask();
        const unsigned peers = __match_any_sync(act, key);
        const int lane = threadIdx.x & 31;
        const int leader = __ffs(peers) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(cursors + key, __popc(peers));
        base = __shfl_sync(peers, base, leader);
        const int rank = base + __popc(peers & ((1u << lane) - 1u));
        const int tile = key / t.cells_per_tile;
        const int t0 = tile_start[tile], t1 = tile_start[tile + 1];
        perm[t0 + interleaved_slot(rank - t0, t1 - t0)] = (int)p;
    }
}

// Gather pass in destination order: coalesced writes, reads through L2.
template <int NDIM>
__global__ void k_gather(SpeciesMixed src, SpeciesMixed dst, long long n, const int *perm) {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int p = perm[q];
        dst.cell[q] = __ldg(src.cell + p);
        dst.off[0][q] = __ldg(src.off[0] + p);
        dst.off[1][q] = __ldg(src.off[1] + p);
        if (NDIM == 3) dst.off[2][q] = __ldg(src.off[2] + p);
        dst.u[0][q] = __ldg(src.u[0] + p);
        dst.u[1][q] = __ldg(src.u[1] + p);
        dst.u[2][q] = __ldg(src.u[2] + p);
        dst.id[q] = __ldg(src.id + p);
    }
}

inline int blocks_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    const long long cap = 152LL * 32;
    return (int)(b < 1 ? 1 : (b < cap ? b : cap));
}

}  // namespace

size_t sort_scan_scratch(long long nkeys) { return (size_t)((nkeys + kScanTile - 1) / kScanTile + 1); }

void launch_sort(const SortArgs &a, cudaStream_t s) {
    const long long nkeys = (long long)a.t.ntiles * a.t.cells_per_tile;
    SrcWalk w;
    w.old_start = a.old_tile_start;
    w.n = a.n;
    const int wblocks = a.old_tile_start ? a.t.ntiles : blocks_for(a.n, 256);
    k_zero<<<blocks_for(nkeys, 256), 256, 0, s>>>(a.counts, nkeys);
    if (a.n > 0) {
        if (a.g.ndim == 3) k_histogram<3><<<wblocks, 256, 0, s>>>(a.t, a.src.cell, w, a.counts, nkeys, a.err);
        else k_histogram<2><<<wblocks, 256, 0, s>>>(a.t, a.src.cell, w, a.counts, nkeys, a.err);
    }
    const int nb = (int)((nkeys + kScanTile - 1) / kScanTile);
    k_scan_blocks<<<nb, kScanThreads, 0, s>>>(a.counts, a.offsets, a.block_sums, nkeys);
    k_scan_sums<<<1, kScanThreads, 0, s>>>(a.block_sums, nb);
    k_scan_finish<<<blocks_for(nkeys, 256), 256, 0, s>>>(a.offsets, a.counts, a.block_sums, nkeys,
                                                         a.t.cells_per_tile, a.t.ntiles, a.tile_start, a.n);
    if (a.n > 0) {
        if (a.g.ndim == 3) {
            k_rank<3><<<wblocks, 256, 0, s>>>(a.t, a.src.cell, w, a.counts, nkeys, a.tile_start, a.perm);
            k_gather<3><<<blocks_for(a.n, 256), 256, 0, s>>>(a.src, a.dst, a.n, a.perm);
        } else {
            k_rank<2><<<wblocks, 256, 0, s>>>(a.t, a.src.cell, w, a.counts, nkeys, a.tile_start, a.perm);
            k_gather<2><<<blocks_for(a.n, 256), 256, 0, s>>>(a.src, a.dst, a.n, a.perm);
        }
    }
}

}  // namespace pic
