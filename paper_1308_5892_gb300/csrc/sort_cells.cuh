// sort_cells.cuh -- phase bodies of the counting sort of the mixed-path
// particles (see sort.cu): key histogram, block scans, rank pass and gather,
// each written for block b of nb blocks of one sort.  Shared by the sort
// kernels (sort.cu) and the persistent ensemble step (walk.cu).
#pragma once
#include "pic_internal.cuh"

namespace pic {

namespace {

constexpr int kScanTile = 4096;      // keys per scan block
constexpr int kScanThreads = 1024;   // threads of the scan kernels (4 keys each)

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
// With a tiled source, block b takes part b % parts of old tile b / parts (its
// share of the tile's ranks, in order).
struct SrcWalk {
    const int *old_start;   // old tile offsets, or nullptr when the source is untiled
    long long n;
    int b, nb;              // this block and the block count of the walk
    int parts = 1;          // blocks per old tile
    __device__ __forceinline__ void begin(long long &i, long long &end, int &t0, int &nt) const {
        if (old_start) {
            const int tile = b / parts, part = b - tile * parts;
            t0 = ldro(old_start + tile);
            nt = ldro(old_start + tile + 1) - t0;
            i = (long long)nt * part / parts + threadIdx.x;
            end = (long long)nt * (part + 1) / parts;
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

// Keys of the V source elements i + v * step (v = 0..V-1) of a walk, -1 past its end.
template <int NDIM, int V>
__device__ __forceinline__ void walk_keys(const SortArgs &a, const SrcWalk &w, long long i, long long end, int t0,
                                          int nt, long long nkeys, long long (&p)[V], int (&key)[V]) {
    uint32_t c[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const long long iv = i + v * w.step();
        p[v] = iv < end ? w.pos(iv, t0, nt) : -1;
        c[v] = p[v] >= 0 ? ldro(a.src.cell + p[v]) : 0u;
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
        key[v] = p[v] >= 0 ? cell_key<NDIM>(a.t, c[v]) : -1;
        if (p[v] >= 0 && (key[v] < 0 || key[v] >= nkeys)) {
            atomicOr(a.err, ERR_SORT);
            key[v] = -1;
        }
    }
}

// V elements per thread and iteration (independent loads in flight).
template <int NDIM, int V>
__device__ inline void histogram_body(const SortArgs &a, const SrcWalk &w, long long nkeys) {
    long long i, end;
    int t0, nt;
    w.begin(i, end, t0, nt);
    // the loop is warp-uniform (every lane takes part in the warp aggregation)
    const int lane = threadIdx.x & 31;
    for (long long ib = i - lane; ib < end; ib += V * w.step()) {
        long long p[V];
        int key[V];
        walk_keys<NDIM, V>(a, w, ib + lane, end, t0, nt, nkeys, p, key);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            // warp aggregation: lanes with the same key add once
            const unsigned peers = __match_any_sync(0xffffffffu, key[v]);
            const int leader = __ffs(peers) - 1;
            if (key[v] >= 0 && (int)(threadIdx.x & 31) == leader) atomicAdd(a.counts + key[v], __popc(peers));
        }
    }
}

// Block-level exclusive scan of kScanTile ints held THREADS x (kScanTile /
// THREADS) in registers (sh: 33 ints); returns the block total.
template <int THREADS>
__device__ inline int block_scan(int (&v)[kScanTile / THREADS], int *sh) {
    constexpr int kScanItems = kScanTile / THREADS;
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
        int w = lane < (THREADS / 32) ? sh[lane] : 0;
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
template <int THREADS>
__device__ inline void scan_blocks_body(const int *in, int *out, int *block_sums, long long n, int b, int *sh) {
    constexpr int kScanItems = kScanTile / THREADS;
    const long long base = (long long)b * kScanTile + (long long)threadIdx.x * kScanItems;
    int v[kScanItems];
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) v[q] = base + q < n ? in[base + q] : 0;
    const int total = block_scan<THREADS>(v, sh);
#pragma unroll
    for (int q = 0; q < kScanItems; ++q)
        if (base + q < n) out[base + q] = v[q];
    if (threadIdx.x == 0) block_sums[b] = total;
}

// Exclusive scan of the block sums in one block (any count, in chunks).
template <int THREADS>
__device__ inline void scan_sums_body(int *block_sums, int nb, int *sh) {
    constexpr int kScanItems = kScanTile / THREADS;
    int carry = 0;
    for (int base = 0; base < nb; base += kScanTile) {
        int v[kScanItems];
        const int b0 = base + threadIdx.x * kScanItems;
#pragma unroll
        for (int q = 0; q < kScanItems; ++q) v[q] = b0 + q < nb ? block_sums[b0 + q] : 0;
        const int total = block_scan<THREADS>(v, sh);
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
// V elements per thread and iteration; their cursor atomics are all issued
// before the first result is used, so they are in flight together.
template <int NDIM, int V>
__device__ inline void rank_body(const SortArgs &a, const SrcWalk &w, long long nkeys) {
    long long i, end;
    int t0s, nts;
    w.begin(i, end, t0s, nts);
    const int lane = threadIdx.x & 31;
    for (long long ib = i - lane; ib < end; ib += V * w.step()) {   // warp-uniform loop
        long long p[V];
        int key[V];
        walk_keys<NDIM, V>(a, w, ib + lane, end, t0s, nts, nkeys, p, key);
        unsigned peers[V];
        int leader[V], b[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            // lanes that share a key take consecutive slots with one atomic
            peers[v] = __match_any_sync(0xffffffffu, key[v]);
            leader[v] = __ffs(peers[v]) - 1;
            b[v] = 0;
            if (key[v] >= 0 && lane == leader[v]) b[v] = atomicAdd(a.counts + key[v], __popc(peers[v]));
        }
        int base[V];
#pragma unroll
        for (int v = 0; v < V; ++v)
            base[v] = __shfl_sync(0xffffffffu, b[v], leader[v]) + __popc(peers[v] & ((1u << lane) - 1u));
#pragma unroll
        for (int v = 0; v < V; ++v) {
            if (key[v] < 0) continue;
            const int tile = key_tile(a.t, key[v]);
            const int t0 = ldro(a.tile_start + tile), t1 = ldro(a.tile_start + tile + 1);
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
// THREADS threads, LOADS independent loads in flight per thread.
constexpr int kGatherThreads = 256;
constexpr int kGatherChunk = 4096;

template <int NDIM, int THREADS, int LOADS>
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
        for (long long q = q0 + threadIdx.x; q < q1; q += LOADS * THREADS) {
            int p[LOADS];
#pragma unroll
            for (int v = 0; v < LOADS; ++v) {
                const long long qq = q + v * THREADS;
                p[v] = qq < q1 ? ldro(perm + qq) : -1;
            }
            uint32_t x[LOADS];
            // an out-of-range entry exists only after a bad key, which the sort has flagged
#pragma unroll
            for (int v = 0; v < LOADS; ++v) x[v] = (p[v] >= 0 && p[v] < n) ? ldro(sa + p[v]) : 0u;
#pragma unroll
            for (int v = 0; v < LOADS; ++v) {
                const long long qq = q + v * THREADS;
                if (qq < q1) da[qq] = x[v];
            }
        }
    }
}

// Gather of one chunk with every array per read of the permutation: LOADS
// slots per thread, all NDIM + 5 arrays loaded before any is stored (more
// independent loads in flight for a block that runs at few warps per SM).
template <int NDIM, int THREADS, int LOADS>
__device__ inline void gather_all_body(const SpeciesMixed &src, const SpeciesMixed &dst, long long n, const int *perm,
                                       int b) {
    constexpr int NA = NDIM + 5;   // cell, offsets, 3 momenta, id
    const uint32_t *sa[NA];
    uint32_t *da[NA];
    sa[0] = src.cell; da[0] = dst.cell;
#pragma unroll
    for (int a = 0; a < NDIM; ++a) {
        sa[1 + a] = reinterpret_cast<const uint32_t *>(src.off[a]);
        da[1 + a] = reinterpret_cast<uint32_t *>(dst.off[a]);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        sa[1 + NDIM + a] = reinterpret_cast<const uint32_t *>(src.u[a]);
        da[1 + NDIM + a] = reinterpret_cast<uint32_t *>(dst.u[a]);
    }
    sa[NA - 1] = reinterpret_cast<const uint32_t *>(src.id);
    da[NA - 1] = reinterpret_cast<uint32_t *>(dst.id);
    const long long q0 = (long long)b * kGatherChunk;
    const long long q1 = q0 + kGatherChunk < n ? q0 + kGatherChunk : n;
    for (long long q = q0 + threadIdx.x; q < q1; q += LOADS * THREADS) {
        int p[LOADS];
#pragma unroll
        for (int v = 0; v < LOADS; ++v) {
            const long long qq = q + v * THREADS;
            p[v] = qq < q1 ? ldro(perm + qq) : -1;
        }
        uint32_t x[NA][LOADS];
        // an out-of-range entry exists only after a bad key, which the sort has flagged
#pragma unroll
        for (int a = 0; a < NA; ++a)
#pragma unroll
            for (int v = 0; v < LOADS; ++v) x[a][v] = (p[v] >= 0 && p[v] < n) ? ldro(sa[a] + p[v]) : 0u;
#pragma unroll
        for (int a = 0; a < NA; ++a)
#pragma unroll
            for (int v = 0; v < LOADS; ++v) {
                const long long qq = q + v * THREADS;
                if (qq < q1) da[a][qq] = x[a][v];
            }
    }
}

// Keys and scan blocks of one sort.
__host__ __device__ inline long long nkeys_of(const SortArgs &a) { return (long long)a.t.ntiles * a.t.cells_per_tile; }
__host__ __device__ inline int scan_blocks(const SortArgs &a) { return (int)((nkeys_of(a) + kScanTile - 1) / kScanTile); }

}  // namespace

}  // namespace pic
