// push_mixed.cu -- the mixed-precision tile kernel: gather, Boris push, move and
// charge-conserving deposit (main loop steps 2, 3, 8, 9 of App. A.3.1) for
// all species of one tile of cells per CTA.
//
// Data (per tile of T cells with a halo of H cells on every side, R = T + 2H):
//  - node fields E, B at time t (App. A.3.3 averages, computed once per step
//    by the field kernels) for the R^d nodes of the tile + halo are staged in
//    shared memory as one float4 {E_x,E_y,E_z,B_x} and one float2 {B_y,B_z}
//    per node; particles are sorted by cell inside the tile, so the lanes of a
//    warp mostly read the same node (broadcast);
//  - the current of the tile + halo is accumulated in shared memory in exact
//    fixed point: each flux v (units of the particle volume times sgn q) is
//    rounded to a multiple of 2^-36 and split into two int32 limbs, v*2^18
//    rounded (hi) and the remainder times 2^18 rounded (lo), added with
//    integer atomics.  GB300 resolves same-address integer atomics of a warp
//    at full rate, whereas FP32 shared atomics serialise on conflicts (which
//    cell-sorted lanes cause on every deposit).  Integer sums are exact and
//    associative, so the current is independent of the order of the
//    particles; at the end hi*2^18 + lo is added once per node to the global
//    int64 current;
//  - particles (packed cell, FP32 offsets, FP32 momenta) are streamed once:
//    read 24 B (2D) / 28 B (3D) and write the same.
// A particle whose stencil leaves the staged box (it drifted far since the
// last sort) takes a slow path that gathers from global memory and deposits
// with global int64 atomics of the same fixed-point values, so the result
// never depends on the sort interval.
//
// Roofline: HBM bound.  Algorithmic bytes per particle-step = 2 x 24 B (2D) or
// 2 x 28 B (3D); field and current traffic per cell is amortised over the
// particles per cell.
#include <algorithm>

#include "particle_core.cuh"
#include "pic_internal.cuh"

namespace pic {

namespace {

constexpr float kFx1 = 262144.0f;   // 2^18: scale of the hi limb and of the lo remainder

// Shared-memory current sink, two int32 fixed-point limbs per value.
struct SmemSinkFx {
    int *hi, *lo;
    int sx, sxy, nodes;
    int base0, base;
    __device__ __forceinline__ void set_cell(int di, int dj, int dk) { base = base0 + di + dj * sx + dk * sxy; }
    __device__ __forceinline__ void operator()(int comp, int di, int dj, int dk, float v) {
        const int q = comp * nodes + base + di + dj * sx + dk * sxy;
        const float x = v * kFx1;
        const float h = rintf(x);
        atomicAdd(hi + q, (int)h);
        atomicAdd(lo + q, __float2int_rn((x - h) * kFx1));
    }
};

// Global current sink for particles outside the staged box: the same
// fixed-point value, added as one int64 at the interior-wrapped padded index.
struct GlobalSinkFx {
    const Geom *g;
    unsigned long long *J[3];
    int ci, cj, ck, oi, oj, ok;
    __device__ void set_cell(int di, int dj, int dk) { oi = ci + di; oj = cj + dj; ok = ck + dk; }
    __device__ void operator()(int comp, int di, int dj, int dk, float v) {
        const float x = v * kFx1;
        const float h = rintf(x);
        const long long f = (long long)h * 262144LL + (long long)__float2int_rn((x - h) * kFx1);
        atomicAdd(J[comp] + g->widx(oi + di, oj + dj, ok + dk), (unsigned long long)f);
    }
};

// Slow path of a particle outside the staged box: deposit with global atomics.
template <int NDIM>
__device__ __noinline__ void deposit_global(const Geom &g, unsigned long long *J0, unsigned long long *J1,
                                            unsigned long long *J2, int ci, int cj, int ck, const float d[3],
                                            const int s[3], const float d1[3], float dz, float sgn) {
    GlobalSinkFx gs;
    gs.g = &g;
    gs.J[0] = J0; gs.J[1] = J1; gs.J[2] = J2;
    gs.ci = ci; gs.cj = cj; gs.ck = ck;
    PieceDeposit<NDIM, float, GlobalSinkFx> pd(gs);
    deposit_path<NDIM, float>(d, s, d1, dz, sgn, pd);
}

template <int NDIM>
__device__ __forceinline__ void gather_nodes(const float4 *nA, const float2 *nB, int q0, int sx, int sxy,
                                             const float d[3], float E[3], float B[3]) {
    E[0] = E[1] = E[2] = B[0] = B[1] = B[2] = 0.f;
#pragma unroll
    for (int xi = 0; xi < (NDIM == 3 ? 2 : 1); ++xi)
#pragma unroll
        for (int eta = 0; eta < 2; ++eta)
#pragma unroll
            for (int eps = 0; eps < 2; ++eps) {
                float w = (eps ? d[0] : 1.f - d[0]) * (eta ? d[1] : 1.f - d[1]);
                if (NDIM == 3) w *= (xi ? d[2] : 1.f - d[2]);
                const int q = q0 + eps + eta * sx + xi * sxy;
                const float4 a = nA[q];
                const float2 b = nB[q];
                E[0] += w * a.x; E[1] += w * a.y; E[2] += w * a.z;
                B[0] += w * a.w; B[1] += w * b.x; B[2] += w * b.y;
            }
}

template <int NDIM>
__device__ __noinline__ void gather_global(const Geom &g, const float4 *nA, const float2 *nB, int ci, int cj, int ck,
                                     const float d[3], float E[3], float B[3]) {
    E[0] = E[1] = E[2] = B[0] = B[1] = B[2] = 0.f;
#pragma unroll
    for (int xi = 0; xi < (NDIM == 3 ? 2 : 1); ++xi)
#pragma unroll
        for (int eta = 0; eta < 2; ++eta)
#pragma unroll
            for (int eps = 0; eps < 2; ++eps) {
                float w = (eps ? d[0] : 1.f - d[0]) * (eta ? d[1] : 1.f - d[1]);
                if (NDIM == 3) w *= (xi ? d[2] : 1.f - d[2]);
                const long long q = g.widx(ci + eps, cj + eta, ck + xi);
                const float4 a = __ldg(nA + q);
                const float2 b = __ldg(nB + q);
                E[0] += w * a.x; E[1] += w * a.y; E[2] += w * a.z;
                B[0] += w * a.w; B[1] += w * b.x; B[2] += w * b.y;
            }
}

// Kahan-compensated FP32 running sum (per thread).
struct KahanF {
    float s = 0.f, c = 0.f;
    __device__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// First-segment currents of consecutive particles of one thread that start in
// the same cell, accumulated exactly in registers (the same two fixed-point
// limbs as the shared-memory sink) and added to shared memory once per cell.
// Value index: 3D comp 0 (dj + 2dk), comp 1 4 + (di + 2dk), comp 2 8 + (di + 2dj);
// 2D comp 0 dj, comp 1 2 + di, comp 2 4 + (di + 2dj).
template <int NDIM>
struct RegAcc {
    static constexpr int NV = NDIM == 3 ? 12 : 8;
    int hi[NV], lo[NV];
    int q0;   // local node index of the accumulation cell, -1 when empty
    __device__ __forceinline__ void reset(int q) {
#pragma unroll
        for (int v = 0; v < NV; ++v) { hi[v] = 0; lo[v] = 0; }
        q0 = q;
    }
    __device__ __forceinline__ static int index(int comp, int di, int dj, int dk) {
        if (NDIM == 3) return comp == 0 ? dj + 2 * dk : (comp == 1 ? 4 + di + 2 * dk : 8 + di + 2 * dj);
        return comp == 0 ? dj : (comp == 1 ? 2 + di : 4 + di + 2 * dj);
    }
    __device__ __forceinline__ void flush(int *Jhi, int *Jlo, int nodes, int sx, int sxy) {
        if (q0 < 0) return;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            int comp, di = 0, dj = 0, dk = 0;
            if (NDIM == 3) {
                comp = v / 4;
                const int r = v % 4;
                if (comp == 0) { dj = r & 1; dk = r >> 1; }
                else if (comp == 1) { di = r & 1; dk = r >> 1; }
                else { di = r & 1; dj = r >> 1; }
            } else {
                if (v < 2) { comp = 0; dj = v; }
                else if (v < 4) { comp = 1; di = v - 2; }
                else { comp = 2; di = (v - 4) & 1; dj = (v - 4) >> 1; }
            }
            const int q = comp * nodes + q0 + di + dj * sx + dk * sxy;
            atomicAdd(Jhi + q, hi[v]);
            atomicAdd(Jlo + q, lo[v]);
        }
        q0 = -1;
    }
};

// Per-warp ring buffer of path pieces waiting to be deposited (128 entries):
// local node index of the piece's cell, start offset and displacement.
constexpr int kQueue = 128;
struct PieceQueue {
    int *base;      // [kQueue]
    float *d;       // [3][kQueue]
    float *D;       // [3][kQueue]
    int *count;     // pieces waiting (shared, per warp)
};

// Piece sink of the fast path: the piece in the start cell goes to the
// register accumulator; pieces in the neighbour cells (after a node-plane
// crossing) are appended to the warp's queue, so that they are deposited
// later by all 32 lanes together instead of by the few crossing lanes.
template <int NDIM>
struct QueueSink {
    RegAcc<NDIM> *acc;
    PieceQueue q;
    int qhead;      // warp-uniform ring position of the oldest waiting piece
    int q0, sx, sxy;
    __device__ __forceinline__ void set_cell(int, int, int) {}
    // value sink used for the start-cell piece
    __device__ __forceinline__ void operator()(int comp, int di, int dj, int dk, float v) {
        const float x = v * kFx1;
        const float h = rintf(x);
        const int k = RegAcc<NDIM>::index(comp, di, dj, dk);
        acc->hi[k] += (int)h;
        acc->lo[k] += __float2int_rn((x - h) * kFx1);
    }
    __device__ __forceinline__ void piece(int k, int di, int dj, int dk, const float d[3], const float D[3],
                                          float alpha) {
        if (k == 0) {
            deposit_segment<NDIM, float>(d, D, alpha, *this);
            return;
        }
        // lanes appending together reserve consecutive slots with one atomic
        const unsigned mask = __activemask();
        const int lane = threadIdx.x & 31;
        const int leader = __ffs(mask) - 1;
        int start = 0;
        if (lane == leader) start = atomicAdd(q.count, __popc(mask));
        start = __shfl_sync(mask, start, leader);
        const int idx = (qhead + start + __popc(mask & ((1u << lane) - 1u))) & (kQueue - 1);
        q.base[idx] = q0 + di + dj * sx + dk * sxy;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            q.d[a * kQueue + idx] = d[a];
            q.D[a * kQueue + idx] = D[a];
        }
    }
};

// Per-CTA constants of the tile.
struct TileCtx {
    int x0, y0, z0, Rx, Ry, Rz, sx, sxy, nodes, H, T0, T1, T2;
    const float4 *nA;
    const float2 *nB;
    int *Jhi, *Jlo;
};

// One particle: gather, Boris, move, deposit.  c/d/u are updated in place.
// With ACC the start-cell piece of the path goes to the register accumulator.
template <int NDIM>
__device__ __forceinline__ void push_one(const MixedStepArgs &a, const TileCtx &tc, QueueSink<NDIM> &qs, float h,
                                         float sgn, uint32_t &cell, float d[3], float u[3], KahanF &k0,
                                         KahanF &k1) {
    RegAcc<NDIM> &acc = *qs.acc;
    const Geom &g = a.g;
    int ci, cj, ck;
    unpack_cell(NDIM, cell, ci, cj, ck);
    // local cell in the staged box, nearest periodic image of the tile
    int lx = ci - tc.x0, ly = cj - tc.y0, lz = NDIM == 3 ? ck - tc.z0 : 0;
    if (lx >= tc.T0 + tc.H) lx -= g.nx; else if (lx < -tc.H) lx += g.nx;
    if (ly >= tc.T1 + tc.H) ly -= g.ny; else if (ly < -tc.H) ly += g.ny;
    if (NDIM == 3) { if (lz >= tc.T2 + tc.H) lz -= g.nz; else if (lz < -tc.H) lz += g.nz; }
    lx += tc.H; ly += tc.H; lz += NDIM == 3 ? tc.H : 0;
    // fast path: the gather reads nodes l..l+1 and the deposit writes nodes
    // l-1..l+2 of the staged box, all of which must also lie in the padded grid
    bool fast = lx >= 1 && lx <= tc.Rx - 3 && ly >= 1 && ly <= tc.Ry - 3 && tc.x0 + lx + 2 < g.px &&
                tc.y0 + ly + 2 < g.py;
    if (NDIM == 3) fast = fast && lz >= 1 && lz <= tc.Rz - 3 && tc.z0 + lz + 2 < g.pz;
    const int q0 = lx + ly * tc.sx + lz * tc.sxy;
    float E[3], B[3];
    if (fast) gather_nodes<NDIM>(tc.nA, tc.nB, q0, tc.sx, tc.sxy, d, E, B);
    else gather_global<NDIM>(g, a.nfA, a.nfB, ci, cj, ck, d, E, B);
    const float u2_0 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const float dt = a.dt;
    boris<float>(u, E, B, h, dt);
    const float u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const float inv_gam = rsqrtf(1.f + u2);
    // gamma - 1 = u^2 / (1 + gamma), free of cancellation
    k0.add(u2_0 / (1.f + sqrtf(1.f + u2_0)));
    k1.add(u2 / (1.f + 1.f / inv_gam));
    const float D[3] = {dt * u[0] * inv_gam, dt * u[1] * inv_gam, dt * u[2] * inv_gam};
    int s[3] = {0, 0, 0};
    float d1[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int ax = 0; ax < NDIM; ++ax) {
        const float pa = d[ax] + D[ax];
        float sa = floorf(pa);
        float da = pa - sa;
        if (da >= 1.f) { da = 0.f; sa += 1.f; }
        if (!(sa >= -1.f && sa <= 1.f)) {   // faster than one cell per step, or not finite:
            atomicOr(a.err, ERR_FAST_MOVE);  // flag it and keep every index in bounds
            sa = 0.f;
            da = d[ax];
        }
        s[ax] = (int)sa;
        d1[ax] = da;
    }
    if (fast) {
        if (acc.q0 != q0) {
            acc.flush(tc.Jhi, tc.Jlo, tc.nodes, tc.sx, tc.sxy);
            acc.reset(q0);
        }
        qs.q0 = q0;
        deposit_path<NDIM, float>(d, s, d1, D[2], sgn, qs);
    } else {
        deposit_global<NDIM>(g, a.J[0], a.J[1], a.J[2], ci, cj, ck, d, s, d1, D[2], sgn);
    }
    const int ni = g.wx(ci + s[0]), nj = g.wy(cj + s[1]), nk = NDIM == 3 ? g.wz(ck + s[2]) : 0;
    cell = pack_cell(NDIM, ni, nj, nk);
#pragma unroll
    for (int ax = 0; ax < NDIM; ++ax) d[ax] = d1[ax];
}

// Deposit the queued piece at ring position qhead + j with shared-memory atomics.
template <int NDIM>
__device__ __forceinline__ void drain_one(const QueueSink<NDIM> &qs, const TileCtx &tc, int j, float sgn) {
    const int idx = (qs.qhead + j) & (kQueue - 1);
    const float d[3] = {qs.q.d[idx], qs.q.d[kQueue + idx], qs.q.d[2 * kQueue + idx]};
    const float D[3] = {qs.q.D[idx], qs.q.D[kQueue + idx], qs.q.D[2 * kQueue + idx]};
    SmemSinkFx sd;
    sd.hi = tc.Jhi; sd.lo = tc.Jlo; sd.sx = tc.sx; sd.sxy = tc.sxy; sd.nodes = tc.nodes;
    sd.base0 = qs.q.base[idx];
    sd.set_cell(0, 0, 0);
    deposit_segment<NDIM, float>(d, D, sgn, sd);
}

// All species of one tile of one run (the body of both launch forms below).
template <int NDIM, int THREADS>
__device__ __forceinline__ void push_tile(const MixedStepArgs &a, const int tile) {
    extern __shared__ float4 smem4[];
    const Geom &g = a.g;
    const TileGeom &T = a.t;
    const int tx = tile % T.ntile[0];
    const int ty = (tile / T.ntile[0]) % T.ntile[1];
    const int tz = tile / (T.ntile[0] * T.ntile[1]);
    TileCtx tc;
    tc.x0 = tx * T.T[0]; tc.y0 = ty * T.T[1]; tc.z0 = NDIM == 3 ? tz * T.T[2] : 0;
    tc.Rx = T.R[0]; tc.Ry = T.R[1]; tc.Rz = NDIM == 3 ? T.R[2] : 1;
    tc.sx = tc.Rx; tc.sxy = tc.Rx * tc.Ry;
    tc.nodes = tc.Rx * tc.Ry * tc.Rz;
    tc.H = T.H; tc.T0 = T.T[0]; tc.T1 = T.T[1]; tc.T2 = T.T[2];
    const int nodes = tc.nodes;
    float4 *nA = smem4;
    float2 *nB = reinterpret_cast<float2 *>(smem4 + nodes);
    int *Jhi = reinterpret_cast<int *>(nB + nodes);
    int *Jlo = Jhi + 3 * nodes;
    tc.nA = nA; tc.nB = nB; tc.Jhi = Jhi; tc.Jlo = Jlo;

    // Stage node fields of the box [x0-H, x0+T+H) (padded coordinates x0 .. x0+R).
    for (int q = threadIdx.x; q < nodes; q += THREADS) {
        const int lx = q % tc.Rx, ly = (q / tc.Rx) % tc.Ry, lz = q / tc.sxy;
        const int gx = tc.x0 + lx, gy = tc.y0 + ly, gz = tc.z0 + lz;
        float4 va = make_float4(0.f, 0.f, 0.f, 0.f);
        float2 vb = make_float2(0.f, 0.f);
        if (gx < g.px && gy < g.py && gz < g.pz) {
            const long long p = ((long long)gz * g.py + gy) * g.px + gx;
            va = __ldg(a.nfA + p);
            vb = __ldg(a.nfB + p);
        }
        nA[q] = va;
        nB[q] = vb;
    }
    for (int q = threadIdx.x; q < 6 * nodes; q += THREADS) Jhi[q] = 0;   // hi and lo limbs
    __syncthreads();

    double kin0 = 0.0, kin1 = 0.0;
    RegAcc<NDIM> acc;
    acc.q0 = -1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ int work_ctr[4];
    __shared__ int qcount[THREADS / 32];
    if (threadIdx.x < 4) work_ctr[threadIdx.x] = 0;
    if (lane == 0) qcount[warp] = 0;
    QueueSink<NDIM> qs;
    qs.acc = &acc;
    qs.q.base = reinterpret_cast<int *>(Jlo + 3 * nodes) + warp * 7 * kQueue;
    qs.q.d = reinterpret_cast<float *>(qs.q.base + kQueue);
    qs.q.D = qs.q.d + 3 * kQueue;
    qs.q.count = &qcount[warp];
    qs.qhead = 0;
    qs.sx = tc.sx;
    qs.sxy = tc.sxy;
    __syncthreads();
    for (int sp = 0; sp < a.nspecies; ++sp) {
        const SpeciesMixed P = a.sp[sp];
        const float h = a.h[sp], sgn = a.sgn[sp];
        KahanF k0, k1;
        const int pbeg = a.tile_start[sp][tile], pend = a.tile_start[sp][tile + 1];
        const int nt = pend - pbeg;
        const int nblk = nt >> 10;                       // full 1024-blocks, stored transposed
        const int nitems = nblk + ((nt - (nblk << 10)) + 31) / 32;   // + 32-particle tail chunks
        // work items are taken by whole warps from a shared counter
        for (;;) {
            int item = 0;
            if (lane == 0) item = atomicAdd(&work_ctr[sp], 1);
            item = __shfl_sync(0xffffffffu, item, 0);
            if (item >= nitems) break;
            // block item: lane walks base + 32k + lane, k = 0..31 (consecutive ranks);
            // tail chunk: one element per lane in rank order
            const int base = item < nblk ? pbeg + (item << 10) : pbeg + (nblk << 10) + ((item - nblk) << 5);
            const int kn = item < nblk ? 32 : 1;
#pragma unroll 1
            for (int k = 0; k < kn; ++k) {
                const int p = base + (k << 5) + lane;
                if (p < pend) {
                    uint32_t c = P.cell[p];
                    float d[3] = {P.off[0][p], P.off[1][p], NDIM == 3 ? P.off[2][p] : 0.f};
                    float u[3] = {P.u[0][p], P.u[1][p], P.u[2][p]};
                    push_one<NDIM>(a, tc, qs, h, sgn, c, d, u, k0, k1);
                    P.cell[p] = c;
                    P.off[0][p] = d[0];
                    P.off[1][p] = d[1];
                    if (NDIM == 3) P.off[2][p] = d[2];
                    P.u[0][p] = u[0]; P.u[1][p] = u[1]; P.u[2][p] = u[2];
                }
                __syncwarp();
                int waiting = qcount[warp];
                // deposit waiting pieces 32 at a time, one per lane, all lanes active
                const bool last = k + 1 == kn;
                while (waiting >= 32 || (last && waiting > 0)) {
                    if (lane < waiting) drain_one<NDIM>(qs, tc, lane, sgn);
                    const int took = waiting < 32 ? waiting : 32;
                    qs.qhead = (qs.qhead + took) & (kQueue - 1);
                    waiting -= took;
                }
                __syncwarp();
                if (lane == 0) qcount[warp] = waiting;
                __syncwarp();
            }
            acc.flush(Jhi, Jlo, nodes, tc.sx, tc.sxy);
        }
        kin0 += a.m_over_me[sp] * ((double)k0.s - (double)k0.c);
        kin1 += a.m_over_me[sp] * ((double)k1.s - (double)k1.c);
    }
    __syncthreads();

    // Flush the tile current into the padded global int64 current.
    for (int q = threadIdx.x; q < 3 * nodes; q += THREADS) {
        const long long v = (long long)Jhi[q] * 262144LL + (long long)Jlo[q];
        if (v == 0) continue;
        const int comp = q / nodes, r = q - comp * nodes;
        const int lx = r % tc.Rx, ly = (r / tc.Rx) % tc.Ry, lz = r / tc.sxy;
        const int gx = tc.x0 + lx, gy = tc.y0 + ly, gz = tc.z0 + lz;
        if (gx < g.px && gy < g.py && gz < g.pz)
            atomicAdd(a.J[comp] + ((long long)gz * g.py + gy) * g.px + gx, (unsigned long long)v);
    }
    if (a.kin_acc) {
        for (int o = 16; o > 0; o >>= 1) {
            kin0 += __shfl_xor_sync(0xffffffffu, kin0, o);
            kin1 += __shfl_xor_sync(0xffffffffu, kin1, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(a.kin_acc, kin0);
            atomicAdd(a.kin_acc + 1, kin1);
        }
    }
    __syncthreads();   // shared memory is reused by the next tile of a persistent CTA
}

// One CTA per tile of one run.
template <int NDIM, int THREADS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) k_push_mixed(MixedStepArgs a) {
    push_tile<NDIM, THREADS>(a, blockIdx.x);
}

// Persistent form for a batch of independent runs of uneven size: resident
// CTAs take (run, tile) work items from one counter until all tiles of all
// runs are done, so small runs do not leave most of the GPU idle.
// tile_prefix[r] is the number of tiles of runs 0..r-1.
template <int NDIM, int THREADS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) k_push_mixed_multi(const MixedStepArgs *runs, const int *tile_prefix,
                                                                    int nruns, int *counter) {
    __shared__ int item_sh;
    __shared__ __align__(16) MixedStepArgs args_sh;
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
        push_tile<NDIM, THREADS>(args_sh, item - tile_prefix[lo]);
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

template <int NDIM, int THREADS, int MINB>
void launch_t(const MixedStepArgs &a, size_t smem, cudaStream_t s) {
    cudaFuncSetAttribute(k_push_mixed<NDIM, THREADS, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_push_mixed<NDIM, THREADS, MINB><<<a.t.ntiles, THREADS, smem, s>>>(a);
}

}  // namespace

size_t mixed_smem_bytes(const TileGeom &t, int ndim) {
    const size_t nodes = (size_t)t.R[0] * t.R[1] * (ndim == 3 ? t.R[2] : 1);
    const int warps = (ndim == 3 ? 512 : 256) / 32;
    return nodes * (sizeof(float4) + sizeof(float2) + 6 * sizeof(int)) + (size_t)warps * 7 * kQueue * sizeof(int);
}

void launch_half_back_mixed(const Geom &g, const float4 *nfA, const float2 *nfB, SpeciesMixed sp, long long n,
                            float h, float dt, cudaStream_t s) {
    if (n <= 0) return;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 152LL * 16);
    if (g.ndim == 3) k_half_back_mixed<3><<<blocks, 256, 0, s>>>(g, nfA, nfB, sp, n, h, dt);
    else k_half_back_mixed<2><<<blocks, 256, 0, s>>>(g, nfA, nfB, sp, n, h, dt);
}

template <int NDIM, int THREADS, int MINB>
void launch_multi_t(const MixedStepArgs *runs, const int *tile_prefix, int nruns, int *counter, size_t smem,
                    cudaStream_t s) {
    auto k = k_push_mixed_multi<NDIM, THREADS, MINB>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, THREADS, smem);
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k<<<std::max(1, per_sm) * sms, THREADS, smem, s>>>(runs, tile_prefix, nruns, counter);
}

void launch_push_mixed_multi(const MixedStepArgs *runs_dev, const int *tile_prefix_dev, int nruns, int ndim,
                             const TileGeom &t, int *counter, cudaStream_t s) {
    const size_t smem = mixed_smem_bytes(t, ndim);
    if (ndim == 3) launch_multi_t<3, 512, 1>(runs_dev, tile_prefix_dev, nruns, counter, smem, s);
    else launch_multi_t<2, 256, 2>(runs_dev, tile_prefix_dev, nruns, counter, smem, s);
}

void launch_push_mixed(const MixedStepArgs &a, cudaStream_t s) {
    const size_t smem = mixed_smem_bytes(a.t, a.g.ndim);
    if (a.g.ndim == 3) launch_t<3, 512, 1>(a, smem, s);
    else launch_t<2, 256, 2>(a, smem, s);
}

}  // namespace pic
