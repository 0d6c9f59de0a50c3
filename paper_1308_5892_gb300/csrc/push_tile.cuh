// push_tile.cuh -- the mixed-precision tile body: gather, Boris push, move and
// charge-conserving deposit (main loop steps 2, 3, 8, 9 of App. A.3.1) for
// all species of one tile of cells per CTA.
//
// Data (per tile of T cells with a halo of H cells on every side, R = T + 2H):
//  - node fields E, B at time t (App. A.3.3 averages, computed once per step
//    by the field kernels) for the R^d nodes of the tile + halo are staged in
//    shared memory as one float4 {E_x,E_y,E_z,B_x} and one float2 {B_y,B_z}
//    per node, by two TMA tensor copies (coalesced loads when the geometry
//    breaks a TMA alignment rule);
//  - the current of the tile + halo is accumulated in shared memory in exact
//    fixed point.  Every flux v (units of the particle volume times sgn q;
//    |v| < 1 because |D| < dt < 1) is rounded once, x = rint(v 2^26), an
//    int32, and x is added as two int32 limbs, hi += x >> 12 and
//    lo += x & 4095.  Range: the pieces of one particle move it by at most
//    dt < 1 in all, so the fluxes one particle leaves at one slot sum to less
//    than 1 in magnitude, and one slot receives at most 4 pieces of it.  A
//    tile of N particles (all species) therefore puts |hi| < N 2^14 and
//    lo < 4 N 2^12 into a slot: both stay below 2^31 while N < 2^17 = 131072.
//    A tile works through its particles in rounds of at most 64 work items
//    (65536 particles), and before a round that could bring the particles
//    summed since the last flush to 2^17 the limbs are added to the global
//    current and cleared, so no tile size or particle density can overflow
//    them (dense filaments put several times the mean count into a tile).
//    Integer sums are exact and associative, so the current does not depend
//    on the order of the particles, on the tiling or on the sort interval.  At
//    the end hi 2^22 + lo 2^10 (units 2^-36) is added once per node to the
//    global int64 current.  The rounding, 2^-27 at most per flux, is below the
//    FP32 rounding of the flux itself.  (FP32 shared atomics would serialise
//    on the address conflicts that cell-sorted particles cause on every
//    deposit; integer atomics and the register accumulation below avoid that.)
//  - particles (packed cell, FP32 offsets, FP32 momenta) are streamed once:
//    read 24 B (2D) / 28 B (3D) and written back.  Each warp prefetches the
//    particles of its next iterations with cp.async into a ring of
//    shared-memory stages, so the DRAM latency overlaps the arithmetic.
// Work of a warp: 1024-particle blocks, which the sort stores 32 x 32
// transposed, so lane a walks 32 consecutive cell-sorted particles (and keeps
// their start-cell current in registers until its cell changes) while one
// load instruction still reads one contiguous 128-byte row.  The pieces of a
// path after a node-plane crossing are queued per warp and deposited 32 at a
// time by all lanes together.
// A particle whose stencil leaves the staged box (it drifted far since the
// last sort), or that a conducting wall reflects, takes a slow path that
// gathers from global memory and deposits with global int64 atomics of the
// same fixed-point values, so the result never depends on the sort interval.
// On the step before a sort the kernel also counts the sort's key histogram.
//
// Roofline: HBM bound at 2 x 24 B (2D) or 2 x 28 B (3D) per particle-step;
// field and current traffic per cell is amortised over the particles per cell.
// Measured: the kernel moves its algorithmic bytes and is bound by instruction
// issue and dependent-arithmetic latency at 16 warps per SM (128 registers).
// The kernels that run this body are in push_mixed.cu (one tile per CTA, and
// a persistent batch) and walk.cu (the persistent ensemble step).
#pragma once
#include "particle_core.cuh"
#include "pic_internal.cuh"

namespace pic {

namespace {

constexpr float kFx26 = 67108864.0f;   // 2^26: fixed-point scale of one flux
constexpr unsigned kFull = 0xffffffffu;

// The fixed-point value of one flux (see the header comment).  The deposit's
// prefactor carries the scale (alpha 2^26, a power of two, so every product is
// the flux times 2^26 exactly), and v26 only needs rounding here.
__device__ __forceinline__ int fx(float v26) { return __float2int_rn(v26); }

// Global current sink for particles outside the staged box: the same
// fixed-point value in units 2^-36, added as one int64 at the interior-wrapped
// padded index.
struct GlobalSinkFx {
    const Geom *g;
    unsigned long long *J[3];
    int ci, cj, ck, oi, oj, ok;
    __device__ void set_cell(int di, int dj, int dk) { oi = ci + di; oj = cj + dj; ok = ck + dk; }
    __device__ void operator()(int comp, int di, int dj, int dk, float v) {
        const long long f = (long long)fx(v) * 1024LL;
        atomicAdd(J[comp] + g->widx(oi + di, oj + dj, ok + dk), (unsigned long long)f);
    }
};

// Slow path of a particle outside the staged box: deposit with global atomics.
template <int NDIM>
__device__ __noinline__ void deposit_global(const Geom &g, unsigned long long *J0, unsigned long long *J1,
                                            unsigned long long *J2, int ci, int cj, int ck, const float d[3],
                                            const int s[3], const float d1[3], float dz, float alpha26) {
    GlobalSinkFx gs;
    gs.g = &g;
    gs.J[0] = J0; gs.J[1] = J1; gs.J[2] = J2;
    gs.ci = ci; gs.cj = cj; gs.ck = ck;
    PieceDeposit<NDIM, float, GlobalSinkFx> pd(gs);
    deposit_path<NDIM, float>(d, s, d1, dz, alpha26, pd);
}

// Slow path of a particle reflected by a conducting wall in x (App. A.4):
// the path to the wall and the mirrored remainder are deposited as two legs.
// side -1: wall at the low face of cell ci (x = 0), +1: at its high face (x = nx).
template <int NDIM>
__device__ __noinline__ void deposit_reflect(const Geom &g, unsigned long long *J0, unsigned long long *J1,
                                             unsigned long long *J2, int ci, int cj, int ck, const float d0[3],
                                             const float D[3], int side, float alpha26) {
    const float wall = side < 0 ? 0.f : 1.f;           // in the x coordinates of cell ci
    const float t = (wall - d0[0]) / D[0];             // parameter of the wall hit, in [0, 1]
    const float L1[3] = {wall - d0[0], D[1] * t, D[2] * t};
    const float L2[3] = {-(D[0] - L1[0]), D[1] - L1[1], D[2] - L1[2]};
    int c[3] = {ci, cj, ck};
    float st[3] = {d0[0], d0[1], d0[2]};
#pragma unroll 1
    for (int leg = 0; leg < 2; ++leg) {
        const float *L = leg == 0 ? L1 : L2;
        int s[3] = {0, 0, 0};
        float d1[3] = {0.f, 0.f, 0.f};
        // x stays in cell ci: the first leg ends on the wall, the second starts there
        d1[0] = leg == 0 ? wall : fminf(fmaxf(wall + L[0], 0.f), 1.f);
        for (int a = 1; a < NDIM; ++a) {
            const float pa = st[a] + L[a];
            float sa = floorf(pa);
            float da = pa - sa;
            if (da >= 1.f) { da = 0.f; sa += 1.f; }
            sa = fminf(fmaxf(sa, -1.f), 1.f);
            s[a] = (int)sa;
            d1[a] = da;
        }
        deposit_global<NDIM>(g, J0, J1, J2, c[0], c[1], c[2], st, s, d1, L[2], alpha26);
        // the second leg starts where the first ended
        st[0] = wall;
        for (int a = 1; a < NDIM; ++a) { c[a] += s[a]; st[a] = d1[a]; }
    }
}

template <int NDIM>
__device__ __forceinline__ void gather_nodes(const float4 *nA, const float2 *nB, int q0, int sx, int sxy,
                                             const float d[3], float E[3], float B[3]) {
    // paired FP32 multiply-adds (two lanes of one instruction, each rounded as a
    // single fused multiply-add): E_x E_y, E_z B_x and B_y B_z
    float2 e01 = make_float2(0.f, 0.f), e2b0 = e01, b12 = e01;
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
                const float2 ww = make_float2(w, w);
                e01 = __ffma2_rn(ww, make_float2(a.x, a.y), e01);
                e2b0 = __ffma2_rn(ww, make_float2(a.z, a.w), e2b0);
                b12 = __ffma2_rn(ww, b, b12);
            }
    E[0] = e01.x; E[1] = e01.y; E[2] = e2b0.x;
    B[0] = e2b0.y; B[1] = b12.x; B[2] = b12.y;
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
                // with walls the x node is not wrapped: node nx lies in the padding and holds the
                // masked averages of the high wall, which differ from node 0's
                const long long q = g.bcx == 1 ? g.pidx(ci + eps, g.wy(cj + eta), g.wz(ck + xi))
                                               : g.widx(ci + eps, cj + eta, ck + xi);
                const float4 a = ldro(nA + q);
                const float2 b = ldro(nB + q);
                E[0] += w * a.x; E[1] += w * a.y; E[2] += w * a.z;
                B[0] += w * a.w; B[1] += w * b.x; B[2] += w * b.y;
            }
}

// Value index of a start-cell flux in the register accumulator:
// 3D comp 0 (dj + 2dk), comp 1 4 + (di + 2dk), comp 2 8 + (di + 2dj);
// 2D comp 0 dj, comp 1 2 + di, comp 2 4 + (di + 2dj).
template <int NDIM>
__device__ __forceinline__ int acc_index(int comp, int di, int dj, int dk) {
    if (NDIM == 3) return comp == 0 ? dj + 2 * dk : (comp == 1 ? 4 + di + 2 * dk : 8 + di + 2 * dj);
    return comp == 0 ? dj : (comp == 1 ? 2 + di : 4 + di + 2 * dj);
}
template <int NDIM>
__device__ __forceinline__ void acc_offset(int v, int &comp, int &di, int &dj, int &dk) {
    di = dj = dk = 0;
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
}

// Start-cell fluxes of consecutive particles of one lane that start in the
// same cell, summed exactly in registers (units 2^-26; at most 32 particles of
// |v| <= |D| < dt < 2^-1/2 each, so |sum| < 2^30.5: no overflow) and added to
// shared memory once per cell.
template <int NDIM>
struct RegAcc {
    static constexpr int NV = NDIM == 3 ? 12 : 8;
    int x[NV];
    int q0;   // local node index of the accumulation cell, -1 when empty
    __device__ __forceinline__ void reset(int q) {
#pragma unroll
        for (int v = 0; v < NV; ++v) x[v] = 0;
        q0 = q;
    }
    __device__ __forceinline__ void operator()(int comp, int di, int dj, int dk, float v) {
        x[acc_index<NDIM>(comp, di, dj, dk)] += fx(v);
    }
    __device__ __forceinline__ void flush(int *Jhi, int *Jlo, int nodes, int sx, int sxy) {
        if (q0 < 0) return;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            int comp, di, dj, dk;
            acc_offset<NDIM>(v, comp, di, dj, dk);
            const int q = comp * nodes + q0 + di + dj * sx + dk * sxy;
            atomicAdd(Jhi + q, x[v] >> 12);
            atomicAdd(Jlo + q, x[v] & 4095);
        }
        q0 = -1;
    }
};

// Shared-memory value sink of queued pieces: both limbs with integer atomics.
struct SmemSinkFx {
    int *hi, *lo;
    int sx, sxy, nodes, base;
    __device__ __forceinline__ void operator()(int comp, int di, int dj, int dk, float v) {
        const int q = comp * nodes + base + di + dj * sx + dk * sxy;
        const int x = fx(v);
        atomicAdd(hi + q, x >> 12);
        atomicAdd(lo + q, x & 4095);
    }
};

// cp.async of one 4-byte word, global -> shared, and its group fences.
__device__ __forceinline__ void cp_async4(uint32_t saddr, const void *gptr) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(saddr), "l"(__cvta_generic_to_global(gptr))
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// mbarrier and TMA tensor copies (node-field staging).
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint32_t bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for phase `parity` of the barrier; false if it did not complete
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, int limit) {
    for (int it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load(int ndim, uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                                         uint32_t bar) {
    if (ndim == 3)
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
            "[%5];\n" ::"r"(dst), "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
            : "memory");
    else
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
            "[%4];\n" ::"r"(dst), "l"(map), "r"(c0), "r"(c1), "r"(bar)
            : "memory");
}

constexpr int kQueue = 64;      // per-warp ring of waiting pieces (at most 63 wait at any time)
constexpr int kRoundItems = 64; // work items per round of a tile (at most 64 x 1024 particles)
constexpr int kStages = 3;      // per-warp particle prefetch ring
// words of one particle in a stage: cell, NDIM offsets, 3 momenta
template <int NDIM> __host__ __device__ constexpr int words_per_particle() { return NDIM + 4; }

// Shared memory of one warp after the node fields and the current limbs: the
// piece queue (cell base, d[3], D[3]: 7 x kQueue words) and the particle
// stages (kStages x words_per_particle x 32 words, word-major).
template <int NDIM>
__host__ __device__ constexpr int warp_smem_words() { return 7 * kQueue + kStages * words_per_particle<NDIM>() * 32; }

// Per-CTA constants of the tile.
struct TileCtx {
    int x0, y0, z0, Rx, Ry, Rz, sx, sxy, nodes, H, T0, T1, T2;
    const float4 *nA;
    const float2 *nB;
    int *Jhi, *Jlo;
};

// Gather, Boris and move of one particle.  On return c, d, u hold the new
// state; d0, s, D describe the path for the deposit; fast tells whether the
// stencil stays in the staged box, and q0 is then the local node index of the
// start cell.
template <int NDIM, bool WALLS>
__device__ __forceinline__ void push_one(const MixedStepArgs &a, const TileCtx &tc, float h, uint32_t &c, float d[3],
                                         float u[3], float d0[3], int s[3], float D[3], bool &fast, int &q0,
                                         int &ci, int &cj, int &ck, float &kin0, float &kin1, int &side) {
    const Geom &g = a.g;
    unpack_cell(NDIM, c, ci, cj, ck);
    // local cell in the staged box, nearest periodic image of the tile
    int lx = ci - tc.x0, ly = cj - tc.y0, lz = NDIM == 3 ? ck - tc.z0 : 0;
    if (lx >= tc.T0 + tc.H) lx -= g.nx; else if (lx < -tc.H) lx += g.nx;
    if (ly >= tc.T1 + tc.H) ly -= g.ny; else if (ly < -tc.H) ly += g.ny;
    if (NDIM == 3) { if (lz >= tc.T2 + tc.H) lz -= g.nz; else if (lz < -tc.H) lz += g.nz; }
    lx += tc.H; ly += tc.H; lz += NDIM == 3 ? tc.H : 0;
    // fast path: the gather reads nodes l..l+1 and the deposit writes nodes
    // l-1..l+2 of the staged box, all of which must also lie in the padded grid
    fast = lx >= 1 && lx <= tc.Rx - 3 && ly >= 1 && ly <= tc.Ry - 3 && tc.x0 + lx + 2 < g.px &&
           tc.y0 + ly + 2 < g.py;
    if (NDIM == 3) fast = fast && lz >= 1 && lz <= tc.Rz - 3 && tc.z0 + lz + 2 < g.pz;
    q0 = lx + ly * tc.sx + lz * tc.sxy;
    float E[3], B[3];
    if (fast) gather_nodes<NDIM>(tc.nA, tc.nB, q0, tc.sx, tc.sxy, d, E, B);
    else gather_global<NDIM>(g, a.nfA, a.nfB, ci, cj, ck, d, E, B);
    // explicit roundings (nothing left to contract), so that every kernel that
    // inlines this body computes the same bits
    const float u2_0 = __fmaf_rn(u[2], u[2], __fmaf_rn(u[1], u[1], __fmul_rn(u[0], u[0])));
    const float dt = a.dt;
    boris<float>(u, E, B, h, dt);
    const float u2 = __fmaf_rn(u[2], u[2], __fmaf_rn(u[1], u[1], __fmul_rn(u[0], u[0])));
    const float inv_gam = rsqrtf(__fadd_rn(1.f, u2));
    // gamma - 1 = u^2 / (1 + gamma), free of cancellation
    kin0 = __fadd_rn(kin0, __fdividef(u2_0, __fmaf_rn(__fadd_rn(1.f, u2_0), rsqrtf(__fadd_rn(1.f, u2_0)), 1.f)));
    kin1 = __fadd_rn(kin1, __fdividef(u2, __fmaf_rn(__fadd_rn(1.f, u2), inv_gam, 1.f)));
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        D[ax] = dt * u[ax] * inv_gam;
        d0[ax] = d[ax];
        s[ax] = 0;
    }
    // conducting walls in x (App. A.4): a particle that would cross a wall is reflected
    side = 0;
    if (WALLS) {
        const float px = d[0] + D[0];
        side = (ci == 0 && px < 0.f) ? -1 : ((ci == g.nx - 1 && px > 1.f) ? 1 : 0);
    }
#pragma unroll
    for (int ax = 0; ax < NDIM; ++ax) {
        const float pa = d[ax] + D[ax];
        float sa = floorf(pa);
        float da = snap_offset<float>(pa - sa);   // the end offset on the 2^-24 grid
        if (da >= 1.f) { da = 0.f; sa += 1.f; }
        if (!(sa >= -1.f && sa <= 1.f)) {   // faster than one cell per step, or not finite:
            atomicOr(a.err, ERR_FAST_MOVE);  // flag it and keep every index in bounds
            sa = 0.f;
            da = d[ax];
        }
        s[ax] = (int)sa;
        d[ax] = da;
    }
    if (WALLS && side != 0) {
        // mirrored end in the same cell, x momentum reversed; deposited by the slow path
        s[0] = 0;
        d[0] = fminf(fmaxf(side < 0 ? -(d0[0] + D[0]) : 2.f - (d0[0] + D[0]), 0.f), 1.f);
        u[0] = -u[0];
        fast = false;
    } else if (WALLS && ci + s[0] >= g.nx) {
        // landed exactly on the high wall: it stays in the last cell at offset 1
        s[0] = 0;
        d[0] = 1.f;
    }
    // with walls, x is never wrapped (cell 0 and nx - 1 hold the particles at the walls)
    const int ni = WALLS ? ci + s[0] : g.wx(ci + s[0]);
    const int nj = g.wy(cj + s[1]), nk = NDIM == 3 ? g.wz(ck + s[2]) : 0;
    c = pack_cell(NDIM, ni, nj, nk);
}

// Deposit the queued piece at ring position idx with shared-memory atomics.
template <int NDIM>
__device__ __forceinline__ void drain_one(const int *q_base, const float *q_d, const float *q_D, int idx,
                                          const TileCtx &tc, float alpha26) {
    const float d[3] = {q_d[idx], q_d[kQueue + idx], NDIM == 3 ? q_d[2 * kQueue + idx] : 0.f};
    const float D[3] = {q_D[idx], q_D[kQueue + idx], q_D[2 * kQueue + idx]};
    SmemSinkFx sd;
    sd.hi = tc.Jhi; sd.lo = tc.Jlo; sd.sx = tc.sx; sd.sxy = tc.sxy; sd.nodes = tc.nodes;
    sd.base = q_base[idx];
    deposit_segment<NDIM, float>(d, D, alpha26, sd);
}

// All species of one tile of one run (the body of both launch forms below).
// Offset of the nfB stage after the nfA stage of `nodes` nodes (TMA destinations are 128-byte aligned).
__host__ __device__ inline size_t node_b_offset(int nodes) { return ((size_t)nodes * 16 + 127) & ~size_t(127); }

// tmaps: the arguments' copy whose TMA descriptors are in parameter or global
// memory (the multi-run kernel stages its arguments in shared memory).
// CT: fixed tile geometry code (fixed_tile), 0 for the run-time geometry.
template <int NDIM, int THREADS, bool WALLS, bool HIST, int CT = 0>
__device__ __forceinline__ void push_tile(const MixedStepArgs &a, const int tile, const MixedStepArgs *tmaps) {
    extern __shared__ __align__(128) float4 smem4[];
    __shared__ __align__(8) unsigned long long tma_bar;
    constexpr int WARPS = THREADS / 32;
    constexpr int NW = words_per_particle<NDIM>();
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
    if constexpr (CT != 0) {
        // the same geometry as constants: offsets of nodes and current slots fold into immediates
        constexpr FixedTile F = fixed_tile(CT);
        constexpr int Rx = F.T0 + 2 * F.H, Ry = F.T1 + 2 * F.H, Rz = NDIM == 3 ? F.T2 + 2 * F.H : 1;
        tc.x0 = tx * F.T0; tc.y0 = ty * F.T1; tc.z0 = NDIM == 3 ? tz * F.T2 : 0;
        tc.Rx = Rx; tc.Ry = Ry; tc.Rz = Rz;
        tc.sx = Rx; tc.sxy = Rx * Ry; tc.nodes = Rx * Ry * Rz;
        tc.H = F.H; tc.T0 = F.T0; tc.T1 = F.T1; tc.T2 = F.T2;
    }
    const int nodes = tc.nodes;
    float4 *nA = smem4;
    float2 *nB = reinterpret_cast<float2 *>(reinterpret_cast<char *>(smem4) + node_b_offset(nodes));
    int *Jhi = reinterpret_cast<int *>(nB + nodes);
    int *Jlo = Jhi + 3 * nodes;
    tc.nA = nA; tc.nB = nB; tc.Jhi = Jhi; tc.Jlo = Jlo;

    // Stage node fields of the box [x0-H, x0+T+H) (padded coordinates x0 .. x0+R):
    // one TMA tensor copy per array (zeros beyond the padded grid), or coalesced
    // loads when the geometry breaks a TMA alignment rule.
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&tma_bar);
    if (a.use_tma) {
        if (threadIdx.x == 0) {
            mbar_init(bar, 1);
            asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
            // earlier generic accesses to the stage (a previous tile) come before the copies
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            mbar_expect_tx(bar, (uint32_t)nodes * 24u);
            tma_load(NDIM, (uint32_t)__cvta_generic_to_shared(nA), &tmaps->tmA, 4 * tc.x0, tc.y0, tc.z0, bar);
            tma_load(NDIM, (uint32_t)__cvta_generic_to_shared(nB), &tmaps->tmB, 2 * tc.x0, tc.y0, tc.z0, bar);
        }
    } else {
        for (int q = threadIdx.x; q < nodes; q += THREADS) {
            const int lx = q % tc.Rx, ly = (q / tc.Rx) % tc.Ry, lz = q / tc.sxy;
            const int gx = tc.x0 + lx, gy = tc.y0 + ly, gz = tc.z0 + lz;
            float4 va = make_float4(0.f, 0.f, 0.f, 0.f);
            float2 vb = make_float2(0.f, 0.f);
            if (gx < g.px && gy < g.py && gz < g.pz) {
                const long long p = ((long long)gz * g.py + gy) * g.px + gx;
                va = ldro(a.nfA + p);
                vb = ldro(a.nfB + p);
            }
            nA[q] = va;
            nB[q] = vb;
        }
    }
    for (int q = threadIdx.x; q < 6 * nodes; q += THREADS) Jhi[q] = 0;   // hi and lo limbs

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    __shared__ int work_ctr[4];
    __shared__ double kin_sh[2][WARPS];
    if (threadIdx.x < 4) work_ctr[threadIdx.x] = 0;
    if (lane == 0) { kin_sh[0][warp] = 0.0; kin_sh[1][warp] = 0.0; }
    // this warp's piece queue and particle stages
    int *wsm = Jlo + 3 * nodes + warp * warp_smem_words<NDIM>();
    int *q_base = wsm;
    float *q_d = reinterpret_cast<float *>(wsm + kQueue);        // [3][kQueue]
    float *q_D = q_d + 3 * kQueue;                               // [3][kQueue]
    const uint32_t *stage = reinterpret_cast<const uint32_t *>(wsm + 7 * kQueue);   // [kStages][NW][32]
    const uint32_t stage_s = (uint32_t)__cvta_generic_to_shared(stage) + 4u * lane;
    __syncthreads();
    if (a.use_tma && !mbar_wait_bounded(bar, 0, 1 << 22)) {
        // the copy did not land in time: flag it, give it a second bounded wait, go on
        atomicOr(a.err, ERR_TIMEOUT);
        mbar_wait_bounded(bar, 0, 1 << 22);
    }

    // Add the tile's limbs to the padded global int64 current (CTA-wide; zero:
    // clear them for a further round of deposits).
    auto flush_limbs = [&](bool zero) {
        for (int q = threadIdx.x; q < 3 * nodes; q += THREADS) {
            const long long v = (long long)Jhi[q] * 4194304LL + (long long)Jlo[q] * 1024LL;   // 2^22, 2^10
            if (zero) { Jhi[q] = 0; Jlo[q] = 0; }
            if (v == 0) continue;
            const int comp = q / nodes, r = q - comp * nodes;
            const int lx = r % tc.Rx, ly = (r / tc.Rx) % tc.Ry, lz = r / tc.sxy;
            const int gx = tc.x0 + lx, gy = tc.y0 + ly, gz = tc.z0 + lz;
            if (gx < g.px && gy < g.py && gz < g.pz)
                atomicAdd(a.J[comp] + ((long long)gz * g.py + gy) * g.px + gx, (unsigned long long)v);
        }
    };
    long long since_flush = 0;   // particles summed into the limbs since they were last cleared (uniform)
    RegAcc<NDIM> acc;
    acc.q0 = -1;
    int qhead = 0, qcount = 0;   // warp-uniform state of the piece ring
    for (int sp = 0; sp < a.nspecies; ++sp) {
        const SpeciesMixed &P = a.sp[sp];
        const float h = a.h[sp], alpha26 = a.sgn[sp] * kFx26;   // deposit prefactor in fixed-point units
        const int pbeg = a.tile_start[sp][tile], pend = a.tile_start[sp][tile + 1];
        const int nt = pend - pbeg;
        const int nblk = nt >> 10;                       // full 1024-blocks, stored transposed
        const int nitems = nblk + ((nt - (nblk << 10)) + 31) / 32;   // + 32-particle tail chunks
        // prefetch the particle of iteration j of an item into stage j % kStages (one group per iteration)
        auto issue = [&](int base, int j, int kn) {
            const int p = base + (j << 5) + lane;
            if (j < kn && p < pend) {
                const uint32_t sa = stage_s + (uint32_t)((j % kStages) * NW * 128);
                cp_async4(sa, P.cell + p);
                cp_async4(sa + 128, P.off[0] + p);
                cp_async4(sa + 256, P.off[1] + p);
                if (NDIM == 3) cp_async4(sa + 384, P.off[2] + p);
                cp_async4(sa + (NDIM + 1) * 128, P.u[0] + p);
                cp_async4(sa + (NDIM + 2) * 128, P.u[1] + p);
                cp_async4(sa + (NDIM + 3) * 128, P.u[2] + p);
            }
            cp_async_commit();
        };
        // queued pieces carry this species' sign: they are deposited before the
        // species ends and before a flush of the limbs
        auto drain_queue = [&]() {
            if (qcount > 0) {
                __syncwarp();
                if (lane < qcount) drain_one<NDIM>(q_base, q_d, q_D, (qhead + lane) & (kQueue - 1), tc, alpha26);
                __syncwarp();
                qhead = (qhead + qcount) & (kQueue - 1);
                qcount = 0;
            }
        };
        for (int r0 = 0; r0 < nitems; r0 += kRoundItems) {
        const int r1 = min(nitems, r0 + kRoundItems);
        const bool need_flush = since_flush + (long long)(r1 - r0) * 1024 >= (1LL << 17);   // uniform
        if (r0 > 0 || need_flush) {
            // every warp has left the previous round; its pieces and register sums go to the limbs
            drain_queue();
            acc.flush(Jhi, Jlo, nodes, tc.sx, tc.sxy);
            __syncthreads();
            if (need_flush) {
                flush_limbs(true);
                since_flush = 0;
                __syncthreads();
            }
            if (threadIdx.x == 0) work_ctr[sp] = r0;
            __syncthreads();
        }
        since_flush += (long long)(r1 - r0) * 1024;
        // work items of the round are taken by whole warps from a shared counter
        for (;;) {
            int item = 0;
            if (lane == 0) item = atomicAdd(&work_ctr[sp], 1);
            item = __shfl_sync(kFull, item, 0);
            if (item >= r1) break;
            // block item: lane walks base + 32k + lane, k = 0..31 (consecutive ranks);
            // tail chunk: one element per lane in rank order
            const int base = item < nblk ? pbeg + (item << 10) : pbeg + (nblk << 10) + ((item - nblk) << 5);
            const int kn = item < nblk ? 32 : 1;
            float kin0 = 0.f, kin1 = 0.f;
            int hk = -1, hn = 0;   // HIST: sort key of the lane's current run of particles, and its length
#pragma unroll
            for (int j = 0; j < kStages - 1; ++j) issue(base, j, kn);
#pragma unroll 1
            for (int k = 0; k < kn; ++k) {
                issue(base, k + kStages - 1, kn);
                cp_async_wait<kStages - 1>();   // this lane's words of iteration k have landed
                const int p = base + (k << 5) + lane;
                int nc = 0, q0 = 0;
                PathSplit<NDIM, float> ps;
                if (p < pend) {
                    const uint32_t *st = stage + (k % kStages) * NW * 32 + lane;
                    uint32_t c = st[0];
                    float d[3] = {__uint_as_float(st[32]), __uint_as_float(st[64]),
                                  NDIM == 3 ? __uint_as_float(st[96]) : 0.f};
                    float u[3] = {__uint_as_float(st[(NDIM + 1) * 32]), __uint_as_float(st[(NDIM + 2) * 32]),
                                  __uint_as_float(st[(NDIM + 3) * 32])};
                    float d0[3], D[3];
                    int s[3], ci, cj, ck, side;
                    bool fast;
                    push_one<NDIM, WALLS>(a, tc, h, c, d, u, d0, s, D, fast, q0, ci, cj, ck, kin0, kin1, side);
                    P.cell[p] = c;
                    P.off[0][p] = d[0];
                    P.off[1][p] = d[1];
                    if (NDIM == 3) P.off[2][p] = d[2];
                    P.u[0][p] = u[0]; P.u[1][p] = u[1]; P.u[2][p] = u[2];
                    if (HIST) {
                        // histogram of the next sort: consecutive particles of a lane mostly share a key
                        int ki, kj, kk;
                        unpack_cell(NDIM, c, ki, kj, kk);
                        const int key = tile_key_pow2(a.t, ki, kj, kk);
                        if (key != hk) {
                            if (hn) atomicAdd(a.key_counts[sp] + hk, hn);
                            hk = key;
                            hn = 0;
                        }
                        ++hn;
                    }
                    if (fast) {
                        // the start-cell piece goes to the register accumulator
                        if (acc.q0 != q0) {
                            acc.flush(Jhi, Jlo, nodes, tc.sx, tc.sxy);
                            acc.reset(q0);
                        }
                        ps.init(d0, s, d, D[2]);
                        int cc[3];
                        float pd[3], pD[3];
                        ps.piece(0, cc, pd, pD);
                        deposit_segment<NDIM, float>(pd, pD, alpha26, acc);
                        nc = ps.ncross;
                    } else if (!WALLS || side == 0) {
                        deposit_global<NDIM>(g, a.J[0], a.J[1], a.J[2], ci, cj, ck, d0, s, d, D[2], alpha26);
                    } else {
                        deposit_reflect<NDIM>(g, a.J[0], a.J[1], a.J[2], ci, cj, ck, d0, D, side, alpha26);
                    }
                }
                // pieces after a crossing: append to the warp's ring, drain 32 at a time
                const int kmax = __reduce_max_sync(kFull, nc);
#pragma unroll 1
                for (int kp = 1; kp <= kmax; ++kp) {
                    const bool has = kp <= nc;
                    const unsigned m = __ballot_sync(kFull, has);
                    if (has) {
                        int cc[3];
                        float pd[3], pD[3];
                        ps.piece(kp, cc, pd, pD);
                        const int idx = (qhead + qcount + __popc(m & lt_mask)) & (kQueue - 1);
                        q_base[idx] = q0 + cc[0] + cc[1] * tc.sx + cc[2] * tc.sxy;
                        q_d[idx] = pd[0];
                        q_d[kQueue + idx] = pd[1];
                        if (NDIM == 3) q_d[2 * kQueue + idx] = pd[2];
                        q_D[idx] = pD[0];
                        q_D[kQueue + idx] = pD[1];
                        q_D[2 * kQueue + idx] = pD[2];
                    }
                    qcount += __popc(m);
                    if (qcount >= 32) {
                        __syncwarp();
                        drain_one<NDIM>(q_base, q_d, q_D, (qhead + lane) & (kQueue - 1), tc, alpha26);
                        __syncwarp();
                        qhead = (qhead + 32) & (kQueue - 1);
                        qcount -= 32;
                    }
                }
            }
            if (HIST && hn) atomicAdd(a.key_counts[sp] + hk, hn);
            // kinetic energy of the item (at most 32 values per lane in FP32), summed per warp in FP64
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                kin0 += __shfl_xor_sync(kFull, kin0, o);
                kin1 += __shfl_xor_sync(kFull, kin1, o);
            }
            if (lane == 0) {
                kin_sh[0][warp] += a.m_over_me[sp] * (double)kin0;
                kin_sh[1][warp] += a.m_over_me[sp] * (double)kin1;
            }
        }
        }   // rounds
        drain_queue();
    }
    acc.flush(Jhi, Jlo, nodes, tc.sx, tc.sxy);
    __syncthreads();
    flush_limbs(false);
    double *slot = a.hist.slot();
    if (slot && threadIdx.x < 2) {
        double t = 0.0;
        for (int w = 0; w < WARPS; ++w) t += kin_sh[threadIdx.x][w];
        atomicAdd(slot + threadIdx.x, t);
    }
    __syncthreads();   // shared memory is reused by the next tile of a persistent CTA
    if (a.use_tma && threadIdx.x == 0) mbar_inval(bar);
}

}  // namespace

}  // namespace pic
