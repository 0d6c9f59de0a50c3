// push_mixed.cu -- the mixed-precision tile kernel: gather, Boris push, move and
// charge-conserving deposit (main loop steps 2, 3, 8, 9 of App. A.3.1) for
// the particles of one tile of cells per CTA.
//
// Data (per tile of T cells with a halo of H cells on every side, R = T + 2H):
//  - node fields E, B at time t (App. A.3.3 averages, computed once per step
//    by the field kernels) for the R^d nodes of the tile + halo are staged in
//    shared memory, two float4 per node;
//  - the current of the tile + halo is accumulated in shared memory in FP32
//    with compensated (TwoSum) accumulation: every contribution is added with
//    an atomic that returns the old value, the exact rounding error of that
//    addition is recovered and added to a second (low) accumulator; at the end
//    hi + lo is added once per node to the global current;
//  - particles (packed cell, FP32 offsets, FP32 momenta) are sorted by tile and
//    streamed once: read 24 B (2D) / 28 B (3D) and write the same.
// A particle whose cell has drifted so far from its tile since the last sort
// that its stencil leaves the staged halo is handled by a slow path that
// gathers from global memory and deposits with global atomics, so the result
// never depends on the sort interval.
//
// Roofline: HBM bound.  Algorithmic bytes per particle-step = 2 x 24 B (2D) or
// 2 x 28 B (3D); field and current traffic per cell is amortised over the
// particles per cell.
#include "particle_core.cuh"
#include "pic_internal.cuh"

namespace pic {

namespace {

constexpr int kThreads = 256;

// Shared-memory current sink with compensated accumulation.
struct SmemSink {
    float *hi, *lo;
    int sx, sxy, nodes;   // strides of the local box and its size
    int base0, base;      // local node index of the start cell / of the current segment cell
    __device__ void set_cell(int di, int dj, int dk) { base = base0 + di + dj * sx + dk * sxy; }
    __device__ void operator()(int comp, int di, int dj, int dk, float v) {
        const int q = comp * nodes + base + di + dj * sx + dk * sxy;
        const float old = atomicAdd(hi + q, v);
        // TwoSum: the atomic stored fl(old + v); recover its rounding error exactly
        const float s = old + v;
        const float bb = s - old;
        const float err = (old - (s - bb)) + (v - bb);
        atomicAdd(lo + q, err);
    }
};

// Global current sink for particles outside the staged halo (interior-wrapped
// padded index, FP32 atomics).
struct GlobalSinkF {
    const Geom *g;
    float *J[3];
    int ci, cj, ck, oi, oj, ok;
    __device__ void set_cell(int di, int dj, int dk) { oi = ci + di; oj = cj + dj; ok = ck + dk; }
    __device__ void operator()(int comp, int di, int dj, int dk, float v) {
        atomicAdd(J[comp] + g->widx(oi + di, oj + dj, ok + dk), v);
    }
};

template <int NDIM>
__device__ inline void gather_nodes(const float4 *nodeF, int q0, int sx, int sxy, const float d[3], float E[3],
                                    float B[3]) {
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
                const float4 a = nodeF[2 * q];
                const float4 b = nodeF[2 * q + 1];
                E[0] += w * a.x; E[1] += w * a.y; E[2] += w * a.z;
                B[0] += w * a.w; B[1] += w * b.x; B[2] += w * b.y;
            }
}

template <int NDIM>
__device__ inline void gather_global(const Geom &g, const float4 *nf, int ci, int cj, int ck, const float d[3],
                                     float E[3], float B[3]) {
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
                const float4 a = __ldg(nf + 2 * q);
                const float4 b = __ldg(nf + 2 * q + 1);
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

template <int NDIM>
__global__ void __launch_bounds__(kThreads) k_push_mixed(MixedStepArgs a) {
    extern __shared__ float4 smem4[];
    const Geom &g = a.g;
    const TileGeom &T = a.t;
    const int tile = blockIdx.x;
    const int tx = tile % T.ntile[0];
    const int ty = (tile / T.ntile[0]) % T.ntile[1];
    const int tz = tile / (T.ntile[0] * T.ntile[1]);
    const int x0 = tx * T.T[0], y0 = ty * T.T[1], z0 = NDIM == 3 ? tz * T.T[2] : 0;
    const int Rx = T.R[0], Ry = T.R[1], Rz = NDIM == 3 ? T.R[2] : 1;
    const int sx = Rx, sxy = Rx * Ry;
    const int nodes = Rx * Ry * Rz;
    float4 *nodeF = smem4;
    float *Jhi = reinterpret_cast<float *>(smem4 + 2 * nodes);
    float *Jlo = Jhi + 3 * nodes;
    const int H = T.H;

    // Stage node fields of the box [x0-H, x0+T+H) (padded coordinates x0 .. x0+R).
    for (int q = threadIdx.x; q < nodes; q += blockDim.x) {
        const int lx = q % Rx, ly = (q / Rx) % Ry, lz = q / sxy;
        const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
        float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
        if (gx < g.px && gy < g.py && gz < g.pz) {
            const long long p = ((long long)gz * g.py + gy) * g.px + gx;
            v0 = __ldg(a.nf + 2 * p);
            v1 = __ldg(a.nf + 2 * p + 1);
        }
        nodeF[2 * q] = v0;
        nodeF[2 * q + 1] = v1;
    }
    for (int q = threadIdx.x; q < 6 * nodes; q += blockDim.x) Jhi[q] = 0.f;   // hi and lo
    __syncthreads();

    SmemSink ss;
    ss.hi = Jhi; ss.lo = Jlo; ss.sx = sx; ss.sxy = sxy; ss.nodes = nodes;
    GlobalSinkF gs;
    gs.g = &g;
    gs.J[0] = a.J[0]; gs.J[1] = a.J[1]; gs.J[2] = a.J[2];

    KahanF kin0, kin1;
    const int pbeg = a.tile_start[tile], pend = a.tile_start[tile + 1];
    const float dt = a.dt, h = a.h, alpha = a.alpha;
    for (int p = pbeg + threadIdx.x; p < pend; p += blockDim.x) {
        int ci, cj, ck;
        unpack_cell(NDIM, a.sp.cell[p], ci, cj, ck);
        float d[3] = {a.sp.off[0][p], a.sp.off[1][p], NDIM == 3 ? a.sp.off[2][p] : 0.f};
        float u[3] = {a.sp.u[0][p], a.sp.u[1][p], a.sp.u[2][p]};
        // local cell in the staged box, nearest periodic image of the tile
        int lx = ci - x0, ly = cj - y0, lz = NDIM == 3 ? ck - z0 : 0;
        if (g.bcx == 0) { if (lx >= T.T[0] + H) lx -= g.nx; else if (lx < -H) lx += g.nx; }
        if (ly >= T.T[1] + H) ly -= g.ny; else if (ly < -H) ly += g.ny;
        if (NDIM == 3) { if (lz >= T.T[2] + H) lz -= g.nz; else if (lz < -H) lz += g.nz; }
        lx += H; ly += H; lz += NDIM == 3 ? H : 0;
        // fast path: the gather reads nodes l..l+1 and the deposit writes nodes
        // l-1..l+2 of the staged box, all of which must also lie in the padded grid
        bool fast = lx >= 1 && lx <= Rx - 3 && ly >= 1 && ly <= Ry - 3 && x0 + lx + 2 < g.px && y0 + ly + 2 < g.py;
        if (NDIM == 3) fast = fast && lz >= 1 && lz <= Rz - 3 && z0 + lz + 2 < g.pz;
        const int q0 = lx + ly * sx + lz * sxy;
        float E[3], B[3];
        if (fast) gather_nodes<NDIM>(nodeF, q0, sx, sxy, d, E, B);
        else gather_global<NDIM>(g, a.nf, ci, cj, ck, d, E, B);
        const float u2_0 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        if (a.mode == 1) {   // initial staggering: Boris step of -dt/2, no move
            boris<float>(u, E, B, h, -0.5f * dt);
            a.sp.u[0][p] = u[0]; a.sp.u[1][p] = u[1]; a.sp.u[2][p] = u[2];
            continue;
        }
        boris<float>(u, E, B, h, dt);
        const float u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        const float inv_gam = rsqrtf(1.f + u2);
        // gamma - 1 = u^2 / (1 + gamma), free of cancellation
        kin0.add(u2_0 / (1.f + sqrtf(1.f + u2_0)));
        kin1.add(u2 / (1.f + 1.f / inv_gam));
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
            ss.base0 = q0;
            deposit_path<NDIM, float>(d, s, d1, D[2], alpha, ss);
        } else {
            gs.ci = ci; gs.cj = cj; gs.ck = ck;
            deposit_path<NDIM, float>(d, s, d1, D[2], alpha, gs);
        }
        const int ni = g.wx(ci + s[0]), nj = g.wy(cj + s[1]), nk = NDIM == 3 ? g.wz(ck + s[2]) : 0;
        a.sp.cell[p] = pack_cell(NDIM, ni, nj, nk);
        a.sp.off[0][p] = d1[0];
        a.sp.off[1][p] = d1[1];
        if (NDIM == 3) a.sp.off[2][p] = d1[2];
        a.sp.u[0][p] = u[0]; a.sp.u[1][p] = u[1]; a.sp.u[2][p] = u[2];
    }
    __syncthreads();

    // Flush the tile current (hi + lo) into the padded global current.
    if (a.mode == 0) {
        for (int q = threadIdx.x; q < 3 * nodes; q += blockDim.x) {
            const float v = Jhi[q] + Jlo[q];
            if (v == 0.f) continue;
            const int comp = q / nodes, r = q - comp * nodes;
            const int lx = r % Rx, ly = (r / Rx) % Ry, lz = r / sxy;
            const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
            if (gx < g.px && gy < g.py && gz < g.pz)
                atomicAdd(a.J[comp] + ((long long)gz * g.py + gy) * g.px + gx, v);
        }
        if (a.kin_acc) {
            double k0 = (double)kin0.s - (double)kin0.c, k1 = (double)kin1.s - (double)kin1.c;
            for (int o = 16; o > 0; o >>= 1) {
                k0 += __shfl_xor_sync(0xffffffffu, k0, o);
                k1 += __shfl_xor_sync(0xffffffffu, k1, o);
            }
            if ((threadIdx.x & 31) == 0) {
                atomicAdd(a.kin_acc, a.m_over_me * k0);
                atomicAdd(a.kin_acc + 1, a.m_over_me * k1);
            }
        }
    }
}

}  // namespace

size_t mixed_smem_bytes(const TileGeom &t, int ndim) {
    const size_t nodes = (size_t)t.R[0] * t.R[1] * (ndim == 3 ? t.R[2] : 1);
    return nodes * (2 * sizeof(float4) + 6 * sizeof(float));
}

void launch_push_mixed(const MixedStepArgs &a, cudaStream_t s) {
    const size_t smem = mixed_smem_bytes(a.t, a.g.ndim);
    if (a.g.ndim == 3) {
        cudaFuncSetAttribute(k_push_mixed<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_push_mixed<3><<<a.t.ntiles, kThreads, smem, s>>>(a);
    } else {
        cudaFuncSetAttribute(k_push_mixed<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_push_mixed<2><<<a.t.ntiles, kThreads, smem, s>>>(a);
    }
}

}  // namespace pic
