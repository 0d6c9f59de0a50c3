// field_cells.cuh -- per-cell bodies of the Yee FDTD field updates (App.
// A.3.2), the current fold and the node-averaged fields (App. A.3.3), shared
// by the field kernels (fields.cu) and the persistent ensemble step (walk.cu).
//
// Each body updates one padded cell from the interior images of its
// neighbours and writes only that cell (see fields.cu for the layout).
#pragma once
#include <type_traits>

#include "pic_internal.cuh"

namespace pic {

namespace {

// Padded coordinates of padded index p: multiply-high divisions while the
// grid has fewer than 2^32 padded cells, 64-bit division beyond.
__device__ inline void padded_coords(const Geom &g, long long p, int &pi, int &pj, int &pk) {
    if (g.pcells <= 0xffffffffLL) {
        const uint32_t n = (uint32_t)p;
        const uint32_t q = g.fpx.div(n);
        pi = (int)(n - q * (uint32_t)g.px);
        const uint32_t r = g.fpy.div(q);
        pj = (int)(q - r * (uint32_t)g.py);
        pk = (int)r;
        return;
    }
    pi = (int)(p % g.px);
    long long q = p / g.px;
    pj = (int)(q % g.py);
    pk = (int)(q / g.py);
}

template <typename R>
__device__ inline R ld(const R *a, long long i) { return ldro(a + i); }

// Block-wide FP64 sum of NV values, one atomicAdd per value per block.
template <int NV>
__device__ inline void block_accumulate(double (&v)[NV], double *acc) {
    __shared__ double red[NV][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double x = v[q];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[q][warp] = x;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double x = lane < nw ? red[q][lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0) atomicAdd(acc + q, x);
        }
    }
}

// b <- b - h curl e (Faraday, Eq. dyn3 on the Yee lattice).  When energy_acc
// is given, the interior sums of e^2 and b^2 (after the update) are added to
// energy_acc[0..5] in FP64.
template <typename R>
__device__ __forceinline__ void b_advance_cell(const Geom &g, const FieldPtrs<R> &f, R h, long long p, bool energy,
                                               double (&acc)[6]) {
    {
        int pi, pj, pk;
        padded_coords(g, p, pi, pj, pk);
        const int i = g.wx(pi - g.G), j = g.wy(pj - g.G), k = g.wz(pk - g.Gz);
        const long long c = g.pidx(i, j, k);
        const R ex = ld(f.e[0], c), ey = ld(f.e[1], c), ez = ld(f.e[2], c);
        const R curl_x = (ld(f.e[2], g.widx(i, j + 1, k)) - ez) - (ld(f.e[1], g.widx(i, j, k + 1)) - ey);
        const R curl_y = (ld(f.e[0], g.widx(i, j, k + 1)) - ex) - (ld(f.e[2], g.widx(i + 1, j, k)) - ez);
        const R curl_z = (ld(f.e[1], g.widx(i + 1, j, k)) - ey) - (ld(f.e[0], g.widx(i, j + 1, k)) - ex);
        R bx = f.b[0][p] - h * curl_x;
        R by = f.b[1][p] - h * curl_y;
        R bz = f.b[2][p] - h * curl_z;
        if (g.bcx == 1 && i == 0) bx = R(0);   // normal b vanishes on the conductor wall (App. A.4)
        f.b[0][p] = bx;
        f.b[1][p] = by;
        f.b[2][p] = bz;
        if (energy && pi == i + g.G && pj == j + g.G && pk == k + g.Gz) {
            acc[0] += (double)ex * (double)ex;
            acc[1] += (double)ey * (double)ey;
            acc[2] += (double)ez * (double)ez;
            acc[3] += (double)bx * (double)bx;
            acc[4] += (double)by * (double)by;
            acc[5] += (double)bz * (double)bz;
        }
    }
}

// Padded coordinates of the images of interior coordinate i along one axis
// (n cells, ghost width G): i + G - n, i + G, i + G + n, those inside [0, n + 2G),
// in that order; returns their count.
__device__ __forceinline__ int axis_images(int i, int n, int G, int (&q)[3]) {
    int c = 0;
    if (i >= n - G) q[c++] = i + G - n;
    q[c++] = i + G;
    if (i < G) q[c++] = i + G + n;
    return c;
}

// Sum of the current over every padded image of interior cell (i,j,k), in the
// order of increasing image offset along z, y, then x.
template <typename R>
__device__ inline R folded_current(const Geom &g, const R *J, int i, int j, int k) {
    int qx[3], qy[3], qz[3];
    const int nqx = axis_images(i, g.nx, g.G, qx), nqy = axis_images(j, g.ny, g.G, qy);
    const int nqz = g.ndim == 3 ? axis_images(k, g.nz, g.Gz, qz) : (qz[0] = k + g.Gz, 1);
    R s = R(0);
    for (int c = 0; c < nqz; ++c)
        for (int b = 0; b < nqy; ++b) {
            const long long row = ((long long)qz[c] * g.py + qy[b]) * g.px;
            for (int a = 0; a < nqx; ++a) s += J[row + qx[a]];
        }
    return s;
}

// Mixed path: the same update with the fixed-point current (int64, units of
// 2^-36 of sgn(q) times the volume flux); scale = |alpha| 2^-36, passed as an
// FP32 pair (scale_hi + scale_lo).  e is the FP32 pair e + el (FieldPtrs),
// updated with error-free FP32 transformations (Knuth's TwoSum, and the
// FMA-based exact product): the curl of the FP32 b values, the converted
// integer current and the sum are all carried to about 2^-48 relative, so
// div e - rho~ changes by the rounding of the fluxes alone and does not drift
// with the FP32 rounding of e (a single FP32 e made the Gauss residual grow by
// about 5e-9 of max rho per step in a 128^3 thermal plasma).  The FP32 pipe
// does this at a small fraction of the cost of the same update in FP64.
// Every operation is an explicit round-to-nearest intrinsic, never contracted,
// so the single-run and the batched field kernels give bitwise the same fields.
struct F2 {
    float hi, lo;
};
__device__ __forceinline__ F2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, err};
}
__device__ __forceinline__ F2 two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
// curl component (a - a_m) - (b - b_m) of four FP32 values, as a pair
__device__ __forceinline__ F2 curl_pair(float a, float a_m, float b, float b_m) {
    const F2 d1 = two_sum(a, -a_m), d2 = two_sum(b, -b_m);
    const F2 c = two_sum(d1.hi, -d2.hi);
    return {c.hi, __fadd_rn(__fsub_rn(d1.lo, d2.lo), c.lo)};
}
// an int64 as a pair of FP32 values whose sum is exact (|J| < 2^48)
__device__ __forceinline__ F2 ll_pair(long long J) {
    const float h = __ll2float_rn(J);
    return {h, __ll2float_rn(J - (long long)h)};
}
// The pair's new value (e + el) + h curl + scale J, renormalised.
__device__ __forceinline__ F2 e_pair_update(const FieldPtrs<float> &f, int c, long long p, float h, F2 curl,
                                            F2 scale, long long J) {
    const F2 hc = two_prod(h, curl.hi);
    const F2 j = ll_pair(J);
    const F2 sj = two_prod(scale.hi, j.hi);
    const float hc_lo = __fmaf_rn(h, curl.lo, hc.lo);
    const float sj_lo = __fadd_rn(sj.lo, __fadd_rn(__fmul_rn(scale.hi, j.lo), __fmul_rn(scale.lo, j.hi)));
    const F2 s1 = two_sum(f.e[c][p], hc.hi);
    const F2 s2 = two_sum(s1.hi, sj.hi);
    const float lo = __fadd_rn(__fadd_rn(__fadd_rn(f.el[c][p], hc_lo), __fadd_rn(sj_lo, s1.lo)), s2.lo);
    const float hi = __fadd_rn(s2.hi, lo);
    return {hi, __fsub_rn(lo, __fsub_rn(hi, s2.hi))};
}
__device__ __forceinline__ void e_pair_store(const FieldPtrs<float> &f, int c, long long p, F2 v) {
    f.e[c][p] = v.hi;
    f.el[c][p] = v.lo;
}

__device__ __forceinline__ void e_fx_cell(const Geom &g, const FieldPtrs<float> &f, const unsigned long long *J0,
                                          const unsigned long long *J1, const unsigned long long *J2,
                                          unsigned long long *Z0, unsigned long long *Z1, unsigned long long *Z2,
                                          float dt, F2 scale, long long p) {
    {
        int pi, pj, pk;
        padded_coords(g, p, pi, pj, pk);
        const int i = g.wx(pi - g.G), j = g.wy(pj - g.G), k = g.wz(pk - g.Gz);
        const long long c = g.pidx(i, j, k);
        const float bx = ld(f.b[0], c), by = ld(f.b[1], c), bz = ld(f.b[2], c);
        const F2 curl_x = curl_pair(bz, ld(f.b[2], g.widx(i, j - 1, k)), by, ld(f.b[1], g.widx(i, j, k - 1)));
        const F2 curl_y = curl_pair(bx, ld(f.b[0], g.widx(i, j, k - 1)), bz, ld(f.b[2], g.widx(i - 1, j, k)));
        const F2 curl_z = curl_pair(by, ld(f.b[1], g.widx(i - 1, j, k)), bx, ld(f.b[0], g.widx(i, j - 1, k)));
        F2 ex = e_pair_update(f, 0, p, dt, curl_x, scale, (long long)folded_current(g, J0, i, j, k));
        F2 ey = e_pair_update(f, 1, p, dt, curl_y, scale, (long long)folded_current(g, J1, i, j, k));
        F2 ez = e_pair_update(f, 2, p, dt, curl_z, scale, (long long)folded_current(g, J2, i, j, k));
        if (g.bcx == 1 && i == 0) { ey = F2{0.f, 0.f}; ez = F2{0.f, 0.f}; }
        e_pair_store(f, 0, p, ex);
        e_pair_store(f, 1, p, ey);
        e_pair_store(f, 2, p, ez);
        Z0[p] = 0ull;
        Z1[p] = 0ull;
        Z2[p] = 0ull;
    }
}

// The same update with the smoothed current: Js holds 3 compact planes (nx*ny*nz
// each, indexed (k*ny + j)*nx + i) in the units of the path's current, which
// scale converts (1 in the FP64 path, |alpha| 2^-36 in the mixed path).
template <typename R, typename ZT, typename CT>
__device__ __forceinline__ void e_smoothed_cell(const Geom &g, const FieldPtrs<R> &f, const CT *Js, double scale,
                                                ZT *Z0, ZT *Z1, ZT *Z2, R dt, long long p) {
    int pi, pj, pk;
    padded_coords(g, p, pi, pj, pk);
    const int i = g.wx(pi - g.G), j = g.wy(pj - g.G), k = g.wz(pk - g.Gz);
    const long long c = g.pidx(i, j, k);
    const long long ncell = (long long)g.nx * g.ny * g.nz;
    const long long q = ((long long)k * g.ny + j) * g.nx + i;
    const R bx = ld(f.b[0], c), by = ld(f.b[1], c), bz = ld(f.b[2], c);
    if constexpr (std::is_same<R, float>::value) {
        // the mixed path's FP32 pair, updated as in e_fx_cell (the smoothed current is int64 fixed point)
        const F2 sc = {(float)scale, (float)(scale - (double)(float)scale)};
        const F2 curl_x = curl_pair(bz, ld(f.b[2], g.widx(i, j - 1, k)), by, ld(f.b[1], g.widx(i, j, k - 1)));
        const F2 curl_y = curl_pair(bx, ld(f.b[0], g.widx(i, j, k - 1)), bz, ld(f.b[2], g.widx(i - 1, j, k)));
        const F2 curl_z = curl_pair(by, ld(f.b[1], g.widx(i - 1, j, k)), bx, ld(f.b[0], g.widx(i, j - 1, k)));
        F2 ex = e_pair_update(f, 0, p, dt, curl_x, sc, (long long)ldro(Js + q));
        F2 ey = e_pair_update(f, 1, p, dt, curl_y, sc, (long long)ldro(Js + ncell + q));
        F2 ez = e_pair_update(f, 2, p, dt, curl_z, sc, (long long)ldro(Js + 2 * ncell + q));
        if (g.bcx == 1 && i == 0) { ey = F2{0.f, 0.f}; ez = F2{0.f, 0.f}; }
        e_pair_store(f, 0, p, ex);
        e_pair_store(f, 1, p, ey);
        e_pair_store(f, 2, p, ez);
    } else {
        const R curl_x = (bz - ld(f.b[2], g.widx(i, j - 1, k))) - (by - ld(f.b[1], g.widx(i, j, k - 1)));
        const R curl_y = (bx - ld(f.b[0], g.widx(i, j, k - 1))) - (bz - ld(f.b[2], g.widx(i - 1, j, k)));
        const R curl_z = (by - ld(f.b[1], g.widx(i - 1, j, k))) - (bx - ld(f.b[0], g.widx(i, j - 1, k)));
        const R jx = (R)(scale * (double)ldro(Js + q));
        const R jy = (R)(scale * (double)ldro(Js + ncell + q));
        const R jz = (R)(scale * (double)ldro(Js + 2 * ncell + q));
        R ex = f.e[0][p] + dt * curl_x + jx;
        R ey = f.e[1][p] + dt * curl_y + jy;
        R ez = f.e[2][p] + dt * curl_z + jz;
        if (g.bcx == 1 && i == 0) { ey = R(0); ez = R(0); }
        f.e[0][p] = ex;
        f.e[1][p] = ey;
        f.e[2][p] = ez;
    }
    Z0[p] = ZT(0);
    Z1[p] = ZT(0);
    Z2[p] = ZT(0);
}

// Staggered value read by the gather; with conductor walls a value located
// inside the conductor, or a tangential e / normal b on the wall, reads zero.
__device__ inline float sval(const Geom &g, const float *a, bool xstag, int i, int j, int k) {
    if (g.bcx == 1) {
        if (xstag) { if (i < 0 || i > g.nx - 1) return 0.f; }
        else { if (i <= 0 || i >= g.nx) return 0.f; }
    }
    return ldro(a + g.widx(i, j, k));
}

// Node-averaged fields (App. A.3.3) at every padded node: e over its two edge
// neighbours, b over its four face neighbours.  Stored as {E_x,E_y,E_z,B_x} and {B_y,B_z}.
__device__ __forceinline__ void node_cell(const Geom &g, const FieldPtrs<float> &f, float4 *nfA, float2 *nfB,
                                          long long p) {
    {
        int pi, pj, pk;
        padded_coords(g, p, pi, pj, pk);
        // node coordinate (not wrapped: the conductor masking needs the true x)
        int i = pi - g.G;
        const int j = pj - g.G, k = pk - g.Gz;
        if (g.bcx == 0) i = g.wx(i);
        float E[3], B[3];
        E[0] = 0.5f * (sval(g, f.e[0], true, i - 1, j, k) + sval(g, f.e[0], true, i, j, k));
        E[1] = 0.5f * (sval(g, f.e[1], false, i, j - 1, k) + sval(g, f.e[1], false, i, j, k));
        E[2] = 0.5f * (sval(g, f.e[2], false, i, j, k - 1) + sval(g, f.e[2], false, i, j, k));
        B[0] = 0.25f * (sval(g, f.b[0], false, i, j, k) + sval(g, f.b[0], false, i, j - 1, k) +
                        sval(g, f.b[0], false, i, j, k - 1) + sval(g, f.b[0], false, i, j - 1, k - 1));
        B[1] = 0.25f * (sval(g, f.b[1], true, i, j, k) + sval(g, f.b[1], true, i - 1, j, k) +
                        sval(g, f.b[1], true, i, j, k - 1) + sval(g, f.b[1], true, i - 1, j, k - 1));
        B[2] = 0.25f * (sval(g, f.b[2], true, i, j, k) + sval(g, f.b[2], true, i - 1, j, k) +
                        sval(g, f.b[2], true, i - 1, j - 1, k) + sval(g, f.b[2], true, i, j - 1, k));
        nfA[p] = make_float4(E[0], E[1], E[2], B[0]);
        nfB[p] = make_float2(B[1], B[2]);
    }
}

}  // namespace

}  // namespace pic
