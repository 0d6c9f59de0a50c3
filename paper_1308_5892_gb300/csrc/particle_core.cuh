// particle_core.cuh -- per-particle arithmetic shared by the FP64 and the
// mixed-precision push kernels: the relativistic Boris step (App. A.3.3) and
// the charge-conserving current of straight segments inside one cell (App.
// A.1, A.3.4, Eq. current_dep).  Everything is written with compile-time
// indices only, so no per-thread array spills to local memory.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

namespace pic {

template <typename R> __device__ inline R rsqrt_(R x);
template <> __device__ inline float rsqrt_<float>(float x) { return rsqrtf(x); }
template <> __device__ inline double rsqrt_<double>(double x) { return 1.0 / sqrt(x); }
// Division: IEEE in FP64; in FP32 the fast reciprocal-based quotient (2 ulp for
// divisors in [2^-126, 2^126], which every divisor here is), far below the
// FP32 rounding of the arguments themselves.
// Fused multiply-add with one rounding, written out so that the breakpoints of
// a path do not depend on the compiler's choice to contract or not.
template <typename R> __device__ inline R fma_(R a, R b, R c);
template <> __device__ inline float fma_<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <> __device__ inline double fma_<double>(double a, double b, double c) { return __fma_rn(a, b, c); }
template <typename R> __device__ inline R div_(R a, R b);
template <> __device__ inline float div_<float>(float a, float b) { return __fdividef(a, b); }
template <> __device__ inline double div_<double>(double a, double b) { return a / b; }

// Boris step with h = (q/e)(m_e/m), fields E, B at the particle:
//   u- = u + h E dt/2;  gamma = sqrt(1 + u-^2);  t = h B dt/(2 gamma);
//   s = 2t/(1+t^2);  u' = u- + u- x t;  u+ = u- + u' x s;  u <- u+ + h E dt/2.
// This is the exact solution of the implicit rotation (u+ - u-)/dt =
// h/(2 gamma) (u+ + u-) x B of Eq. mover1.
template <typename R>
__device__ inline void boris(R u[3], const R E[3], const R B[3], R h, R dt) {
    const R qe = h * dt * R(0.5);
    R um[3] = {u[0] + qe * E[0], u[1] + qe * E[1], u[2] + qe * E[2]};
    const R inv_gam = rsqrt_<R>(R(1) + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    const R qb = qe * inv_gam;
    const R t[3] = {qb * B[0], qb * B[1], qb * B[2]};
    const R f = div_<R>(R(2), R(1) + t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    const R s[3] = {f * t[0], f * t[1], f * t[2]};
    const R up[3] = {um[0] + (um[1] * t[2] - um[2] * t[1]), um[1] + (um[2] * t[0] - um[0] * t[2]),
                     um[2] + (um[0] * t[1] - um[1] * t[0])};
    u[0] = um[0] + (up[1] * s[2] - up[2] * s[1]) + qe * E[0];
    u[1] = um[1] + (up[2] * s[0] - up[0] * s[2]) + qe * E[1];
    u[2] = um[2] + (up[0] * s[1] - up[1] * s[0]) + qe * E[2];
}

// Offsets of the mixed path lie on the grid of 2^-24 cells: the difference of
// two such values in [0, 1] is a multiple of 2^-24 below 1 in magnitude, hence
// exact in FP32, so every piece displacement equals its end minus its start and
// the pieces of a path telescope exactly to the stored move (the rounding of a
// displacement would otherwise move the deposited charge away from the stored
// position by up to half an ulp of the displacement, every step).  Identity in
// FP64.
template <typename R> __device__ inline R snap_offset(R x) { return x; }
template <> __device__ inline float snap_offset<float>(float x) {
    return rintf(x * 16777216.0f) * (1.0f / 16777216.0f);
}

// Current of one straight segment inside one cell: the particle (a cube of
// volume 1) starts at offset d within the cell and moves by D.  With
// mid-point weights W^0 = 1 - (d + D/2), W^1 = d + D/2, the flux through the x
// face at (i+1/2, j+eta, k+xi) is D_x [W_y^eta W_z^xi + (-1)^(eta+xi) D_y D_z/12]
// (the exact time integral of the overlap area of the cube with the face), and
// enters Ampere's law as -alpha times that flux; y and z by cyclic permutation.
// In 2D3V the cube is uniform along z: in-plane fluxes D_x W_y^eta and
// D_y W_x^eps, and the out-of-plane flux D_z [W_x^eps W_y^eta + (-1)^(eps+eta)
// D_x D_y / 12] goes to e_z at node (i+eps, j+eta).
// sink(comp, di, dj, dk, value) receives -alpha F for current component comp
// at offset (di, dj, dk) from the segment's cell (set by sink.set_cell).
template <int NDIM, typename R, class Sink>
__device__ __forceinline__ void deposit_segment(const R d[3], const R D[3], R alpha, Sink &sink) {
    R w1[3], w0[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        w1[a] = d[a] + R(0.5) * D[a];
        w0[a] = R(1) - w1[a];
    }
    const R ax = -alpha * D[0], ay = -alpha * D[1], az = -alpha * D[2];
    if constexpr (std::is_same<R, float>::value) {
        // FP32: the same values by paired multiply-adds (two lanes per instruction,
        // each lane rounded exactly as the scalar fused form below)
        const float2 X = make_float2(w0[0], w1[0]), Y = make_float2(w0[1], w1[1]);
        float2 t;
        if (NDIM == 3) {
            const float cyz = D[1] * D[2] * (1.f / 12.f), czx = D[2] * D[0] * (1.f / 12.f),
                        cxy = D[0] * D[1] * (1.f / 12.f);
            const float2 axx = make_float2(ax, ax), ayy = make_float2(ay, ay);
            t = __fmul2_rn(axx, __ffma2_rn(Y, make_float2(w0[2], w0[2]), make_float2(cyz, -cyz)));
            sink(0, 0, 0, 0, t.x); sink(0, 0, 1, 0, t.y);
            t = __fmul2_rn(axx, __ffma2_rn(Y, make_float2(w1[2], w1[2]), make_float2(-cyz, cyz)));
            sink(0, 0, 0, 1, t.x); sink(0, 0, 1, 1, t.y);
            t = __fmul2_rn(ayy, __ffma2_rn(X, make_float2(w0[2], w0[2]), make_float2(czx, -czx)));
            sink(1, 0, 0, 0, t.x); sink(1, 1, 0, 0, t.y);
            t = __fmul2_rn(ayy, __ffma2_rn(X, make_float2(w1[2], w1[2]), make_float2(-czx, czx)));
            sink(1, 0, 0, 1, t.x); sink(1, 1, 0, 1, t.y);
            const float2 azz = make_float2(az, az);
            t = __fmul2_rn(azz, __ffma2_rn(X, make_float2(w0[1], w0[1]), make_float2(cxy, -cxy)));
            sink(2, 0, 0, 0, t.x); sink(2, 1, 0, 0, t.y);
            t = __fmul2_rn(azz, __ffma2_rn(X, make_float2(w1[1], w1[1]), make_float2(-cxy, cxy)));
            sink(2, 0, 1, 0, t.x); sink(2, 1, 1, 0, t.y);
        } else {
            const float cxy = D[0] * D[1] * (1.f / 12.f);
            t = __fmul2_rn(make_float2(ax, ax), Y);
            sink(0, 0, 0, 0, t.x); sink(0, 0, 1, 0, t.y);
            t = __fmul2_rn(make_float2(ay, ay), X);
            sink(1, 0, 0, 0, t.x); sink(1, 1, 0, 0, t.y);
            const float2 azz = make_float2(az, az);
            t = __fmul2_rn(azz, __ffma2_rn(X, make_float2(w0[1], w0[1]), make_float2(cxy, -cxy)));
            sink(2, 0, 0, 0, t.x); sink(2, 1, 0, 0, t.y);
            t = __fmul2_rn(azz, __ffma2_rn(X, make_float2(w1[1], w1[1]), make_float2(-cxy, cxy)));
            sink(2, 0, 1, 0, t.x); sink(2, 1, 1, 0, t.y);
        }
    } else if (NDIM == 3) {
        const R cyz = D[1] * D[2] * R(1.0 / 12.0), czx = D[2] * D[0] * R(1.0 / 12.0),
                cxy = D[0] * D[1] * R(1.0 / 12.0);
        // x faces (i+1/2, j+p, k+q)
        sink(0, 0, 0, 0, ax * (w0[1] * w0[2] + cyz));
        sink(0, 0, 1, 0, ax * (w1[1] * w0[2] - cyz));
        sink(0, 0, 0, 1, ax * (w0[1] * w1[2] - cyz));
        sink(0, 0, 1, 1, ax * (w1[1] * w1[2] + cyz));
        // y faces (i+q, j+1/2, k+p)
        sink(1, 0, 0, 0, ay * (w0[2] * w0[0] + czx));
        sink(1, 1, 0, 0, ay * (w0[2] * w1[0] - czx));
        sink(1, 0, 0, 1, ay * (w1[2] * w0[0] - czx));
        sink(1, 1, 0, 1, ay * (w1[2] * w1[0] + czx));
        // z faces (i+p, j+q, k+1/2)
        sink(2, 0, 0, 0, az * (w0[0] * w0[1] + cxy));
        sink(2, 1, 0, 0, az * (w1[0] * w0[1] - cxy));
        sink(2, 0, 1, 0, az * (w0[0] * w1[1] - cxy));
        sink(2, 1, 1, 0, az * (w1[0] * w1[1] + cxy));
    } else {
        const R cxy = D[0] * D[1] * R(1.0 / 12.0);
        sink(0, 0, 0, 0, ax * w0[1]);
        sink(0, 0, 1, 0, ax * w1[1]);
        sink(1, 0, 0, 0, ay * w0[0]);
        sink(1, 1, 0, 0, ay * w1[0]);
        sink(2, 0, 0, 0, az * (w0[0] * w0[1] + cxy));
        sink(2, 1, 0, 0, az * (w1[0] * w0[1] - cxy));
        sink(2, 0, 1, 0, az * (w0[0] * w1[1] - cxy));
        sink(2, 1, 1, 0, az * (w1[0] * w1[1] + cxy));
    }
}

// Straight path from offset d0 in the start cell to the stored end: per axis a,
// a shift s[a] in {-1,0,1} cells and the end offset d1[a] in the end cell.  The
// path is split at the node planes it crosses (at most one per axis); the
// pieces are taken in increasing crossing parameter, ties in axis order, and
// each piece lies in its own cell.  Positions at the breakpoints are the exact
// plane values and the stored end, so the piece displacements telescope to the
// stored total and charge is conserved up to the rounding of the fluxes.  dz2d
// is the out-of-plane displacement in 2D3V, shared between the pieces in
// proportion to their parameter length.
// init() sets up the split; piece(k, ...) must then be called for k = 0, 1, ...,
// ncross in this order and returns piece k: its cell offset from the start
// cell, its start offset and its displacement.  Two forms compute each value
// by the same arithmetic:
//  - PathSplitSelect (FP32, the mixed path's warps) has no data-dependent
//    branches: every candidate value is computed and the right one selected,
//    so the lanes of a warp whose particles cross different planes stay
//    converged;
//  - PathSplitBranch (FP64, one thread per particle, bound by GB300's FP64
//    pipe and its registers) branches, skipping the work of the axes that are
//    not crossed.
template <int NDIM, typename R>
struct PathSplitSelect {
    R cur[3], dv[3], tc[3], d1[3];
    int code;     // per axis a, bits 4a..4a+3: (s[a] + 1) | rank[a] << 2, rank 3 if the axis is not crossed
    int ncross;
    R tprev, dz;
    __device__ __forceinline__ int sh(int a) const { return ((code >> (4 * a)) & 3) - 1; }
    __device__ __forceinline__ int rk(int a) const { return (code >> (4 * a + 2)) & 3; }
    __device__ __forceinline__ void init(const R d0[3], const int s[3], const R d1_[3], R dz2d) {
        ncross = 0;
        code = 0;
        bool cr[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cur[a] = a < NDIM ? d0[a] : R(0);
            d1[a] = a < NDIM ? d1_[a] : R(0);
            const int sa = a < NDIM ? s[a] : 0;
            code |= (sa + 1) << (4 * a);
            cr[a] = a < NDIM && sa != 0;
            // crossing: the plane in start-cell coordinates, then the rest in end-cell coordinates
            const R plane = sa > 0 ? R(1) : R(0), pn = sa > 0 ? R(0) : R(1);
            const R first = plane - cur[a];
            const R dv_cross = first + (d1[a] - pn);
            const R q = div_<R>(first, dv_cross);   // selected away when the axis is not crossed
            dv[a] = a < NDIM ? (cr[a] ? dv_cross : d1[a] - cur[a]) : R(0);
            tc[a] = cr[a] ? (dv_cross != R(0) ? q : R(0)) : R(2);
            ncross += cr[a] ? 1 : 0;
        }
        // rank of each crossing among the crossings, ties by axis order (an axis
        // that is not crossed has tc = 2 and never counts below a crossing)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            int r = 0;
#pragma unroll
            for (int b = 0; b < 3; ++b)
                if (b != a) r += (tc[b] < tc[a] || (tc[b] == tc[a] && b < a)) ? 1 : 0;
            code |= (cr[a] ? r : 3) << (4 * a + 2);
        }
        tprev = R(0);
        dz = dz2d;
    }
    __device__ __forceinline__ void piece(int k, int c[3], R d[3], R D[3]) {
        R tn = R(1);
#pragma unroll
        for (int a = 0; a < NDIM; ++a) tn = rk(a) == k ? tc[a] : tn;
        const bool last = (k == ncross);
        const R dt = tn - tprev;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int ra = rk(a), sa = sh(a);
            c[a] = ra < k ? sa : 0;
            d[a] = cur[a];
            if (a >= NDIM) { D[a] = R(0); continue; }
            const R mid = snap_offset<R>(fma_<R>(dv[a], dt, cur[a]));
            const R endp = ra == k ? (sa > 0 ? R(1) : R(0)) : (last ? d1[a] : mid);
            D[a] = endp - cur[a];
            cur[a] = ra == k ? (sa > 0 ? R(0) : R(1)) : endp;
        }
        if (NDIM == 2) D[2] = dz * dt;
        tprev = tn;
    }
};

template <int NDIM, typename R>
struct PathSplitBranch {
    R cur[3], dv[3], tc[3], d1[3];
    int code;     // per axis a, bits 4a..4a+3: (s[a] + 1) | rank[a] << 2, rank 3 if the axis is not crossed
    int ncross;
    R tprev, dz;
    __device__ __forceinline__ int sh(int a) const { return ((code >> (4 * a)) & 3) - 1; }
    __device__ __forceinline__ int rk(int a) const { return (code >> (4 * a + 2)) & 3; }
    __device__ __forceinline__ R plo(int a) const { return sh(a) > 0 ? R(1) : R(0); }   // plane, start-cell coords
    __device__ __forceinline__ R pnew(int a) const { return sh(a) > 0 ? R(0) : R(1); }  // same plane, end-cell coords
    __device__ __forceinline__ void init(const R d0[3], const int s[3], const R d1_[3], R dz2d) {
        ncross = 0;
        code = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cur[a] = a < NDIM ? d0[a] : R(0);
            d1[a] = a < NDIM ? d1_[a] : R(0);
            tc[a] = R(2);
            dv[a] = R(0);
            const int sa = a < NDIM ? s[a] : 0;
            code |= (sa + 1) << (4 * a);
            if (a < NDIM) {
                if (sa != 0) {
                    const R first = (sa > 0 ? R(1) : R(0)) - cur[a];
                    dv[a] = first + (d1[a] - (sa > 0 ? R(0) : R(1)));
                    tc[a] = dv[a] != R(0) ? div_<R>(first, dv[a]) : R(0);
                    ++ncross;
                } else {
                    dv[a] = d1[a] - cur[a];
                }
            }
        }
        // rank of each crossing among the crossings, ties by axis order
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            int r = 3;
            if (a < NDIM && sh(a) != 0) {
                r = 0;
#pragma unroll
                for (int b = 0; b < NDIM; ++b)
                    if (b != a && sh(b) != 0 && (tc[b] < tc[a] || (tc[b] == tc[a] && b < a))) ++r;
            }
            code |= r << (4 * a + 2);
        }
        tprev = R(0);
        dz = dz2d;
    }
    __device__ __forceinline__ void piece(int k, int c[3], R d[3], R D[3]) {
        R tn = R(1);
#pragma unroll
        for (int a = 0; a < NDIM; ++a)
            if (rk(a) == k) tn = tc[a];
        const bool last = (k == ncross);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            c[a] = rk(a) < k ? sh(a) : 0;
            d[a] = cur[a];
            if (a >= NDIM) { D[a] = R(0); continue; }
            R endp;
            if (rk(a) == k) endp = plo(a);
            else if (last) endp = d1[a];
            else endp = snap_offset<R>(cur[a] + dv[a] * (tn - tprev));
            D[a] = endp - cur[a];
            cur[a] = rk(a) == k ? pnew(a) : endp;
        }
        if (NDIM == 2) D[2] = dz * (tn - tprev);
        tprev = tn;
    }
};


template <int NDIM, typename R>
using PathSplit = typename std::conditional<sizeof(R) == sizeof(float), PathSplitSelect<NDIM, R>,
                                            PathSplitBranch<NDIM, R>>::type;

// All pieces of the path, in order: sink.piece(k, di, dj, dk, d, D, alpha).
template <int NDIM, typename R, class Sink>
__device__ __forceinline__ void deposit_path(const R d0[3], const int s[3], const R d1[3], R dz2d, R alpha,
                                             Sink &sink) {
    PathSplit<NDIM, R> ps;
    ps.init(d0, s, d1, dz2d);
    // one rolled loop over the pieces keeps a single copy of the deposit in the
    // instruction stream; every array is still indexed by unrolled axes
#pragma unroll 1
    for (int k = 0; k <= ps.ncross; ++k) {
        int c[3];
        R d[3], D[3];
        ps.piece(k, c, d, D);
        sink.piece(k, c[0], c[1], c[2], d, D, alpha);
    }
}

// Adapter: a value sink (set_cell + operator()) that deposits every piece at once.
template <int NDIM, typename R, class ValueSink>
struct PieceDeposit {
    ValueSink &vs;
    __device__ __forceinline__ explicit PieceDeposit(ValueSink &v) : vs(v) {}
    __device__ __forceinline__ void piece(int, int di, int dj, int dk, const R d[3], const R D[3], R alpha) {
        vs.set_cell(di, dj, dk);
        deposit_segment<NDIM, R>(d, D, alpha, vs);
    }
};

}  // namespace pic
