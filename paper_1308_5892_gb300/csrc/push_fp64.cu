// push_fp64.cu -- the plain FP64 particle kernel: one thread per particle,
// gather from global memory, Boris push, move, and charge-conserving deposit
// with global FP64 atomics (main loop steps 2, 3, 8, 9 of App. A.3.1).
//
// This is the double-precision baseline the mixed path is measured against.
// Roofline: per particle-step 40 B (2D) / 48 B (3D) read and written each, plus
// ~ (8 to 12) x segments FP64 atomics into L2 and ~300 FP64 flops, so on GB300
// (FP64 far below FP32) it is expected to be bound by the FP64 pipe and the
// atomics rather than by HBM.
#include "particle_core.cuh"
#include "pic_internal.cuh"

namespace pic {

namespace {

// Global-memory current sink: interior-wrapped padded index, FP64 atomics.
struct GlobalSink64 {
    const Geom *g;
    double *J[3];
    int ci, cj, ck, oi, oj, ok;
    __device__ void set_cell(int di, int dj, int dk) { oi = ci + di; oj = cj + dj; ok = ck + dk; }
    __device__ void operator()(int comp, int di, int dj, int dk, double v) {
        atomicAdd(J[comp] + g->widx_mod(oi + di, oj + dj, ok + dk), v);
    }
};

__device__ inline double sval64(const Geom &g, const double *a, bool xstag, int i, int j, int k) {
    if (g.bcx == 1) {
        if (xstag) { if (i < 0 || i > g.nx - 1) return 0.0; }
        else { if (i <= 0 || i >= g.nx) return 0.0; }
    }
    return __ldg(a + g.widx_mod(i, j, k));
}

// Node-averaged fields at node (i,j,k) (App. A.3.3).
__device__ inline void node64(const Geom &g, const FieldPtrs<double> &f, int i, int j, int k, double E[3],
                              double B[3]) {
    E[0] = 0.5 * (sval64(g, f.e[0], true, i - 1, j, k) + sval64(g, f.e[0], true, i, j, k));
    E[1] = 0.5 * (sval64(g, f.e[1], false, i, j - 1, k) + sval64(g, f.e[1], false, i, j, k));
    E[2] = 0.5 * (sval64(g, f.e[2], false, i, j, k - 1) + sval64(g, f.e[2], false, i, j, k));
    B[0] = 0.25 * (sval64(g, f.b[0], false, i, j, k) + sval64(g, f.b[0], false, i, j - 1, k) +
                   sval64(g, f.b[0], false, i, j, k - 1) + sval64(g, f.b[0], false, i, j - 1, k - 1));
    B[1] = 0.25 * (sval64(g, f.b[1], true, i, j, k) + sval64(g, f.b[1], true, i - 1, j, k) +
                   sval64(g, f.b[1], true, i, j, k - 1) + sval64(g, f.b[1], true, i - 1, j, k - 1));
    B[2] = 0.25 * (sval64(g, f.b[2], true, i, j, k) + sval64(g, f.b[2], true, i - 1, j, k) +
                   sval64(g, f.b[2], true, i - 1, j - 1, k) + sval64(g, f.b[2], true, i, j - 1, k));
}

template <int NDIM>
__device__ inline void gather64(const Geom &g, const FieldPtrs<double> &f, const int c[3], const double d[3],
                                double E[3], double B[3]) {
    E[0] = E[1] = E[2] = B[0] = B[1] = B[2] = 0.0;
#pragma unroll
    for (int xi = 0; xi < (NDIM == 3 ? 2 : 1); ++xi)
#pragma unroll
        for (int eta = 0; eta < 2; ++eta)
#pragma unroll
            for (int eps = 0; eps < 2; ++eps) {
                double w = (eps ? d[0] : 1.0 - d[0]) * (eta ? d[1] : 1.0 - d[1]);
                if (NDIM == 3) w *= (xi ? d[2] : 1.0 - d[2]);
                double En[3], Bn[3];
                node64(g, f, c[0] + eps, c[1] + eta, c[2] + xi, En, Bn);
#pragma unroll
                for (int q = 0; q < 3; ++q) { E[q] += w * En[q]; B[q] += w * Bn[q]; }
            }
}

__device__ inline void split64(double x, int n, bool conductor, int &c, double &d) {
    double f = floor(x);
    c = (int)f;
    d = x - f;
    if (conductor && c >= n) { c = n - 1; d = 1.0; }
}

template <int NDIM>
__global__ void __launch_bounds__(256, 2) k_push_fp64(Geom g, FieldPtrs<double> f, double *J0, double *J1, double *J2,
                                                   Species64 sp, long long n, double h, double alpha, double dt,
                                                   int mode, double m_over_me, double *kin_acc, int *err) {
    GlobalSink64 sink;
    sink.g = &g;
    sink.J[0] = J0; sink.J[1] = J1; sink.J[2] = J2;
    double kin0 = 0.0, kin1 = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
        double x[3] = {sp.x[0][p], sp.x[1][p], NDIM == 3 ? sp.x[2][p] : 0.0};
        double u[3] = {sp.u[0][p], sp.u[1][p], sp.u[2][p]};
        int c[3] = {0, 0, 0};
        double d[3] = {0.0, 0.0, 0.0};
        split64(x[0], g.nx, g.bcx == 1, c[0], d[0]);
        split64(x[1], g.ny, false, c[1], d[1]);
        if (NDIM == 3) split64(x[2], g.nz, false, c[2], d[2]);
        double E[3], B[3];
        gather64<NDIM>(g, f, c, d, E, B);
        const double gam0 = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        if (mode == 1) {   // initial staggering: one Boris step of -dt/2, no move
            boris<double>(u, E, B, h, -0.5 * dt);
            sp.u[0][p] = u[0]; sp.u[1][p] = u[1]; sp.u[2][p] = u[2];
            continue;
        }
        boris<double>(u, E, B, h, dt);
        const double inv_gam = 1.0 / sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        kin0 += gam0 - 1.0;
        kin1 += 1.0 / inv_gam - 1.0;
        double D[3] = {dt * u[0] * inv_gam, dt * u[1] * inv_gam, dt * u[2] * inv_gam};
        // conductor walls (App. A.4): specular reflection, deposit of the path
        // to the wall and of the mirrored remainder
        double xn = (double)c[0] + d[0] + D[0];
        const bool reflect = g.bcx == 1 && (xn < 0.0 || xn > (double)g.nx);
        int legs = 1;
        double dleg[2][3];
        double start[2][3];
        if (reflect) {
            const double wall = xn < 0.0 ? 0.0 : (double)g.nx;
            const double t = (wall - (c[0] + d[0])) / D[0];
            dleg[0][0] = wall - (c[0] + d[0]); dleg[0][1] = D[1] * t; dleg[0][2] = D[2] * t;
            dleg[1][0] = -(D[0] - dleg[0][0]); dleg[1][1] = D[1] - dleg[0][1]; dleg[1][2] = D[2] - dleg[0][2];
            start[0][0] = c[0] + d[0]; start[0][1] = c[1] + d[1]; start[0][2] = c[2] + d[2];
            start[1][0] = wall; start[1][1] = start[0][1] + dleg[0][1]; start[1][2] = start[0][2] + dleg[0][2];
            legs = 2;
            u[0] = -u[0];
        } else {
            for (int a = 0; a < 3; ++a) { dleg[0][a] = D[a]; start[0][a] = c[a] + d[a]; }
        }
        double endabs[3] = {0, 0, 0};
        for (int leg = 0; leg < legs; ++leg) {
            int c0[3] = {0, 0, 0}, s[3] = {0, 0, 0};
            double d0[3] = {0, 0, 0}, d1[3] = {0, 0, 0};
            for (int a = 0; a < NDIM; ++a) {
                const double st = start[leg][a];
                double fl = floor(st);
                // a leg that starts on a node plane and moves down starts at offset 1 of the lower cell
                if (st == fl && dleg[leg][a] < 0.0) fl -= 1.0;
                c0[a] = (int)fl;
                d0[a] = st - fl;
                const double pa = d0[a] + dleg[leg][a];
                double sa = floor(pa);
                double da = pa - sa;
                if (da >= 1.0) { da = 0.0; sa += 1.0; }
                if (!(sa >= -1.0 && sa <= 1.0)) {   // faster than one cell per step, or not finite
                    atomicOr(err, ERR_FAST_MOVE);
                    sa = 0.0;
                    da = d0[a];
                }
                s[a] = (int)sa;
                d1[a] = da;
                endabs[a] = (double)(c0[a] + s[a]) + da;
            }
            sink.ci = c0[0]; sink.cj = c0[1]; sink.ck = NDIM == 3 ? c0[2] : 0;
            PieceDeposit<NDIM, double, GlobalSink64> pd(sink);
            deposit_path<NDIM, double>(d0, s, d1, dleg[leg][2], alpha, pd);
        }
        // store: periodic wrap into [0, n)
        double xo = endabs[0];
        if (g.bcx == 0) { if (xo < 0.0) xo += g.nx; if (xo >= g.nx) xo -= g.nx; }
        double yo = endabs[1];
        if (yo < 0.0) yo += g.ny;
        if (yo >= g.ny) yo -= g.ny;
        sp.x[0][p] = xo;
        sp.x[1][p] = yo;
        if (NDIM == 3) {
            double zo = endabs[2];
            if (zo < 0.0) zo += g.nz;
            if (zo >= g.nz) zo -= g.nz;
            sp.x[2][p] = zo;
        }
        sp.u[0][p] = u[0]; sp.u[1][p] = u[1]; sp.u[2][p] = u[2];
    }
    if (kin_acc && mode == 0) {
        for (int o = 16; o > 0; o >>= 1) {
            kin0 += __shfl_xor_sync(0xffffffffu, kin0, o);
            kin1 += __shfl_xor_sync(0xffffffffu, kin1, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(kin_acc, m_over_me * kin0);
            atomicAdd(kin_acc + 1, m_over_me * kin1);
        }
    }
}

}  // namespace

void launch_push_fp64(const Geom &g, FieldPtrs<double> f, double *const J[3], Species64 sp, long long n, double h,
                      double alpha, double dt, int mode, double m_over_me, double *kin_acc, int *err,
                      cudaStream_t s) {
    if (n <= 0) return;
    long long blocks = (n + 255) / 256;
    if (blocks > 152LL * 8 * 64) blocks = 152LL * 8 * 64;
    if (g.ndim == 3)
        k_push_fp64<3><<<(int)blocks, 256, 0, s>>>(g, f, J[0], J[1], J[2], sp, n, h, alpha, dt, mode, m_over_me,
                                                   kin_acc, err);
    else
        k_push_fp64<2><<<(int)blocks, 256, 0, s>>>(g, f, J[0], J[1], J[2], sp, n, h, alpha, dt, mode, m_over_me,
                                                   kin_acc, err);
}

}  // namespace pic
