// mj_common.cuh -- device parts of the drifting Maxwell-Juttner loader shared
// by the exact sampler (mj.cu) and the learned sampler (mlp.cu): Philox
// streams, the tabulated marginal and its inversion, the conditional of
// Eq. finding_u, and the particle assembly kernel.
#pragma once
#include <cmath>

#include "pic_internal.cuh"

namespace pic {
namespace mjk {

// ---------------------------------------------------------------- Philox-4x32-10

struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox_round(U4 c, uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    return U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
}

__device__ inline U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        c = philox_round(c, k0, k1);
    }
    return c;
}

__device__ __forceinline__ double to_unit(uint32_t hi, uint32_t lo) {
    const unsigned long long m = ((unsigned long long)(hi >> 5) << 26) + (unsigned long long)(lo >> 6);
    return ((double)m + 0.5) * 0x1p-53;
}

__device__ inline void uniforms6(unsigned long long seed, int species, long long p, double w[6]) {
    const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFull), k1 = (uint32_t)(seed >> 32);
    for (int call = 0; call < 3; ++call) {
        const U4 r = philox4x32_10(U4{(uint32_t)(p & 0xFFFFFFFFll), (uint32_t)((unsigned long long)p >> 32),
                                      (uint32_t)call, (uint32_t)species},
                                   k0, k1);
        w[2 * call] = to_unit(r.x, r.y);
        w[2 * call + 1] = to_unit(r.z, r.w);
    }
}

// ---------------------------------------------------------------- marginal in s = asinh(y)

// density of sigma = s - psi, up to the normalisation Z of the table:
// (1 + mu G0 cosh s) cosh s exp(-2 mu sinh^2(sigma/2)),  s = sigma + psi
struct Marg {
    double mu, G0, psi, Z;
    __host__ __device__ double g(double sig) const {
        const double cs = cosh(sig + psi);
        const double sh = sinh(0.5 * sig);
        return (1.0 + mu * G0 * cs) * cs * exp(-2.0 * mu * sh * sh) / Z;
    }
};

// 8-point Gauss-Legendre nodes and weights on [-1, 1]
__host__ __device__ inline double gl_x(int i) {
    const double x[4] = {0.1834346424956498, 0.5255324099163290, 0.7966664774136267, 0.9602898564975363};
    return i < 4 ? -x[3 - i] : x[i - 4];
}
__host__ __device__ inline double gl_w(int i) {
    const double w[4] = {0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};
    return i < 4 ? w[3 - i] : w[i - 4];
}

__host__ __device__ inline double gl_integral(const Marg &m, double a, double b) {
    const double c = 0.5 * (a + b), h = 0.5 * (b - a);
    double s = 0.0;
    for (int i = 0; i < 8; ++i) s += gl_w(i) * m.g(c + h * gl_x(i));
    return s * h;
}

struct Table {
    Marg m;
    double s0, h;       // sigma_k = s0 + k h
    int n;              // intervals
    const double *F;    // n + 1 cumulative values, F[0] = 0, F[n] = 1
};

__device__ inline double inverse_marginal(const Table &t, double w) {
    int lo = 0, hi = t.n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (t.F[mid] <= w) lo = mid; else hi = mid;
    }
    const double a = t.s0 + lo * t.h;
    const double Fa = t.F[lo], Fb = t.F[lo + 1];
    double sig = a + (Fb > Fa ? (w - Fa) / (Fb - Fa) : 0.5) * t.h;
    for (int it = 0; it < 4; ++it) {
        const double F = Fa + gl_integral(t.m, a, sig);
        const double g = t.m.g(sig);
        if (!(g > 0.0)) break;
        double nxt = sig - (F - w) / g;
        nxt = fmin(fmax(nxt, a), a + t.h);
        sig = nxt;
    }
    return sinh(sig + t.m.psi);
}

// t = a (u - 1) >= 0 from l(a + t) = w l(a) (Eq. finding_u), written as
// log1p(t / (1 + a)) - t = log w and solved by Newton from t = -log w (the
// large-a limit); the function is concave and decreasing in t, so the steps
// converge monotonically once on the right of the root.
__device__ inline double conditional_t(double a, double w) {
    const double lw = log(w);
    double t = -lw;
    for (int it = 0; it < 60; ++it) {
        const double f = log1p(t / (1.0 + a)) - t - lw;
        const double fp = 1.0 / (1.0 + a + t) - 1.0;
        double nt = t - f / fp;
        if (nt < 0.0) nt = 0.5 * t;
        const bool done = fabs(nt - t) <= 1e-16 * (nt + 1e-300);
        t = nt;
        if (done) break;
    }
    return t;
}

struct LoadArgs {
    Geom g;
    int ndim;
    long long n;
    int species;
    unsigned long long seed;
    int profile;
    double L, x0;
    double theta;
    double sb0;                 // drift speed the momenta are sampled with (0 for the naive control)
    double beta0;               // drift speed of the distribution
    double nvec[3], e1[3], e2[3];
    int naive;                  // rest-frame sample boosted particle by particle
    Table tab;
    int colocate;               // positions copied from src_* arrays
    // FP64 destination
    double *x64[3], *u64[3];
    const double *cx64[3];
    // mixed destination
    SpeciesMixed mx;
    SpeciesMixed cmx;
    int mixed;
    int *err;
};

// Drift-component samplers: the exact inverse of the tabulated marginal, or
// the learned network (mlp.cu).
struct ExactPar {
    __device__ double operator()(const LoadArgs &a, double w) const { return inverse_marginal(a.tab, w); }
};

template <class Par>
__global__ void k_load_mj(LoadArgs a, Par par_of) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < a.n; p += (long long)gridDim.x * blockDim.x) {
        double w[6];
        uniforms6(a.seed, a.species, p, w);
        // momentum along n and in the orthogonal plane
        const double y = par_of(a, w[3]);
        const double mu = 1.0 / a.theta;
        const double G0 = 1.0 / sqrt(1.0 - a.sb0 * a.sb0);
        const double gy = sqrt(1.0 + y * y);
        const double aa = mu * G0 * gy;
        const double um1 = conditional_t(aa, w[4]) / aa;   // u - 1
        const double r = sqrt(um1 * (um1 + 2.0));
        double sphi, cphi;
        sincospi(2.0 * w[5], &sphi, &cphi);
        double par = y, q1 = gy * r * cphi, q2 = gy * r * sphi;
        if (a.naive) {
            // the same sample drawn at rest (its table was built with beta0 = 0), then boosted
            const double g0 = sqrt(1.0 + par * par + q1 * q1 + q2 * q2);
            const double Gb = 1.0 / sqrt(1.0 - a.beta0 * a.beta0);
            par = Gb * (par + a.beta0 * g0);
        }
        double mom[3];
        for (int c = 0; c < 3; ++c) mom[c] = a.nvec[c] * par + a.e1[c] * q1 + a.e2[c] * q2;
        // position
        double pos[3] = {0.0, 0.0, 0.0};
        if (!a.colocate) {
            pos[0] = a.g.nx * w[0];
            pos[1] = a.g.ny * w[1];
            if (a.ndim == 3) pos[2] = a.g.nz * w[2];
            if (a.profile == 1) {
                const double ta = tanh(-a.x0 / a.L), tb = tanh((a.g.nx - a.x0) / a.L);
                pos[0] = a.x0 + a.L * atanh(ta + w[0] * (tb - ta));
                pos[0] = fmin(fmax(pos[0], 0.0), (double)a.g.nx);
            }
        }
        if (!a.mixed) {
            for (int c = 0; c < 3; ++c) {
                if (a.colocate) pos[c] = a.cx64[c][p];
                a.x64[c][p] = pos[c];
                a.u64[c][p] = mom[c];
            }
            if (a.g.bcx == 0 && a.x64[0][p] >= a.g.nx) a.x64[0][p] = 0.0;
            if (a.x64[1][p] >= a.g.ny) a.x64[1][p] = 0.0;
            if (a.ndim == 3 && a.x64[2][p] >= a.g.nz) a.x64[2][p] = 0.0;
        } else {
            if (a.colocate) {
                a.mx.cell[p] = a.cmx.cell[p];
                a.mx.off[0][p] = a.cmx.off[0][p];
                a.mx.off[1][p] = a.cmx.off[1][p];
                if (a.ndim == 3) a.mx.off[2][p] = a.cmx.off[2][p];
            } else {
                int ci[3] = {0, 0, 0};
                float of[3] = {0.f, 0.f, 0.f};
                const int n3[3] = {a.g.nx, a.g.ny, a.g.nz};
                for (int c = 0; c < a.ndim; ++c) {
                    const double f = floor(pos[c]);
                    int k = (int)f;
                    // the offset on the 2^-24 grid of the mixed path (see snap_offset)
                    float o = (float)(rint((pos[c] - f) * 16777216.0) * (1.0 / 16777216.0));
                    if (o >= 1.0f) { o = 0.0f; k += 1; }
                    if (c == 0 && a.g.bcx == 1 && k >= n3[0]) { k = n3[0] - 1; o = 1.0f; }
                    else if (k >= n3[c]) k -= n3[c];
                    ci[c] = k;
                    of[c] = o;
                }
                a.mx.cell[p] = pack_cell(a.ndim, ci[0], ci[1], ci[2]);
                a.mx.off[0][p] = of[0];
                a.mx.off[1][p] = of[1];
                if (a.ndim == 3) a.mx.off[2][p] = of[2];
            }
            a.mx.u[0][p] = (float)mom[0];
            a.mx.u[1][p] = (float)mom[1];
            a.mx.u[2][p] = (float)mom[2];
            a.mx.id[p] = (int32_t)p;
        }
    }
}

inline LoadArgs make_load_args(const Geom &g, int ndim, long long n, int species, unsigned long long seed, int profile,
                               double L, double x0, double theta, const double beta[3], int naive, const double *Fdev,
                               double s0, double h, int ntab, double psi, double Z, int colocate, Species64 d64,
                               Species64 c64, SpeciesMixed dmx, SpeciesMixed cmx, int mixed, int *err) {
    LoadArgs a{};
    a.g = g;
    a.ndim = ndim;
    a.n = n;
    a.species = species;
    a.seed = seed;
    a.profile = profile;
    a.L = L;
    a.x0 = x0;
    a.theta = theta;
    const double b0 = std::sqrt(beta[0] * beta[0] + beta[1] * beta[1] + beta[2] * beta[2]);
    a.beta0 = b0;
    a.sb0 = naive ? 0.0 : b0;
    double nv[3] = {0.0, 0.0, 1.0};
    if (b0 > 0) for (int c = 0; c < 3; ++c) nv[c] = beta[c] / b0;
    double av[3] = {1.0, 0.0, 0.0};
    if (!(std::fabs(nv[0]) < 0.9)) { av[0] = 0.0; av[1] = 1.0; }
    const double dot = av[0] * nv[0] + av[1] * nv[1] + av[2] * nv[2];
    double e1[3] = {av[0] - dot * nv[0], av[1] - dot * nv[1], av[2] - dot * nv[2]};
    const double ne = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    for (int c = 0; c < 3; ++c) e1[c] /= ne;
    const double e2[3] = {nv[1] * e1[2] - nv[2] * e1[1], nv[2] * e1[0] - nv[0] * e1[2], nv[0] * e1[1] - nv[1] * e1[0]};
    for (int c = 0; c < 3; ++c) { a.nvec[c] = nv[c]; a.e1[c] = e1[c]; a.e2[c] = e2[c]; }
    a.naive = naive;
    const double mu = 1.0 / theta;
    const double G0 = naive ? 1.0 : 1.0 / std::sqrt(1.0 - b0 * b0);
    a.tab.m = Marg{mu, G0, psi, Z};
    a.tab.s0 = s0;
    a.tab.h = h;
    a.tab.n = ntab;
    a.tab.F = Fdev;
    a.colocate = colocate;
    for (int c = 0; c < 3; ++c) {
        a.x64[c] = d64.x[c];
        a.u64[c] = d64.u[c];
        a.cx64[c] = c64.x[c];
    }
    a.mx = dmx;
    a.cmx = cmx;
    a.mixed = mixed;
    a.err = err;
    return a;
}


}  // namespace mjk
}  // namespace pic
