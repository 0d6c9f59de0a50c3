// mj.cu -- drifting Maxwell-Juttner loader (Sect. 4.3, App. D, Eq. Jutt).
//
// For each particle index p the loader draws six uniforms from Philox-4x32-10
// (key = seed, counter = (p low, p high, call, species), two 32-bit words per
// double in (0,1)), then
//   position  uniform in the box, or x from the truncated sech^2((x-x0)/L)
//             density by its exact inverse cumulative distribution (App. C);
//   y         the momentum along the drift direction n, from the marginal
//             j_Y of Eq. distr_y: y = J^-1(w), found in s = asinh(y) by
//             bisection in a table of J (Gauss-Legendre on 4096 intervals,
//             built on the host in FP64) and Newton steps on the exact
//             density, J being re-integrated from the nearest table node;
//   u         from Eq. finding_u, l(a u) = w' l(a), l(x) = (1+x) e^-x,
//             a = mu Gamma0 sqrt(1+y^2), by Newton on t = a (u - 1);
//   p_perp    gamma_y sqrt(u^2-1) (cos phi, sin phi), phi uniform (undoing the
//             change of variables of App. D), in the plane orthogonal to n.
// All arithmetic of the momenta is FP64; the mixed path stores the result as
// cell + FP32 offset and FP32 momenta.
#include <algorithm>
#include <cmath>
#include <vector>

#include "mj_common.cuh"

namespace pic {

using namespace mjk;

// Host: table of the cumulative marginal for (theta, beta0).  Returns the
// table with F in host memory (caller uploads it).
void build_marginal_table(double theta, double beta0, int n, std::vector<double> &F, double &s0, double &h,
                          double &psi, double &Z) {
    const double mu = 1.0 / theta;
    const double G0 = 1.0 / std::sqrt(1.0 - beta0 * beta0);
    psi = std::atanh(beta0);
    Marg m{mu, G0, psi, 1.0};
    // support: the density in sigma falls below 1e-27 of its largest sampled value
    double S = std::acosh(1.0 + 60.0 / mu) + 1.0;
    for (int it = 0; it < 60; ++it) {
        double gmax = 0.0;
        for (int k = 0; k <= 4000; ++k) gmax = std::max(gmax, m.g(-S + 2.0 * S * k / 4000.0));
        if (m.g(-S) < 1e-27 * gmax && m.g(S) < 1e-27 * gmax) break;
        S *= 1.25;
    }
    s0 = -S;
    h = 2.0 * S / n;
    F.assign(n + 1, 0.0);
    double acc = 0.0;
    for (int k = 0; k < n; ++k) {
        acc += gl_integral(m, s0 + k * h, s0 + (k + 1) * h);
        F[k + 1] = acc;
    }
    Z = acc;
    for (auto &v : F) v /= Z;
    F[n] = 1.0;
}

void launch_load_mj(const Geom &g, int ndim, long long n, int species, unsigned long long seed, int profile, double L,
                    double x0, double theta, const double beta[3], int naive, const double *Fdev, double s0,
                    double h, int ntab, double psi, double Z, int colocate, Species64 d64, Species64 c64,
                    SpeciesMixed dmx, SpeciesMixed cmx, int mixed, int *err, cudaStream_t s) {
    LoadArgs a = make_load_args(g, ndim, n, species, seed, profile, L, x0, theta, beta, naive, Fdev, s0, h, ntab, psi,
                                Z, colocate, d64, c64, dmx, cmx, mixed, err);
    if (n <= 0) return;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 152LL * 16);
    k_load_mj<ExactPar><<<blocks, 256, 0, s>>>(a, ExactPar{});
}

}  // namespace pic
