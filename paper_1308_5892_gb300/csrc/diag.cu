// diag.cu -- FP64 diagnostics (Sect. 3.1 energies, Eq. Fourier k = 0 momentum,
// Gauss residual of Sect. 2.1): reductions over fields and particles, charge
// deposition onto the nodes (CIC, the same weights as the gather of App. A.3.3)
// and the discrete divergence of e.
#include "pic_internal.cuh"

namespace pic {

namespace {

template <int NV>
__device__ inline void block_sum_atomic(double (&v)[NV], double *acc) {
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

__device__ inline void atomic_max_nonneg(double *addr, double v) {
    // non-negative doubles order like their bit patterns as signed 64-bit integers
    atomicMax(reinterpret_cast<long long *>(addr), __double_as_longlong(v));
}

__device__ inline void block_max_atomic(double v, double *out) {
    __shared__ double red[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        double x = lane < nw ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
        if (lane == 0) atomic_max_nonneg(out, x);
    }
}

inline int blocks_for(long long n) {
    long long b = (n + 255) / 256;
    const long long cap = 152LL * 16;
    return (int)(b < 1 ? 1 : (b < cap ? b : cap));
}

__device__ inline long long interior_to_padded(const Geom &g, long long q) {
    const int i = (int)(q % g.nx);
    const long long r = q / g.nx;
    const int j = (int)(r % g.ny);
    const int k = (int)(r / g.ny);
    return g.pidx(i, j, k);
}

template <typename R>
__global__ void k_field_diag(Geom g, FieldPtrs<R> f, double *acc, unsigned long long *nonfinite) {
    const long long n = (long long)g.nx * g.ny * g.nz;
    double v[6] = {0, 0, 0, 0, 0, 0};
    unsigned long long bad = 0;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const long long p = interior_to_padded(g, q);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double e = e_full(f, c, p), b = (double)f.b[c][p];
            if (!isfinite(e)) ++bad;
            if (!isfinite(b)) ++bad;
            v[c] += e * e;
            v[3 + c] += b * b;
        }
    }
    if (bad) atomicAdd(nonfinite, bad);
    block_sum_atomic<6>(v, acc);
}

// acc: [0] sum (gamma-1), [1..3] sum u, [4] sum u.v, [5] count
__global__ void k_particle_diag64(Species64 sp, long long n, double *acc, unsigned long long *nonfinite) {
    double v[6] = {0, 0, 0, 0, 0, 0};
    unsigned long long bad = 0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const double ux = sp.u[0][p], uy = sp.u[1][p], uz = sp.u[2][p];
        const double u2 = ux * ux + uy * uy + uz * uz;
        const double gam = sqrt(1.0 + u2);
        if (!isfinite(u2) || !isfinite(sp.x[0][p]) || !isfinite(sp.x[1][p])) ++bad;
        v[0] += u2 / (1.0 + gam);
        v[1] += ux; v[2] += uy; v[3] += uz;
        v[4] += u2 / gam;
        v[5] += 1.0;
    }
    if (bad) atomicAdd(nonfinite, bad);
    block_sum_atomic<6>(v, acc);
}

__global__ void k_particle_diag_mixed(SpeciesMixed sp, long long n, double *acc, unsigned long long *nonfinite) {
    double v[6] = {0, 0, 0, 0, 0, 0};
    unsigned long long bad = 0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const double ux = sp.u[0][p], uy = sp.u[1][p], uz = sp.u[2][p];
        const double u2 = ux * ux + uy * uy + uz * uz;
        const double gam = sqrt(1.0 + u2);
        if (!isfinite(u2) || !isfinite(sp.off[0][p]) || !isfinite(sp.off[1][p])) ++bad;
        v[0] += u2 / (1.0 + gam);
        v[1] += ux; v[2] += uy; v[3] += uz;
        v[4] += u2 / gam;
        v[5] += 1.0;
    }
    if (bad) atomicAdd(nonfinite, bad);
    block_sum_atomic<6>(v, acc);
}

// rho~ at the nodes (interior array, wrapped): CIC weight alpha * prod(1-d or d).
template <int NDIM>
__device__ inline void rho_one(const Geom &g, int i, int j, int k, const double d[3], double alpha, double *rho) {
#pragma unroll
    for (int xi = 0; xi < (NDIM == 3 ? 2 : 1); ++xi)
#pragma unroll
        for (int eta = 0; eta < 2; ++eta)
#pragma unroll
            for (int eps = 0; eps < 2; ++eps) {
                double w = (eps ? d[0] : 1.0 - d[0]) * (eta ? d[1] : 1.0 - d[1]);
                if (NDIM == 3) w *= (xi ? d[2] : 1.0 - d[2]);
                const long long q = ((long long)g.wz(k + xi) * g.ny + g.wy(j + eta)) * g.nx + g.wx(i + eps);
                atomicAdd(rho + q, alpha * w);
            }
}

template <int NDIM>
__global__ void k_rho64(Geom g, Species64 sp, long long n, double alpha, double *rho) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        double d[3] = {0, 0, 0};
        int c[3] = {0, 0, 0};
        for (int a = 0; a < NDIM; ++a) {
            const double x = sp.x[a][p];
            const double f = floor(x);
            c[a] = (int)f;
            d[a] = x - f;
        }
        if (g.bcx == 1 && c[0] >= g.nx) { c[0] = g.nx - 1; d[0] = 1.0; }
        rho_one<NDIM>(g, c[0], c[1], c[2], d, alpha, rho);
    }
}

template <int NDIM>
__global__ void k_rho_mixed(Geom g, SpeciesMixed sp, long long n, double alpha, double *rho) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        unpack_cell(NDIM, sp.cell[p], i, j, k);
        double d[3] = {sp.off[0][p], sp.off[1][p], NDIM == 3 ? sp.off[2][p] : 0.0};
        rho_one<NDIM>(g, i, j, k, d, alpha, rho);
    }
}

// div e at the nodes (interior layout).
template <typename R>
__global__ void k_div_e(Geom g, FieldPtrs<R> f, double *out) {
    const long long n = (long long)g.nx * g.ny * g.nz;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % g.nx);
        const long long r = q / g.nx;
        const int j = (int)(r % g.ny);
        const int k = (int)(r / g.ny);
        const long long c = g.pidx(i, j, k);
        out[q] = (e_full(f, 0, c) - e_full(f, 0, g.widx(i - 1, j, k))) +
                 (e_full(f, 1, c) - e_full(f, 1, g.widx(i, j - 1, k))) +
                 (e_full(f, 2, c) - e_full(f, 2, g.widx(i, j, k - 1)));
    }
}

__global__ void k_max_abs_diff(const double *a, const double *b, long long n, double *out) {
    double m = 0.0;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        m = fmax(m, fabs(a[q] - (b ? b[q] : 0.0)));
    block_max_atomic(m, out);
}

}  // namespace

template <typename R>
void launch_field_diag(const Geom &g, FieldPtrs<R> f, double *acc, long long *nonfinite, cudaStream_t s) {
    k_field_diag<R><<<blocks_for((long long)g.nx * g.ny * g.nz), 256, 0, s>>>(
        g, f, acc, reinterpret_cast<unsigned long long *>(nonfinite));
}
template void launch_field_diag<float>(const Geom &, FieldPtrs<float>, double *, long long *, cudaStream_t);
template void launch_field_diag<double>(const Geom &, FieldPtrs<double>, double *, long long *, cudaStream_t);

void launch_particle_diag64(const Geom &g, Species64 sp, long long n, double m_over_me, double *acc,
                            long long *nonfinite, cudaStream_t s) {
    (void)g; (void)m_over_me;
    if (n > 0) k_particle_diag64<<<blocks_for(n), 256, 0, s>>>(sp, n, acc, reinterpret_cast<unsigned long long *>(nonfinite));
}

void launch_particle_diag_mixed(const Geom &g, SpeciesMixed sp, long long n, double m_over_me, double *acc,
                                long long *nonfinite, cudaStream_t s) {
    (void)g; (void)m_over_me;
    if (n > 0)
        k_particle_diag_mixed<<<blocks_for(n), 256, 0, s>>>(sp, n, acc, reinterpret_cast<unsigned long long *>(nonfinite));
}

template <typename R>
void launch_div_e(const Geom &g, FieldPtrs<R> f, double *out, cudaStream_t s) {
    k_div_e<R><<<blocks_for((long long)g.nx * g.ny * g.nz), 256, 0, s>>>(g, f, out);
}
template void launch_div_e<float>(const Geom &, FieldPtrs<float>, double *, cudaStream_t);
template void launch_div_e<double>(const Geom &, FieldPtrs<double>, double *, cudaStream_t);

void launch_rho64(const Geom &g, Species64 sp, long long n, double alpha, double *rho, cudaStream_t s) {
    if (n <= 0) return;
    if (g.ndim == 3) k_rho64<3><<<blocks_for(n), 256, 0, s>>>(g, sp, n, alpha, rho);
    else k_rho64<2><<<blocks_for(n), 256, 0, s>>>(g, sp, n, alpha, rho);
}

void launch_rho_mixed(const Geom &g, SpeciesMixed sp, long long n, double alpha, double *rho, cudaStream_t s) {
    if (n <= 0) return;
    if (g.ndim == 3) k_rho_mixed<3><<<blocks_for(n), 256, 0, s>>>(g, sp, n, alpha, rho);
    else k_rho_mixed<2><<<blocks_for(n), 256, 0, s>>>(g, sp, n, alpha, rho);
}

void launch_max_abs_diff(const double *a, const double *b, long long n, double *out_max, cudaStream_t s) {
    k_max_abs_diff<<<blocks_for(n), 256, 0, s>>>(a, b, n, out_max);
}

}  // namespace pic
