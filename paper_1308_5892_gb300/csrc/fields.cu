// fields.cu -- Yee FDTD field kernels (App. A.3.2) and the node-averaged fields
// used by the gather (App. A.3.3).
//
// Every kernel runs one thread per padded cell, ghosts included.  A thread
// computes the update of its cell from the interior images of the
// neighbours, so a ghost cell receives exactly the value of the interior cell
// it mirrors and the padded arrays stay periodic without a separate copy.
// Each thread reads its own cell and neighbours, and writes only its own cell,
// of arrays that are not read at neighbour positions in the same kernel, so
// no two threads race.
//
// Roofline: HBM bound.  Algorithmic bytes per cell: b advance 6 reads +
// 3 writes; e advance 6 + 3 (J) reads, 3 writes, 3 zero-writes; node fields 6
// reads + 8 writes, in units of sizeof(Real) (float4 pairs for node fields).
#include <type_traits>

#include "field_cells.cuh"
#include "pic_internal.cuh"

namespace pic {

namespace {

// b <- b - h curl e over every padded cell; with a history slot, the interior
// sums of e^2 and b^2 are added to it.
template <typename R>
__global__ void k_b_advance(Geom g, FieldPtrs<R> f, R h, HistRef hist) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    double *slot = hist.slot();
    double *energy_acc = slot ? slot + 2 : nullptr;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.pcells; p += stride)
        b_advance_cell<R>(g, f, h, p, energy_acc != nullptr, acc);
    if (energy_acc) block_accumulate<6>(acc, energy_acc);
}

// e <- e + dt curl b + J (Ampere, Eq. dyn4 with the deposited current, main
// loop steps 6, 11, 12), and zeroing of the other current buffer.
template <typename R>
__global__ void k_e_advance(Geom g, FieldPtrs<R> f, const R *J0, const R *J1, const R *J2, R *Z0, R *Z1, R *Z2,
                            R dt) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.pcells; p += stride) {
        int pi, pj, pk;
        padded_coords(g, p, pi, pj, pk);
        const int i = g.wx(pi - g.G), j = g.wy(pj - g.G), k = g.wz(pk - g.Gz);
        const long long c = g.pidx(i, j, k);
        const R bx = ld(f.b[0], c), by = ld(f.b[1], c), bz = ld(f.b[2], c);
        const R curl_x = (bz - ld(f.b[2], g.widx(i, j - 1, k))) - (by - ld(f.b[1], g.widx(i, j, k - 1)));
        const R curl_y = (bx - ld(f.b[0], g.widx(i, j, k - 1))) - (bz - ld(f.b[2], g.widx(i - 1, j, k)));
        const R curl_z = (by - ld(f.b[1], g.widx(i - 1, j, k))) - (bx - ld(f.b[0], g.widx(i, j - 1, k)));
        R ex = f.e[0][p] + dt * curl_x + folded_current(g, J0, i, j, k);
        R ey = f.e[1][p] + dt * curl_y + folded_current(g, J1, i, j, k);
        R ez = f.e[2][p] + dt * curl_z + folded_current(g, J2, i, j, k);
        if (g.bcx == 1 && i == 0) { ey = R(0); ez = R(0); }   // tangential e vanishes on the wall
        f.e[0][p] = ex;
        f.e[1][p] = ey;
        f.e[2][p] = ez;
        Z0[p] = R(0);
        Z1[p] = R(0);
        Z2[p] = R(0);
    }
}

__global__ void k_e_advance_fx(Geom g, FieldPtrs<float> f, const unsigned long long *J0,
                               const unsigned long long *J1, const unsigned long long *J2, unsigned long long *Z0,
                               unsigned long long *Z1, unsigned long long *Z2, float dt, F2 scale,
                               long long *hist_inc) {
    // no kernel of this launch reads the counter; the next step's kernels see the new value
    if (hist_inc && blockIdx.x == 0 && threadIdx.x == 0) *hist_inc += 1;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.pcells; p += stride)
        e_fx_cell(g, f, J0, J1, J2, Z0, Z1, Z2, dt, scale, p);
}

template <typename R, typename ZT, typename CT>
__global__ void k_e_advance_smoothed(Geom g, FieldPtrs<R> f, const CT *Js, double scale, ZT *Z0, ZT *Z1, ZT *Z2,
                                     R dt, long long *hist_inc) {
    if (hist_inc && blockIdx.x == 0 && threadIdx.x == 0) *hist_inc += 1;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.pcells; p += stride)
        e_smoothed_cell<R, ZT, CT>(g, f, Js, scale, Z0, Z1, Z2, dt, p);
}

__global__ void k_node_fields(Geom g, FieldPtrs<float> f, float4 *nfA, float2 *nfB) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.pcells; p += stride)
        node_cell(g, f, nfA, nfB, p);
}

// Batched over runs: block b belongs to the run r with block_prefix[r] <= b <
// block_prefix[r+1] and updates 256 padded cells of that run.
template <int PHASE>
__global__ void __launch_bounds__(256) k_fields_multi(const FieldRunF *runs, const int *block_prefix, int nruns,
                                                      float h, float dt) {
    __shared__ __align__(16) FieldRunF r;
    __shared__ int run_sh;
    if (threadIdx.x == 0) {
        int lo = 0, hi = nruns;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (block_prefix[mid] <= (int)blockIdx.x) lo = mid; else hi = mid;
        }
        run_sh = lo;
    }
    __syncthreads();
    {
        const int *src = reinterpret_cast<const int *>(runs + run_sh);
        int *dst = reinterpret_cast<int *>(&r);
        for (int q = threadIdx.x; q < (int)(sizeof(FieldRunF) / sizeof(int)); q += blockDim.x) dst[q] = src[q];
    }
    __syncthreads();
    const long long p = (long long)(blockIdx.x - block_prefix[run_sh]) * blockDim.x + threadIdx.x;
    const bool in = p < r.g.pcells;
    if (PHASE == FIELD_B_HALF) {
        double *slot = r.hist.slot();
        double *energy_acc = slot ? slot + 2 : nullptr;
        double acc[6] = {0, 0, 0, 0, 0, 0};
        if (in) b_advance_cell<float>(r.g, r.f, h, p, energy_acc != nullptr, acc);
        if (energy_acc) block_accumulate<6>(acc, energy_acc);
    } else if (PHASE == FIELD_NODE) {
        if (in) node_cell(r.g, r.f, r.nfA, r.nfB, p);
    } else {
        if (r.hist_inc && blockIdx.x == block_prefix[run_sh] && threadIdx.x == 0) *r.hist_inc += 1;
        if (in) {
            if (r.smooth > 0)
                e_smoothed_cell<float, unsigned long long, long long>(r.g, r.f, r.sbuf[r.smooth & 1], r.scale,
                                                                      r.Z[0], r.Z[1], r.Z[2], dt, p);
            else
                e_fx_cell(r.g, r.f, r.J[0], r.J[1], r.J[2], r.Z[0], r.Z[1], r.Z[2], dt,
                          F2{(float)r.scale, (float)(r.scale - (double)(float)r.scale)}, p);
        }
    }
}

template <typename R>
__global__ void k_add_uniform(Geom g, FieldPtrs<R> f, double e0, double e1, double e2, double b0, double b1,
                              double b2) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.pcells; p += stride) {
        int pi, pj, pk;
        padded_coords(g, p, pi, pj, pk);
        const int i = g.wx(pi - g.G);
        double v[6] = {e0, e1, e2, b0, b1, b2};
        if (g.bcx == 1 && i == 0) { v[1] = 0.0; v[2] = 0.0; v[3] = 0.0; }
        if constexpr (std::is_same<R, float>::value) {
            for (int c = 0; c < 3; ++c) {
                const double x = __dadd_rn(e_full(f, c, p), v[c]);
                const float hi = (float)x;
                f.e[c][p] = hi;
                f.el[c][p] = (float)(x - (double)hi);
            }
        } else {
            f.e[0][p] += (R)v[0]; f.e[1][p] += (R)v[1]; f.e[2][p] += (R)v[2];
        }
        f.b[0][p] += (R)v[3]; f.b[1][p] += (R)v[4]; f.b[2][p] += (R)v[5];
    }
}

inline int grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    const long long cap = 152LL * 16;   // 16 resident 256-thread blocks per SM on 152 SMs
    return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

}  // namespace

template <typename R>
void launch_b_advance(const Geom &g, FieldPtrs<R> f, R h, HistRef energy, cudaStream_t s) {
    k_b_advance<R><<<grid_for(g.pcells, 256), 256, 0, s>>>(g, f, h, energy);
}

template <typename R>
void launch_e_advance(const Geom &g, FieldPtrs<R> f, const R *const J[3], R *const Jzero[3], R dt,
                      cudaStream_t s) {
    k_e_advance<R><<<grid_for(g.pcells, 256), 256, 0, s>>>(g, f, J[0], J[1], J[2], Jzero[0], Jzero[1], Jzero[2],
                                                           dt);
}

void launch_node_fields(const Geom &g, FieldPtrs<float> f, float4 *nfA, float2 *nfB, cudaStream_t s) {
    k_node_fields<<<grid_for(g.pcells, 256), 256, 0, s>>>(g, f, nfA, nfB);
}

void launch_fields_multi(int phase, const FieldRunF *runs_dev, const int *block_prefix_dev, int nblocks, int nruns,
                         float h, float dt, cudaStream_t s) {
    if (phase == FIELD_B_HALF) k_fields_multi<FIELD_B_HALF><<<nblocks, 256, 0, s>>>(runs_dev, block_prefix_dev, nruns, h, dt);
    else if (phase == FIELD_NODE) k_fields_multi<FIELD_NODE><<<nblocks, 256, 0, s>>>(runs_dev, block_prefix_dev, nruns, h, dt);
    else k_fields_multi<FIELD_E_FX><<<nblocks, 256, 0, s>>>(runs_dev, block_prefix_dev, nruns, h, dt);
}

void launch_e_advance_fx(const Geom &g, FieldPtrs<float> f, const unsigned long long *const J[3],
                         unsigned long long *const Jzero[3], float dt, double alpha_abs, long long *hist_inc,
                         cudaStream_t s) {
    const double scale = alpha_abs * 0x1p-36;
    const F2 sc = {(float)scale, (float)(scale - (double)(float)scale)};
    k_e_advance_fx<<<grid_for(g.pcells, 256), 256, 0, s>>>(g, f, J[0], J[1], J[2], Jzero[0], Jzero[1], Jzero[2],
                                                           dt, sc, hist_inc);
}

template <typename R, typename ZT, typename CT>
void launch_e_advance_smoothed(const Geom &g, FieldPtrs<R> f, const CT *Js, double scale, ZT *const Jzero[3],
                               R dt, long long *hist_inc, cudaStream_t s) {
    k_e_advance_smoothed<R, ZT, CT><<<grid_for(g.pcells, 256), 256, 0, s>>>(g, f, Js, scale, Jzero[0], Jzero[1],
                                                                            Jzero[2], dt, hist_inc);
}

template <typename R>
void launch_add_uniform(const Geom &g, FieldPtrs<R> f, const double e0[3], const double b0[3], cudaStream_t s) {
    k_add_uniform<R><<<grid_for(g.pcells, 256), 256, 0, s>>>(g, f, e0[0], e0[1], e0[2], b0[0], b0[1], b0[2]);
}

template void launch_b_advance<float>(const Geom &, FieldPtrs<float>, float, HistRef, cudaStream_t);
template void launch_b_advance<double>(const Geom &, FieldPtrs<double>, double, HistRef, cudaStream_t);
template void launch_e_advance<float>(const Geom &, FieldPtrs<float>, const float *const[3], float *const[3], float,
                                      cudaStream_t);
template void launch_e_advance<double>(const Geom &, FieldPtrs<double>, const double *const[3], double *const[3],
                                       double, cudaStream_t);
template void launch_e_advance_smoothed<double, double, double>(const Geom &, FieldPtrs<double>, const double *,
                                                               double, double *const[3], double, long long *,
                                                               cudaStream_t);
template void launch_e_advance_smoothed<float, unsigned long long, long long>(const Geom &, FieldPtrs<float>,
                                                                              const long long *, double,
                                                                              unsigned long long *const[3], float,
                                                                              long long *, cudaStream_t);
template void launch_add_uniform<float>(const Geom &, FieldPtrs<float>, const double[3], const double[3],
                                        cudaStream_t);
template void launch_add_uniform<double>(const Geom &, FieldPtrs<double>, const double[3], const double[3],
                                         cudaStream_t);

}  // namespace pic
