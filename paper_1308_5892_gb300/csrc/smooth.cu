// smooth.cu -- current smoothing (App. A.3.4, main-loop step 10).
//
// One pass replaces the current of every cell by the weighted mean of its
// 3x3x3 neighbourhood: weight 1 for the cell, 1/2, 1/4 and 1/8 for the
// neighbours shifted in one, two and three indices, divided by their sum 8.
// That is the product over the axes of the 1-2-1 stencil (1/4, 1/2, 1/4), and
// each thread evaluates it in that factored form: rows along x, then y, then
// z, each as (a[-1] + 2 a[0]) + a[+1].  In 2D3V the z factor is the identity
// (a z-independent field).
//
// Arithmetic.  The mixed path's current is an int64 fixed-point sum (units of
// 2^-36 of sgn(q) times the volume flux); a pass forms the weighted sum
// exactly in int64 and rounds it once to the same units, (S + 32) >> 6 in 3D
// and (S + 8) >> 4 in 2D (|S| < 2^53 for any current the push can deposit).
// The result is a deterministic function of the exact current, so it does not
// depend on the order of the particles.  The FP64 path smooths in FP64 in the
// same order.  (Integer arithmetic also keeps the mixed path off GB300's FP64
// pipe, which the stencil would otherwise saturate.)
//
// Data flow of a smoothed step (one run).  The deposit fills the padded
// current J, ghost images included.  k_fold_shell adds the ghost images of
// every interior cell within G of an edge into that cell, in place (J is
// consumed by this step; the e advance of the next step zeroes it).  The first
// pass reads the interior of J and writes a compact array indexed
// (k*ny + j)*nx + i; later passes map compact arrays.  The e advance reads the
// last one.  The batched form for ensembles folds every image into a compact
// array first (k_smooth_multi phase 0) and then smooths compact arrays, with
// the same values.
//
// Roofline: HBM.  Algorithmic bytes per interior cell and pass: 3 x 8 B read +
// 3 x 8 B written (neighbours in x and y come from L1/L2, the z neighbours from
// registers of the thread walking the column); the shell fold touches only the
// 2G-wide boundary layers.
#include <algorithm>

#include "pic_internal.cuh"
#include "smooth_cells.cuh"

namespace pic {

namespace {

constexpr int kRowThreads = 128;   // largest block along x of the row kernels
constexpr int kColumn = 16;        // z planes walked by one thread of k_smooth_cols

// Interior cells within G of an edge receive the sum of their ghost images, in
// place.  Grid (ceil(nx/bx), ny, nz) of bx threads.  A thread reads only ghost
// cells and writes only its own interior cell, so threads do not race.
template <typename JT>
__global__ void __launch_bounds__(kRowThreads) k_fold_shell(Geom g, JT *J0, JT *J1, JT *J2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.nx) return;
    const int j = blockIdx.y, k = blockIdx.z;
    const bool edge = i < g.G || i >= g.nx - g.G || j < g.G || j >= g.ny - g.G ||
                      (g.ndim == 3 && (k < g.Gz || k >= g.nz - g.Gz));
    if (!edge) return;
    const long long c = g.pidx(i, j, k);
#pragma unroll 1
    for (int q = 0; q < 3; ++q) {
        JT *const Jq = q == 0 ? J0 : (q == 1 ? J1 : J2);
        Jq[c] += image_sum<JT>(g, Jq, i, j, k, true);
    }
}

// One smoothing pass of planes in0..in2 into the compact planes out, grid
// (ceil(nx/bx), ny, nplanes * ceil(nz/kColumn)) of bx threads.  A thread walks
// up to kColumn z planes of one (i, j) column and keeps the x-y sums of the
// planes k-1, k, k+1 in registers, so that every plane's 3x3 sum is loaded
// once per column instead of three times.  Same arithmetic as smooth_cell.
template <typename T, typename V>
__global__ void __launch_bounds__(kRowThreads) k_smooth_cols(Geom g, V in0, V in1, V in2, T *out, int zchunks) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.nx) return;
    const int j = blockIdx.y;
    const int q = blockIdx.z / zchunks, zc = blockIdx.z - q * zchunks;
    const V v{q == 0 ? in0.a : (q == 1 ? in1.a : in2.a)};
    T *o = out + (long long)q * g.nx * g.ny * g.nz;
    const XYIndex x(g, i, j);
    if (g.ndim == 2) {
        o[(long long)j * g.nx + i] = norm16(xy_sum<T>(g, v, x, 0));
        return;
    }
    const int k0 = zc * kColumn, k1 = min(k0 + kColumn, g.nz);
    T pm = xy_sum<T>(g, v, x, k0 == 0 ? g.nz - 1 : k0 - 1);
    T p0 = xy_sum<T>(g, v, x, k0);
    for (int k = k0; k < k1; ++k) {
        const T pp = xy_sum<T>(g, v, x, k == g.nz - 1 ? 0 : k + 1);
        o[((long long)k * g.ny + j) * g.nx + i] = norm64((pm + (p0 + p0)) + pp);
        pm = p0;
        p0 = pp;
    }
}

// Batched over runs (mixed path), with the block map of the field kernels
// (block_prefix counts 256-cell blocks of every run's padded grid, which covers
// its interior).  PHASE 0 writes the folded current of every smoothing run to
// sbuf[0]; PHASE 1 is smoothing pass `pass` (0-based) of the runs that smooth
// more than `pass` times.
template <int PHASE>
__global__ void __launch_bounds__(256) k_smooth_multi(const FieldRunF *runs, const int *block_prefix, int nruns,
                                                      int pass) {
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
    const FieldRunF &r = runs[run_sh];
    if (r.smooth <= pass) return;
    const Geom g = r.g;
    const long long ncell = (long long)g.nx * g.ny * g.nz;
    const long long c = (long long)(blockIdx.x - block_prefix[run_sh]) * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    if (PHASE == 0) {
        int i, j, k;
        compact_coords(g, c, i, j, k);
        for (int q = 0; q < 3; ++q)
            r.sbuf[0][q * ncell + c] = (long long)image_sum<unsigned long long>(g, r.J[q], i, j, k, false);
    } else {
        for (int q = 0; q < 3; ++q)
            smooth_cell<long long>(g, r.sbuf[pass & 1] + q * ncell, r.sbuf[(pass + 1) & 1] + q * ncell, c);
    }
}

// threads along x: the row length rounded up to a warp, at most kRowThreads
int row_threads(const Geom &g) { return std::min(kRowThreads, (g.nx + 31) / 32 * 32); }

template <typename T, typename V>
void launch_cols(const Geom &g, V in0, V in1, V in2, T *out, int nplanes, cudaStream_t s) {
    const int bx = row_threads(g);
    const int zchunks = g.ndim == 3 ? (g.nz + kColumn - 1) / kColumn : 1;
    const dim3 grid((g.nx + bx - 1) / bx, g.ny, nplanes * zchunks);
    k_smooth_cols<T, V><<<grid, bx, 0, s>>>(g, in0, in1, in2, out, zchunks);
}

}  // namespace

template <typename JT>
const typename SmoothValue<JT>::type *launch_smooth_current(const Geom &g, JT *const J[3], int passes,
                                                            typename SmoothValue<JT>::type *const buf[2],
                                                            cudaStream_t s) {
    typedef typename SmoothValue<JT>::type T;
    if (g.G > 0 || g.Gz > 0) {
        const int bx = row_threads(g);
        const dim3 grid((g.nx + bx - 1) / bx, g.ny, g.nz);
        k_fold_shell<JT><<<grid, bx, 0, s>>>(g, J[0], J[1], J[2]);
    }
    launch_cols<T>(g, PaddedPlane<JT>{J[0]}, PaddedPlane<JT>{J[1]}, PaddedPlane<JT>{J[2]}, buf[0], 3, s);
    const long long ncell = (long long)g.nx * g.ny * g.nz;
    for (int p = 1; p < passes; ++p) {
        const T *in = buf[(p - 1) & 1];
        launch_cols<T>(g, CompactPlane<T>{in}, CompactPlane<T>{in + ncell}, CompactPlane<T>{in + 2 * ncell},
                       buf[p & 1], 3, s);
    }
    return buf[(passes - 1) & 1];
}

void launch_smooth(const Geom &g, const double *in, double *out, cudaStream_t s) {
    launch_cols<double>(g, CompactPlane<double>{in}, CompactPlane<double>{in}, CompactPlane<double>{in}, out, 1, s);
}

void launch_smooth_multi(int phase, int pass, const FieldRunF *runs_dev, const int *block_prefix_dev, int nblocks,
                         int nruns, cudaStream_t s) {
    if (phase == 0) k_smooth_multi<0><<<nblocks, 256, 0, s>>>(runs_dev, block_prefix_dev, nruns, pass);
    else k_smooth_multi<1><<<nblocks, 256, 0, s>>>(runs_dev, block_prefix_dev, nruns, pass);
}

template const double *launch_smooth_current<double>(const Geom &, double *const[3], int, double *const[2],
                                                    cudaStream_t);
template const long long *launch_smooth_current<unsigned long long>(const Geom &, unsigned long long *const[3], int,
                                                                   long long *const[2], cudaStream_t);

}  // namespace pic
