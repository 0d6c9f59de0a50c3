// smooth.cu -- current smoothing (App. A.3.4, main-loop step 10).
//
// One pass replaces the current of every cell by the weighted mean of its
// 3x3x3 neighbourhood: weight 1 for the cell, 1/2, 1/4 and 1/8 for the
// neighbours shifted in one, two and three indices, divided by their sum 8.
// That is the product over the axes of the 1-2-1 stencil (1/4, 1/2, 1/4), and
// each thread evaluates it in that factored form: rows along x, then y, then
// z.  In 2D3V the z factor is the identity (a z-independent field).
//
// Data flow of a smoothed step (one run).  The deposit fills the padded
// current J, ghost images included.  k_fold_shell adds the ghost images of
// every interior cell within G of an edge into that cell, in place (J is
// consumed by this step; the e advance of the next step zeroes it).  The first
// pass reads the interior of J, converted to FP64 (exact: the fixed-point sums
// of the mixed path stay far below 2^53 units), and writes a compact FP64
// array indexed (k*ny + j)*nx + i; later passes map compact arrays.  The e
// advance reads the last one.  The mixed current is an exact integer sum up to
// the first pass, so the smoothed current does not depend on the order of the
// particles; the passes run in a fixed order.
//
// The batched form for ensembles folds every image into a compact array first
// (k_smooth_multi phase 0) and then smooths compact arrays; it gives the same
// values.
//
// Roofline: HBM.  Algorithmic bytes per interior cell and pass: 3 x 8 B read +
// 3 x 8 B written (neighbours in x and y come from L1/L2, the z neighbours from
// registers of the thread walking the column); the shell fold touches only the
// 2G-wide boundary layers.
#include "pic_internal.cuh"

namespace pic {

namespace {

__device__ inline void compact_coords(const Geom &g, long long c, int &i, int &j, int &k) {
    i = (int)(c % g.nx);
    const long long q = c / g.nx;
    j = (int)(q % g.ny);
    k = (int)(q / g.ny);
}

__device__ inline double as_double(unsigned long long v) { return (double)(long long)v; }
__device__ inline double as_double(double v) { return v; }

// Sum of J over every padded image of interior cell (i,j,k), in J's own type
// (modular int64 arithmetic for the fixed-point current: exact).
template <typename JT>
__device__ inline double folded(const Geom &g, const JT *J, int i, int j, int k) {
    JT s = JT(0);
    const int zlo = g.ndim == 3 ? -1 : 0, zhi = g.ndim == 3 ? 1 : 0;
    for (int mz = zlo; mz <= zhi; ++mz) {
        const int qk = k + g.Gz + mz * g.nz;
        if (qk < 0 || qk >= g.pz) continue;
        for (int my = -1; my <= 1; ++my) {
            const int qj = j + g.G + my * g.ny;
            if (qj < 0 || qj >= g.py) continue;
            for (int mx = -1; mx <= 1; ++mx) {
                const int qi = i + g.G + mx * g.nx;
                if (qi < 0 || qi >= g.px) continue;
                s += J[((long long)qk * g.py + qj) * g.px + qi];
            }
        }
    }
    return as_double(s);
}

template <typename JT>
__device__ inline void fold_cell(const Geom &g, const JT *const J[3], double *out, long long ncell, long long c) {
    int i, j, k;
    compact_coords(g, c, i, j, k);
#pragma unroll
    for (int q = 0; q < 3; ++q) out[q * ncell + c] = folded<JT>(g, J[q], i, j, k);
}

// x-y part of the stencil at (i, j) of plane kk of compact array a:
// rows (a[i-1] + 2 a[i]) + a[i+1], then (row[j-1] + 2 row[j]) + row[j+1].
struct XYStencil {
    int i, im, ip, j, jm, jp;
    __device__ inline XYStencil(const Geom &g, int i_, int j_) : i(i_), j(j_) {
        im = i == 0 ? g.nx - 1 : i - 1;
        ip = i == g.nx - 1 ? 0 : i + 1;
        jm = j == 0 ? g.ny - 1 : j - 1;
        jp = j == g.ny - 1 ? 0 : j + 1;
    }
    __device__ inline double row(const Geom &g, const double *a, int jj, int kk) const {
        const double *r = a + ((long long)kk * g.ny + jj) * g.nx;
        return (__ldg(r + im) + 2.0 * __ldg(r + i)) + __ldg(r + ip);
    }
    __device__ inline double plane(const Geom &g, const double *a, int kk) const {
        return (row(g, a, jm, kk) + 2.0 * row(g, a, j, kk)) + row(g, a, jp, kk);
    }
};

// One smoothing pass of cell c of one compact plane a, written to out[c]
// (the per-cell form of the batched kernel; k_smooth_cols gives the same values).
__device__ inline void smooth_cell(const Geom &g, const double *a, double *out, long long c) {
    int i, j, k;
    compact_coords(g, c, i, j, k);
    const XYStencil st(g, i, j);
    double v;
    if (g.ndim == 3) {
        const int km = k == 0 ? g.nz - 1 : k - 1, kp = k == g.nz - 1 ? 0 : k + 1;
        v = ((st.plane(g, a, km) + 2.0 * st.plane(g, a, k)) + st.plane(g, a, kp)) * 0.015625;   // / 64
    } else {
        v = st.plane(g, a, k) * 0.0625;                                                          // / 16
    }
    out[c] = v;
}

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
    const int zlo = g.ndim == 3 ? -1 : 0, zhi = g.ndim == 3 ? 1 : 0;
#pragma unroll 1
    for (int q = 0; q < 3; ++q) {
        JT *const Jq = q == 0 ? J0 : (q == 1 ? J1 : J2);
        JT s = JT(0);
        for (int mz = zlo; mz <= zhi; ++mz) {
            const int qk = k + g.Gz + mz * g.nz;
            if (qk < 0 || qk >= g.pz) continue;
            for (int my = -1; my <= 1; ++my) {
                const int qj = j + g.G + my * g.ny;
                if (qj < 0 || qj >= g.py) continue;
                for (int mx = -1; mx <= 1; ++mx) {
                    const int qi = i + g.G + mx * g.nx;
                    if (qi < 0 || qi >= g.px || (mx == 0 && my == 0 && mz == 0)) continue;
                    s += Jq[((long long)qk * g.py + qj) * g.px + qi];
                }
            }
        }
        Jq[c] += s;
    }
}

// Read views of the input of a pass: the interior of a padded current plane
// (first pass) or a compact FP64 plane.
template <typename JT>
struct PaddedPlane {
    const JT *a;
    __device__ inline double at(const Geom &g, int i, int j, int k) const {
        return as_double(__ldg(a + g.pidx(i, j, k)));
    }
};
struct CompactPlane {
    const double *a;
    __device__ inline double at(const Geom &g, int i, int j, int k) const {
        return __ldg(a + ((long long)k * g.ny + j) * g.nx + i);
    }
};

// x-y part of the stencil read through a view V (same arithmetic as XYStencil).
template <typename V>
__device__ inline double xy_sum(const Geom &g, const V &v, const XYStencil &st, int k) {
    auto row = [&](int jj) { return (v.at(g, st.im, jj, k) + 2.0 * v.at(g, st.i, jj, k)) + v.at(g, st.ip, jj, k); };
    return (row(st.jm) + 2.0 * row(st.j)) + row(st.jp);
}

// One smoothing pass of the 3 planes in[0..2] into the compact planes out,
// grid (ceil(nx/bx), ny, nplanes * ceil(nz/kColumn)) of bx threads.  A thread
// walks up to kColumn z planes of one (i, j) column and keeps the x-y sums of
// the planes k-1, k, k+1 in registers, so that every plane's 3x3 sum is loaded
// once per column instead of three times.  The arithmetic is that of
// smooth_cell, in the same order.
template <typename V>
__global__ void __launch_bounds__(kRowThreads) k_smooth_cols(Geom g, V in0, V in1, V in2, double *out, int zchunks) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.nx) return;
    const int j = blockIdx.y;
    const int q = blockIdx.z / zchunks, zc = blockIdx.z - q * zchunks;
    const V v{q == 0 ? in0.a : (q == 1 ? in1.a : in2.a)};
    double *o = out + (long long)q * g.nx * g.ny * g.nz;
    const XYStencil st(g, i, j);
    if (g.ndim == 2) {
        o[(long long)j * g.nx + i] = xy_sum(g, v, st, 0) * 0.0625;    // / 16
        return;
    }
    const int k0 = zc * kColumn, k1 = min(k0 + kColumn, g.nz);
    double pm = xy_sum(g, v, st, k0 == 0 ? g.nz - 1 : k0 - 1);
    double p0 = xy_sum(g, v, st, k0);
    for (int k = k0; k < k1; ++k) {
        const double pp = xy_sum(g, v, st, k == g.nz - 1 ? 0 : k + 1);
        o[((long long)k * g.ny + j) * g.nx + i] = ((pm + 2.0 * p0) + pp) * 0.015625;   // / 64
        pm = p0;
        p0 = pp;
    }
}

// Batched over runs, with the block map of the field kernels (block_prefix
// counts 256-cell blocks of every run's padded grid, which covers its
// interior).  PHASE 0 folds; PHASE 1 is smoothing pass `pass` (0-based), run
// by the runs that smooth more than `pass` times.
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
    const int passes = r.smooth;
    if (passes <= pass) return;
    const Geom g = r.g;
    const long long ncell = (long long)g.nx * g.ny * g.nz;
    const long long c = (long long)(blockIdx.x - block_prefix[run_sh]) * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    if (PHASE == 0) fold_cell<unsigned long long>(g, r.J, r.sbuf[0], ncell, c);
    else
        for (int q = 0; q < 3; ++q) smooth_cell(g, r.sbuf[pass & 1] + q * ncell, r.sbuf[(pass + 1) & 1] + q * ncell, c);
}

}  // namespace

// threads along x: the row length rounded up to a warp, at most kRowThreads
static int row_threads(const Geom &g) { return std::min(kRowThreads, (g.nx + 31) / 32 * 32); }

template <typename V>
static void launch_cols(const Geom &g, V in0, V in1, V in2, double *out, int nplanes, cudaStream_t s) {
    const int bx = row_threads(g);
    const int zchunks = g.ndim == 3 ? (g.nz + kColumn - 1) / kColumn : 1;
    const dim3 grid((g.nx + bx - 1) / bx, g.ny, nplanes * zchunks);
    k_smooth_cols<V><<<grid, bx, 0, s>>>(g, in0, in1, in2, out, zchunks);
}

template <typename JT>
const double *launch_smooth_current(const Geom &g, JT *const J[3], int passes, double *const buf[2], cudaStream_t s) {
    if (g.G > 0 || g.Gz > 0) {
        const int bx = row_threads(g);
        const dim3 grid((g.nx + bx - 1) / bx, g.ny, g.nz);
        k_fold_shell<JT><<<grid, bx, 0, s>>>(g, J[0], J[1], J[2]);
    }
    launch_cols(g, PaddedPlane<JT>{J[0]}, PaddedPlane<JT>{J[1]}, PaddedPlane<JT>{J[2]}, buf[0], 3, s);
    const long long ncell = (long long)g.nx * g.ny * g.nz;
    for (int p = 1; p < passes; ++p) {
        const double *in = buf[(p - 1) & 1];
        launch_cols(g, CompactPlane{in}, CompactPlane{in + ncell}, CompactPlane{in + 2 * ncell}, buf[p & 1], 3, s);
    }
    return buf[(passes - 1) & 1];
}

void launch_smooth(const Geom &g, const double *in, double *out, cudaStream_t s) {
    launch_cols(g, CompactPlane{in}, CompactPlane{in}, CompactPlane{in}, out, 1, s);
}

void launch_smooth_multi(int phase, int pass, const FieldRunF *runs_dev, const int *block_prefix_dev, int nblocks,
                         int nruns, cudaStream_t s) {
    if (phase == 0) k_smooth_multi<0><<<nblocks, 256, 0, s>>>(runs_dev, block_prefix_dev, nruns, pass);
    else k_smooth_multi<1><<<nblocks, 256, 0, s>>>(runs_dev, block_prefix_dev, nruns, pass);
}

template const double *launch_smooth_current<double>(const Geom &, double *const[3], int, double *const[2],
                                                    cudaStream_t);
template const double *launch_smooth_current<unsigned long long>(const Geom &, unsigned long long *const[3], int,
                                                                double *const[2], cudaStream_t);

}  // namespace pic
