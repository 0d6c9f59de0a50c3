// pic_internal.cuh -- shared declarations of the GB300 PIC library (not part of the ABI).
//
// Units and staggering follow the paper (App. A.2, A.3.2): cells of size 1,
// time in X0/c, fields e and b = cB in m_e c^2/(e X0).  Field component c at
// interior index (i,j,k): e_x (i+1/2,j,k), e_y (i,j+1/2,k), e_z (i,j,k+1/2),
// b_x (i,j+1/2,k+1/2), b_y (i+1/2,j,k+1/2), b_z (i+1/2,j+1/2,k).
//
// Device layout (HBM):
//  - every grid array is padded by G ghost cells on both sides of each
//    simulated axis (z is not padded in 2D); padded index of interior (i,j,k)
//    is ((k+Gz)*py + (j+G))*px + (i+G), px = nx+2G, ...  Ghost cells hold the
//    periodic images of the interior, so a tile plus halo is one contiguous box.
//  - fields: 6 planes e_x..b_z of Real; currents: 2 buffers x 3 planes (one is
//    accumulated while the other is zeroed); node fields (mixed path): one
//    float4 pair per padded cell, {E_x,E_y,E_z,B_x} {B_y,B_z,0,0}, the node
//    averages of App. A.3.3 at time t.
//  - particles, FP64 path: SoA planes x,y,z,u_x,u_y,u_z of double (absolute
//    positions); mixed path: packed cell coordinates (uint32), FP32 offsets
//    (SoA), FP32 momenta (SoA) and an int32 id, kept sorted by tile.
#pragma once
#include <cstdint>
#include <vector>

#include <cuda.h>   // CUtensorMap (the descriptor type only; encoded through the runtime's driver entry point)
#include <cuda_runtime.h>

namespace pic {

// Device-side error bits (written with atomicOr into ctx error word).
enum : int {
    ERR_FAST_MOVE = 1,   // a particle moved more than one cell in a step
    ERR_TIMEOUT = 2,     // a bounded spin gave up
    ERR_NONFINITE = 4,   // non-finite value met
    ERR_SORT = 8,        // sort bookkeeping overflow
    ERR_RANGE = 16,      // a particle position outside the domain (state upload)
};

// Unsigned 32-bit division by a divisor fixed at set-up, through a
// multiply-high (Granlund and Montgomery, "Division by invariant integers using
// multiplication", 1994): with l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d)
// + 1, n / d = (t + ((n - t) >> 1)) >> (l - 1) with t = mulhi(m, n), for every
// n < 2^32 and d >= 2.  A hardware division takes tens of instructions.
struct FastDiv {
    uint32_t d, m, l;
    __host__ void init(uint32_t dv) {
        d = dv < 1 ? 1 : dv;
        l = 0;
        while (l < 32 && (1ull << l) < d) ++l;
        m = d == 1 ? 0u : (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
    }
    __device__ __forceinline__ uint32_t div(uint32_t n) const {
        if (d == 1) return n;
        const uint32_t t = __umulhi(m, n);
        return (t + ((n - t) >> 1)) >> (l - 1);
    }
};

// Load of an array that the kernel does not write.  A translation unit that
// defines PIC_COHERENT_LOADS before including this header (the persistent
// ensemble step, whose CTAs read arrays that other CTAs of the same launch
// wrote) gets plain loads; the others use the read-only data path.  Internal
// linkage: each translation unit keeps its own form.
template <typename T>
static __device__ __forceinline__ T ldro(const T *p) {
#ifdef PIC_COHERENT_LOADS
    return *p;
#else
    return __ldg(p);
#endif
}

// Periodic wrap into [0, n): arguments within one period of the range (all
// the stencils and ghosts here) take two selects, others the modulo.
__host__ __device__ inline int wrap_index(int i, int n) {
    const int r = i + (i < 0 ? n : 0) - (i >= n ? n : 0);
    if ((unsigned)r < (unsigned)n) return r;
    const int m = i % n;
    return m < 0 ? m + n : m;
}

struct Geom {
    int ndim, nx, ny, nz;
    int G, Gz;            // ghost width in x,y and in z (0 in 2D)
    int px, py, pz;       // padded extents
    long long pcells;     // px*py*pz
    int bcx;              // 0 periodic, 1 conductor walls at x = 0, nx
    FastDiv fpx, fpy;     // division by px and py (set_divisors)
    __host__ void set_divisors() {
        fpx.init((uint32_t)px);
        fpy.init((uint32_t)py);
    }
    __host__ __device__ inline long long pidx(int i, int j, int k) const {
        return ((long long)(k + Gz) * py + (j + G)) * px + (i + G);
    }
    __host__ __device__ inline int wx(int i) const { return wrap_index(i, nx); }
    __host__ __device__ inline int wy(int j) const { return wrap_index(j, ny); }
    __host__ __device__ inline int wz(int k) const { return wrap_index(k, nz); }
    // padded index of the interior image of any integer coordinate
    __host__ __device__ inline long long widx(int i, int j, int k) const { return pidx(wx(i), wy(j), wz(k)); }
    // the same with plain modulo wraps: smaller code where a kernel makes many such
    // calls and registers are short (the FP64 push kernel spills with the selects)
    __host__ __device__ inline long long widx_mod(int i, int j, int k) const {
        int a = i % nx, b = j % ny, c = k % nz;
        a += a < 0 ? nx : 0;
        b += b < 0 ? ny : 0;
        c += c < 0 ? nz : 0;
        return pidx(a, b, c);
    }
};

// Packed cell coordinates of the mixed path: 2D i | j<<16; 3D i | j<<11 | k<<22.
__host__ __device__ inline uint32_t pack_cell(int ndim, int i, int j, int k) {
    return ndim == 2 ? (uint32_t)i | ((uint32_t)j << 16) : (uint32_t)i | ((uint32_t)j << 11) | ((uint32_t)k << 22);
}
__host__ __device__ inline void unpack_cell(int ndim, uint32_t c, int &i, int &j, int &k) {
    if (ndim == 2) { i = c & 0xffff; j = c >> 16; k = 0; }
    else { i = c & 0x7ff; j = (c >> 11) & 0x7ff; k = c >> 22; }
}

// Field planes of one run.  el (mixed path only, null in the FP64 path) holds
// the low-order part of e: the electric field is e + el, carried as an
// unevaluated FP32 pair so that the FP32 rounding of e does not accumulate
// over the steps (the e advance updates the pair with error-free FP32
// transformations from the exact integer current).  The gather reads e alone.
template <typename R>
struct FieldPtrs {
    R *e[3];
    R *b[3];
    R *el[3];
};

// e_c at padded index p in FP64, with its low-order part when there is one.
template <typename R>
__device__ inline double e_full(const FieldPtrs<R> &f, int c, long long p) {
    double v = (double)f.e[c][p];
    if (f.el[c]) v += (double)f.el[c][p];
    return v;
}

struct Species64 {
    double *x[3];
    double *u[3];
};

struct SpeciesMixed {
    uint32_t *cell;
    float *off[3];
    float *u[3];
    int32_t *id;
};

struct TileGeom {
    int T[3];        // tile extent in cells (T[2] = 1 in 2D)
    int H;           // halo (cells) on each side, equal to the ghost width G
    int R[3];        // T + 2H (R[2] = 1 in 2D)
    int ntile[3];    // tiles per axis
    int ntiles;
    int cells_per_tile;
    int lg[3];       // log2 T per axis when every T is a power of two, else -1
};

// Tile shapes that the push is also compiled for with a fixed geometry (the
// autotuner's choices for the 128^3 and 1024^2 workloads), so that node and
// current-slot offsets become immediates, by code: 1: 3D 16x8x4, halo 3; 2: 2D
// 16x16, halo 4.  Code 0: the geometry is read at run time.
struct FixedTile {
    int T0, T1, T2, H;
};
__host__ __device__ constexpr FixedTile fixed_tile(int code) {
    return code == 1 ? FixedTile{16, 8, 4, 3} : code == 2 ? FixedTile{16, 16, 1, 4} : FixedTile{0, 0, 0, 0};
}
// Code of a tile geometry (0 when it has no fixed form).
inline int fixed_tile_code(const TileGeom &t, int ndim) {
    for (int c = 1; c <= 2; ++c) {
        const FixedTile f = fixed_tile(c);
        if ((ndim == 3) == (f.T2 > 1) && t.T[0] == f.T0 && t.T[1] == f.T1 && t.T[2] == f.T2 && t.H == f.H) return c;
    }
    return 0;
}

// Sort key of a cell: tile index * cells_per_tile + index inside the tile
// (tiles with power-of-two sides only, t.lg[0] >= 0).
__host__ __device__ inline int tile_key_pow2(const TileGeom &t, int i, int j, int k) {
    const int ti = i >> t.lg[0], tj = j >> t.lg[1], tk = k >> t.lg[2];
    const int li = i & (t.T[0] - 1), lj = j & (t.T[1] - 1), lk = k & (t.T[2] - 1);
    return ((tk * t.ntile[1] + tj) * t.ntile[0] + ti) * t.cells_per_tile + (((lk << t.lg[1]) + lj) << t.lg[0]) + li;
}

// Energy-history slot of the current step (8 doubles: kinetic at t from both
// half steps, e^2 and b^2 per component).  With idx set, the slot is base +
// 8 * (*idx), idx being a device step counter that the e advance increments,
// so that a captured CUDA graph of several steps can be replayed; without idx
// the slot is base itself.  A null base records nothing.
struct HistRef {
    double *base;
    const long long *idx;
    long long cap;
    __device__ inline double *slot() const {
        if (!base) return nullptr;
        if (!idx) return base;
        const long long i = *idx;
        return i < cap ? base + 8 * i : nullptr;
    }
};

// ---- kernel launchers (implemented in the .cu files) ----

// fields.cu
template <typename R>
void launch_b_advance(const Geom &g, FieldPtrs<R> f, R h, HistRef energy, cudaStream_t s);
template <typename R>
void launch_e_advance(const Geom &g, FieldPtrs<R> f, const R *const J[3], R *const Jzero[3], R dt,
                      cudaStream_t s);
void launch_node_fields(const Geom &g, FieldPtrs<float> f, float4 *nfA, float2 *nfB, cudaStream_t s);
// e += dt curl b + |alpha| * J for the fixed-point current of the mixed path
// hist_inc (nullable): the step counter of the energy history, incremented once
void launch_e_advance_fx(const Geom &g, FieldPtrs<float> f, const unsigned long long *const J[3],
                         unsigned long long *const Jzero[3], float dt, double alpha_abs, long long *hist_inc,
                         cudaStream_t s);
template <typename R>
void launch_add_uniform(const Geom &g, FieldPtrs<R> f, const double e0[3], const double b0[3], cudaStream_t s);
// e += dt curl b + scale * Js with the smoothed compact current Js (3 planes of
// nx*ny*nz values: double in the FP64 path, int64 fixed point in the mixed
// path, in the units of the path's current), and zeroing of Jzero
template <typename R, typename ZT, typename CT>
void launch_e_advance_smoothed(const Geom &g, FieldPtrs<R> f, const CT *Js, double scale, ZT *const Jzero[3],
                               R dt, long long *hist_inc, cudaStream_t s);

// smooth.cu: current smoothing (App. A.3.4).  Compact arrays are indexed
// (k*ny + j)*nx + i over the interior, plane after plane.
// Value type of a smoothed current: int64 fixed point for the mixed path's
// current (unsigned long long storage), double for the FP64 path.
template <typename JT> struct SmoothValue;
template <> struct SmoothValue<unsigned long long> { typedef long long type; };
template <> struct SmoothValue<double> { typedef double type; };
// Smooths the deposited current J (padded planes; its ghost images are folded
// into the interior in place, so J is consumed) `passes` >= 1 times into the
// compact buffers buf[0..1] (3 planes each); returns the buffer with the result.
template <typename JT>
const typename SmoothValue<JT>::type *launch_smooth_current(const Geom &g, JT *const J[3], int passes,
                                                            typename SmoothValue<JT>::type *const buf[2],
                                                            cudaStream_t s);
// one smoothing pass of one compact plane, in -> out (distinct arrays)
void launch_smooth(const Geom &g, const double *in, double *out, cudaStream_t s);

// push_fp64.cu
void launch_push_fp64(const Geom &g, FieldPtrs<double> f, double *const J[3], Species64 sp, long long n,
                      double h, double alpha, double dt, int mode, double m_over_me, double *kin_acc, int *err,
                      cudaStream_t s);

// push_mixed.cu
struct MixedStepArgs {
    Geom g;
    TileGeom t;
    const float4 *nfA;              // node fields {E_x,E_y,E_z,B_x} per padded cell
    const float2 *nfB;              // node fields {B_y,B_z} per padded cell
    unsigned long long *J[3];       // padded int64 fixed-point current planes (units 2^-36 of sgn(q) flux)
    int nspecies;
    SpeciesMixed sp[4];
    const int *tile_start[4];       // per species: ntiles+1 offsets into the particle arrays
    float h[4];                     // (q/e)(m_e/m)
    float sgn[4];                   // sign of the charge
    double m_over_me[4];
    float dt;
    int mode;                       // 0 step, 1 half step back (momenta only)
    HistRef hist;                   // slot[0..1]: kinetic energy of u^{t-1/2} and u^{t+1/2}
    int *err;
    // when non-null: per species, the push adds to key_counts[s][key] the number of
    // particles whose new cell has that sort key (the next sort's histogram)
    int *key_counts[4];
    // TMA descriptors of the node-field arrays nfA (4 floats per node) and nfB
    // (2 floats per node) with a box of one tile + halo; use_tma = 0 when the
    // geometry breaks a TMA alignment rule (odd tile width or odd padded x extent)
    int use_tma;
    CUtensorMap tmA, tmB;
};
void launch_push_mixed(const MixedStepArgs &a, cudaStream_t s);
// persistent launch over the tiles of many runs (same ndim and tile shape)
// count: every run's args carry key_counts (the next sort's histogram)
void launch_push_mixed_multi(const MixedStepArgs *runs_dev, const int *tile_prefix_dev, int nruns, int ndim,
                             const TileGeom &t, bool walls, bool count, int *counter, cudaStream_t s);

// fields.cu, batched over runs: one launch updates every run's grid
struct FieldRunF {
    Geom g;
    FieldPtrs<float> f;
    float4 *nfA;
    float2 *nfB;
    const unsigned long long *J[3];
    unsigned long long *Z[3];
    HistRef hist;           // slot[2..7]: e^2, b^2 sums of the step (null base: none)
    long long *hist_inc;    // E_FX phase: step counter of the history, incremented once (nullable)
    double scale;           // |alpha| 2^-36
    int smooth;             // current smoothing passes (0: off); the E_FX phase then reads sbuf[smooth & 1]
    long long *sbuf[2];     // compact fixed-point smoothing buffers, 3 planes of nx*ny*nz each
};
enum { FIELD_B_HALF = 0, FIELD_NODE = 1, FIELD_E_FX = 2 };
void launch_fields_multi(int phase, const FieldRunF *runs_dev, const int *block_prefix_dev, int nblocks, int nruns,
                         float h, float dt, cudaStream_t s);
// smooth.cu, batched: phase 0 folds every smoothing run's J into sbuf[0]; phase 1 runs pass
// `pass` (sbuf[pass & 1] -> sbuf[(pass + 1) & 1]) of the runs with more passes
void launch_smooth_multi(int phase, int pass, const FieldRunF *runs_dev, const int *block_prefix_dev, int nblocks,
                         int nruns, cudaStream_t s);
void launch_half_back_mixed(const Geom &g, const float4 *nfA, const float2 *nfB, SpeciesMixed sp, long long n,
                            float h, float dt, cudaStream_t s);
size_t mixed_smem_bytes(const TileGeom &t, int ndim);

// walk.cu: the persistent step of a mixed ensemble (one launch per step).
// Phases of one step, in order; every item of phase ph of run r waits until all
// items of run r in phases before ph are done.
struct SortArgs;
enum WalkPhase {
    // the counting sort of one species (steps that sort)
    S_ZERO = 0, S_HIST, S_SCAN_BLOCKS, S_SCAN_SUMS, S_SCAN_FINISH, S_RANK, S_ZERO_AFTER, S_GATHER,
    // the main loop
    W_B_HALF_E, W_NODE, W_PUSH, W_SMOOTH_FOLD, W_SMOOTH_PASS, W_B_HALF, W_E_FX
};
constexpr int kWalkMaxPhases = 32;
struct WalkArgs {
    const MixedStepArgs *push;     // per run
    const FieldRunF *fe, *fp;      // per run: first b half advance (records the energies); other field phases
    const SortArgs *sort;          // [nruns * 4]: run r, species q at 4 r + q (runs that sort this step)
    const int *prefix;             // [nphase * nruns + 1]: first queue item of (phase, slot), phase-major
    const int *base;               // [nruns * (nphase + 1)]: items of run r in the phases before each phase
    const int *order;              // [nruns]: run of each slot of a phase (runs with the longest items first)
    int *head;                     // queue counter (zero before the launch)
    int *abort;                    // set when a wait runs out (zero before the launch)
    int *done;                     // [nruns] items of each run done (zero before the launch)
    int *err;
    int nruns, nphase, total;
    int cells_per_item;            // cells of one field or smoothing item
    int kind[kWalkMaxPhases];      // WalkPhase of each phase
    int pass[kWalkMaxPhases];      // smoothing pass of a W_SMOOTH_PASS phase
    int species[kWalkMaxPhases];   // species of a sort phase
    float h, dt;                   // h = dt/2 (half advances of b)
    long long wait_ns;             // bound of one wait (device global timer, ns)
};
int walk_cells_per_item(int ndim);
// Items of sort phase `kind` of one species' sort in the walker.
int walk_sort_items(const SortArgs &a, int kind, int cells_per_item);
// Can the walker run a step with this push shared memory on this device?
bool walk_fits(int ndim, bool walls, bool count, size_t push_smem);
// tile_code: fixed_tile_code of the runs' (common) tile geometry
void launch_walk(const WalkArgs &w, int ndim, bool walls, bool count, size_t push_smem, int tile_code,
                 cudaStream_t s);
// dynamic shared memory a push CTA may use (227 KB per block, less the kernels' static shared memory)
constexpr size_t kMaxPushSmem = 224 * 1024;

// sort.cu
struct SortArgs {
    Geom g;
    TileGeom t;
    long long n;
    SpeciesMixed src, dst;
    int *counts;     // ntiles*cells_per_tile + 1 scratch
    int *offsets;    // same size: exclusive scan; offsets[key] start of key
    int *block_sums; // scratch for the scan
    int *tile_start; // ntiles+1 output
    const int *old_tile_start;  // tile offsets of the source layout, or nullptr if untiled
    int *perm;       // n scratch: source index of every destination slot
    int *err;
    int counted;     // counts already hold the key histogram of src (counted by the push)
};
void launch_sort(const SortArgs &a, cudaStream_t s);
// many independent sorts in one launch per phase: h_prefix (4 x (nsort + 1) ints)
// is filled by sort_multi_prefixes from the host copy of the arguments and
// uploaded to d_prefix next to d_args
void sort_multi_prefixes(const SortArgs *h_args, int nsort, int *h_prefix);
void launch_sort_multi(const SortArgs *d_args, const int *d_prefix, const int *h_prefix, int nsort, int ndim,
                       cudaStream_t s);
size_t sort_scan_scratch(long long nkeys);

// mj.cu
void build_marginal_table(double theta, double beta0, int n, std::vector<double> &F, double &s0, double &h,
                          double &psi, double &Z);
void launch_load_mj(const Geom &g, int ndim, long long n, int species, unsigned long long seed, int profile, double L,
                    double x0, double theta, const double beta[3], int naive, const double *Fdev, double s0,
                    double h, int ntab, double psi, double Z, int colocate, Species64 d64, Species64 c64,
                    SpeciesMixed dmx, SpeciesMixed cmx, int mixed, int *err, cudaStream_t s);
constexpr int kMjTable = 4096;

// mlp.cu
constexpr int kMlpParams = 64 * 3 + 64 + 64 * 64 + 64 + 64 * 64 + 64 + 64 + 1;
constexpr int kMlpTheta = 16, kMlpBeta = 12;        // training grid of (theta, beta0)
constexpr int kMlpBatchMax = 8192;
size_t mlp_train_smem();
void launch_mlp_fwd_bwd(const float *W, const float *X, const float *T, int n, float *grad, double *loss,
                        cudaStream_t s);
void launch_adam(float *W, float *g, float *m, float *v, int step, float lr, cudaStream_t s);
void launch_mlp_to_half(const float *W, void *Wh, cudaStream_t s);
void launch_mlp_infer(const void *Wh, const float *X, int n, float *out, cudaStream_t s);
void launch_mlp_data(const double *F, const double *par, int ncombo, unsigned long long seed, long long base, int n,
                     float *X, float *T, cudaStream_t s);
void launch_sample_par(const double *F, double s0, double h, double psi, double Z, const void *Wh, int use_mlp,
                       double theta, double beta0, const double *w, int n, double *y, cudaStream_t s);
void launch_load_mj_mlp(const Geom &g, int ndim, long long n, int species, unsigned long long seed, int profile,
                        double L, double x0, double theta, const double beta[3], const void *Wh, int colocate,
                        Species64 d64, Species64 c64, SpeciesMixed dmx, SpeciesMixed cmx, int mixed, int *err,
                        cudaStream_t s);

// diag.cu
template <typename R>
void launch_field_diag(const Geom &g, FieldPtrs<R> f, double *acc /*6*/, long long *nonfinite, cudaStream_t s);
void launch_particle_diag64(const Geom &g, Species64 sp, long long n, double m_over_me, double *acc /*8*/,
                            long long *nonfinite, cudaStream_t s);
void launch_particle_diag_mixed(const Geom &g, SpeciesMixed sp, long long n, double m_over_me, double *acc,
                                long long *nonfinite, cudaStream_t s);
template <typename R>
void launch_div_e(const Geom &g, FieldPtrs<R> f, double *out /*ncell interior*/, cudaStream_t s);
void launch_rho64(const Geom &g, Species64 sp, long long n, double alpha, double *rho, cudaStream_t s);
void launch_rho_mixed(const Geom &g, SpeciesMixed sp, long long n, double alpha, double *rho, cudaStream_t s);
void launch_max_abs_diff(const double *a, const double *b, long long n, double *out_max, cudaStream_t s);

}  // namespace pic
