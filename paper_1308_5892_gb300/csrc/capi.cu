// capi.cu -- host runtime behind the C ABI of include/pic.h: context and device
// memory, state transfer (values validated on the device while converted),
// step orchestration for one run or a batched ensemble, CUDA-graph capture and
// replay of the mixed step, the autotuner, diagnostics, the learned sampler.
//
// One step of one run (main loop of App. A.3.1), state e^t, b^{t-dt/2}, x^t, u^{t-dt/2}:
//   [re-sort particles by tile when due]                    (mixed path)
//   b += -(dt/2) curl e            -> b^t; FP64 sums of e^2, b^2 at t recorded
//   node fields E, B at t            (mixed path, App. A.3.3 averages)
//   per species: gather, Boris, move, deposit into J        (steps 2, 3, 8, 9)
//   b += -(dt/2) curl e            -> b^{t+dt/2}            (steps 4, 5)
//   e += dt curl b + J, zero the other J buffer             (steps 6, 7, 11, 12)
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pic.h"
#include "pic_internal.cuh"

using namespace pic;

namespace {

struct SpeciesState {
    double q_over_e = 0, m_over_me = 1, alpha = 0, h = 0;
    int64_t cap = 0, n = 0;
    Species64 s64{};            // FP64 path
    SpeciesMixed mb[2]{};       // mixed path: current and sort target
    int cur = 0;
    int *tile_start = nullptr;  // ntiles + 1, offsets of the current layout
    int *tile_start_alt = nullptr;
    bool tiled = false;         // current layout comes from a sort
    int tiled_ntiles = 0;       // tile count of the geometry that sort used
    int *counts = nullptr;      // mixed: key histogram / cursors of the sort, zero between sorts
    bool counted = false;       // the last push filled counts for the next sort
};

struct Run {
    pic_run_desc d{};
    Geom g{};
    TileGeom t{};
    int sort_interval = 4;
    int since_sort = 0;
    int max_tiles = 1;          // tile arrays are sized for the autotuner's smallest tile
    long long max_keys = 1;     // sort keys of the largest candidate geometry
    bool sorted = false;
    void *F = nullptr;          // 6 planes of Real (e_x..b_z), padded
    void *J = nullptr;          // 2 buffers x 3 planes, padded: double (FP64) or int64 fixed point (mixed)
    int jcur = 0;
    float4 *nfA = nullptr;      // node fields {E_x,E_y,E_z,B_x} (mixed)
    float2 *nfB = nullptr;      // node fields {B_y,B_z} (mixed)
    bool tma = false;           // TMA descriptors of nfA/nfB for the current tile box are valid
    CUtensorMap tmA{}, tmB{};
    SpeciesState sp[PIC_MAX_SPECIES];
    int *offsets = nullptr, *block_sums = nullptr;
    int *perm = nullptr;        // sort scratch, max species capacity
    double *rho_s = nullptr, *rho_tot = nullptr, *divb = nullptr;
    int smooth = 0;             // current smoothing passes per step (App. A.3.4)
    void *sbuf[2] = {nullptr, nullptr};     // compact smoothing buffers, 3 planes of 8-byte values each
    double *acc = nullptr;      // diagnostics accumulators (64 doubles)
    double *hist = nullptr;     // energy history, 8 doubles per step
    int64_t hist_cap = 0, hist_n = 0;
    long long *hist_idx = nullptr;  // device copy of hist_n, advanced by the e advance (mixed)
    int64_t step = 0;
    double inv_alpha_abs = 1;
};

}  // namespace

constexpr int kKernelClasses = 4;   // PIC_KERNEL_PUSH .. PIC_KERNEL_SMOOTH

struct pic_ctx {
    int precision = PIC_FP64;
    uint32_t flags = 0;
    cudaStream_t stream = nullptr;
    pic_allocator alloc{};
    bool have_alloc = false;
    std::vector<Run> runs;
    int *d_err = nullptr;
    void *staging = nullptr;
    size_t staging_bytes = 0;
    double *mj_table = nullptr;     // cumulative marginal of the loader, kMjTable + 1 values
    // learned sampler of the loader (mlp.cu)
    float *mlpW = nullptr, *mlpG = nullptr, *mlpM = nullptr, *mlpV = nullptr, *mlpX = nullptr, *mlpT = nullptr;
    void *mlpWh = nullptr;
    double *mlpLoss = nullptr, *mlpF = nullptr, *mlpPar = nullptr;
    bool mlp_tables = false, mlp_ready = false, mlp_init = false;
    int mlp_step = 0;
    std::vector<std::pair<void *, size_t>> allocs;
    std::string err;
    int64_t launches_per_step = 0;
    int64_t launch_total = 0;        // launches queued by the current pic_step call
    int64_t graph_launches = 0;      // launches of one replay of the captured period
    double bytes_per_ps = 0;
    // batched ensemble (nruns > 1, mixed): per-run argument tables on the device
    bool multi = false;
    MixedStepArgs *multi_args = nullptr;
    FieldRunF *multi_fe = nullptr, *multi_fp = nullptr;
    int *multi_tiles = nullptr, *multi_blocks = nullptr, *multi_counter = nullptr;
    int *walk_tab = nullptr, *walk_ctl = nullptr;   // step walker: queue tables; head, abort, done[nruns]
    std::vector<int> h_walk;
    SortArgs *walk_sort_dev = nullptr;              // step walker: sort arguments, [nruns * 4]
    std::vector<SortArgs> h_walk_sort;
    int walk_fit[2][2] = {{-1, -1}, {-1, -1}};      // walk_fits() by (walls, count) for walk_fit_smem
    size_t walk_fit_smem = 0;
    int multi_nblocks = 0;
    bool multi_tiles_dirty = false;
    std::vector<MixedStepArgs> h_args;
    SortArgs *sort_args_dev = nullptr;    // one species of every run, for the batched sort
    int *sort_prefix_dev = nullptr;       // 4 x (nruns + 1) block prefixes of its phases
    std::vector<SortArgs> h_sort;
    std::vector<int> h_sort_prefix;
    // CUDA graph of one period of steps (mixed path): captured on a private stream,
    // replayed on the context stream while the host state matches the capture
    cudaGraphExec_t graph = nullptr;
    int graph_period = 0;
    std::vector<long long> graph_sig;
    cudaStream_t cap_stream = nullptr;
    bool capturing = false;
    char *gstage = nullptr;            // pinned per-step copies of the argument tables (ensemble)
    size_t gstage_stride = 0, gstage_bytes = 0;
    // state uploads: host-to-device copies on a stream of their own, overlapped
    // with the conversion kernels through two halves of the staging buffer
    cudaStream_t io_stream = nullptr;
    cudaEvent_t io_ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};   // start, loaded/filled[2], consumed/copied[2]
    std::vector<FieldRunF> h_fe, h_fp;
    // PIC_FLAG_TIMING: event pairs per kernel class, resolved in pic_kernel_time
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending[kKernelClasses];
    std::vector<cudaEvent_t> ev_pool;
    double ev_ms[kKernelClasses] = {0, 0, 0, 0};
    int64_t ev_n[kKernelClasses] = {0, 0, 0, 0};
};

namespace {

constexpr int64_t kHistCap = 1 << 16;

pic_status fail(pic_ctx *c, pic_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return st;
}

#define CK(call)                                                                                       \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return fail(ctx, PIC_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));  \
    } while (0)

cudaEvent_t take_event(pic_ctx *ctx) {
    if (!ctx->ev_pool.empty()) {
        cudaEvent_t e = ctx->ev_pool.back();
        ctx->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Scoped CUDA-event bracket around the kernels of one class (PIC_FLAG_TIMING).
struct KTimer {
    pic_ctx *ctx;
    int cls;
    cudaEvent_t a = nullptr;
    KTimer(pic_ctx *c, int k) : ctx(c), cls(k) {
        if ((ctx->flags & PIC_FLAG_TIMING) && !ctx->capturing) {
            a = take_event(ctx);
            cudaEventRecord(a, ctx->stream);
        }
    }
    ~KTimer() {
        if (a) {
            cudaEvent_t b = take_event(ctx);
            cudaEventRecord(b, ctx->stream);
            ctx->ev_pending[cls].push_back({a, b});
        }
    }
};

void *dev_alloc(pic_ctx *ctx, size_t bytes) {
    if (bytes == 0) bytes = 256;
    bytes = (bytes + 255) & ~size_t(255);
    void *p = nullptr;
    if (ctx->have_alloc) p = ctx->alloc.alloc(bytes, ctx->alloc.user);
    else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
    if (p) ctx->allocs.push_back({p, bytes});
    return p;
}

size_t real_size(const pic_ctx *ctx) { return ctx->precision == PIC_FP64 ? sizeof(double) : sizeof(float); }

template <typename R>
FieldPtrs<R> fields_of(Run &r) {
    FieldPtrs<R> f;
    R *F = (R *)r.F;
    for (int c = 0; c < 3; ++c) {
        f.e[c] = F + (size_t)c * r.g.pcells;
        f.b[c] = F + (size_t)(3 + c) * r.g.pcells;
        // the mixed path keeps the low-order part of e in planes 6..8 (see FieldPtrs)
        f.el[c] = sizeof(R) == sizeof(float) ? F + (size_t)(6 + c) * r.g.pcells : nullptr;
    }
    return f;
}

// Both current types (double, int64) are 8 bytes wide.
template <typename R>
R *jplane(Run &r, int buf, int c) {
    static_assert(sizeof(R) == 8, "current planes are 8-byte values");
    return (R *)r.J + ((size_t)buf * 3 + c) * r.g.pcells;
}

// ------------------------------------------------------------ conversion kernels

// dst_lo (nullable): receives the FP32 remainder v - (float)v (the low-order part of e in the mixed path).
template <typename R>
__global__ void k_pad_field(Geom g, const double *src, R *dst, R *dst_lo, int *err) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.pcells;
         p += (long long)gridDim.x * blockDim.x) {
        const int pi = (int)(p % g.px);
        const long long q = p / g.px;
        const int pj = (int)(q % g.py), pk = (int)(q / g.py);
        const int i = g.wx(pi - g.G), j = g.wy(pj - g.G), k = g.wz(pk - g.Gz);
        const double v = src[((long long)k * g.ny + j) * g.nx + i];
        if (!isfinite(v)) atomicOr(err, ERR_NONFINITE);
        dst[p] = (R)v;
        if (dst_lo) dst_lo[p] = (R)(v - (double)(R)v);
    }
}

// Position x on axis ax inside the domain: [0, n) periodic, [0, n_x] between walls.
__device__ inline bool in_domain(const Geom &g, int ax, double x) {
    const double n = ax == 0 ? g.nx : (ax == 1 ? g.ny : g.nz);
    return (ax == 0 && g.bcx == 1) ? (x >= 0.0 && x <= n) : (x >= 0.0 && x < n);
}

// Validation of an uploaded FP64 particle array (the mixed upload checks as it converts).
__global__ void k_check64(Geom g, Species64 s, long long n, int *err) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        for (int a = 0; a < 3; ++a) {
            if (!isfinite(s.u[a][p])) atomicOr(err, ERR_NONFINITE);
            if (a < g.ndim) {
                const double x = s.x[a][p];
                if (!isfinite(x)) atomicOr(err, ERR_NONFINITE);
                else if (!in_domain(g, a, x)) atomicOr(err, ERR_RANGE);
            }
        }
    }
}

// src_lo (nullable): the low-order part added to src (e in the mixed path).
template <typename R>
__global__ void k_unpad_field(Geom g, const R *src, const R *src_lo, double *dst) {
    const long long n = (long long)g.nx * g.ny * g.nz;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % g.nx);
        const long long r = q / g.nx;
        const int j = (int)(r % g.ny), k = (int)(r / g.ny);
        const long long p = g.pidx(i, j, k);
        dst[q] = (double)src[p] + (src_lo ? (double)src_lo[p] : 0.0);
    }
}

// st: 6 planes (x, y, z, ux, uy, uz) `stride` doubles apart, values for ids [a, a+m)
__global__ void k_upload_mixed(Geom g, const double *st, long long stride, long long m, long long a, SpeciesMixed d,
                               int *err) {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += (long long)gridDim.x * blockDim.x) {
        int c[3] = {0, 0, 0};
        float o[3] = {0.f, 0.f, 0.f};
        const int n3[3] = {g.nx, g.ny, g.nz};
        for (int ax = 0; ax < g.ndim; ++ax) {
            const double x = st[ax * stride + q];
            if (!isfinite(x) || !in_domain(g, ax, x)) {
                atomicOr(err, isfinite(x) ? ERR_RANGE : ERR_NONFINITE);
                continue;   // the state is rejected; keep the stored cell in range
            }
            double f = floor(x);
            int ci = (int)f;
            // the offset on the 2^-24 grid of the mixed path, where offset differences are exact (snap_offset)
            float off = (float)(rint((x - f) * 16777216.0) * (1.0 / 16777216.0));
            if (off >= 1.0f) { off = 0.0f; ci += 1; }
            if (g.bcx == 1 && ax == 0 && ci >= g.nx) { ci = g.nx - 1; off = 1.0f; }
            else if (ci >= n3[ax]) ci -= n3[ax];
            c[ax] = ci;
            o[ax] = off;
        }
        for (int comp = 3; comp < 6; ++comp)
            if (!isfinite(st[comp * stride + q])) atomicOr(err, ERR_NONFINITE);
        d.cell[a + q] = pack_cell(g.ndim, c[0], c[1], c[2]);
        d.off[0][a + q] = o[0];
        d.off[1][a + q] = o[1];
        if (g.ndim == 3) d.off[2][a + q] = o[2];
        d.u[0][a + q] = (float)st[3 * stride + q];
        d.u[1][a + q] = (float)st[4 * stride + q];
        d.u[2][a + q] = (float)st[5 * stride + q];
        d.id[a + q] = (int32_t)(a + q);
    }
}

// inverse map id -> storage index, then gather of the requested ids
__global__ void k_id_index(const int32_t *id, long long n, int *inv) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x)
        if ((unsigned long long)id[p] < (unsigned long long)n) inv[id[p]] = (int)p;   // ids are 0 .. n-1
}

__global__ void k_pick_mixed(Geom g, SpeciesMixed s, const int *inv, const long long *ids, long long m, double *st) {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += (long long)gridDim.x * blockDim.x) {
        const int p = inv[ids[q]];
        int i, j, k;
        unpack_cell(g.ndim, s.cell[p], i, j, k);
        st[q] = (double)i + (double)s.off[0][p];
        st[m + q] = (double)j + (double)s.off[1][p];
        st[2 * m + q] = g.ndim == 3 ? (double)k + (double)s.off[2][p] : 0.0;
        st[3 * m + q] = s.u[0][p];
        st[4 * m + q] = s.u[1][p];
        st[5 * m + q] = s.u[2][p];
    }
}

__global__ void k_pick64(Species64 s, const long long *ids, long long m, int ndim, double *st) {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += (long long)gridDim.x * blockDim.x) {
        const long long p = ids[q];
        for (int c = 0; c < 3; ++c) {
            st[c * m + q] = (c < ndim) ? s.x[c][p] : 0.0;
            st[(3 + c) * m + q] = s.u[c][p];
        }
    }
}

// Download of ids [a, a+m) through the id -> storage index map inv: coalesced
// staging writes, one pass over the chunk's own particles.
// st: 6 planes `stride` doubles apart, written for ids [a, a+m)
__global__ void k_download_by_id(Geom g, SpeciesMixed s, const int *inv, long long a, long long m, double *st,
                                 long long stride) {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += (long long)gridDim.x * blockDim.x) {
        const int p = inv[a + q];
        int i, j, k;
        unpack_cell(g.ndim, s.cell[p], i, j, k);
        st[q] = (double)i + (double)s.off[0][p];
        st[stride + q] = (double)j + (double)s.off[1][p];
        st[2 * stride + q] = g.ndim == 3 ? (double)k + (double)s.off[2][p] : 0.0;
        st[3 * stride + q] = s.u[0][p];
        st[4 * stride + q] = s.u[1][p];
        st[5 * stride + q] = s.u[2][p];
    }
}

inline int nblk(long long n) {
    long long b = (n + 255) / 256;
    return (int)std::max(1LL, std::min(b, 152LL * 16));
}

// ------------------------------------------------------------ validation

bool validate(const pic_run_desc &d, int precision, std::string &why) {
    char b[256];
    if (d.ndim != 2 && d.ndim != 3) { why = "ndim must be 2 or 3"; return false; }
    if (d.ndim == 2 && d.nz != 1) { why = "nz must be 1 when ndim = 2"; return false; }
    const int lim = d.ndim == 2 ? 65535 : 2047;
    if (d.nx < 2 || d.ny < 2 || (d.ndim == 3 && d.nz < 2) || d.nx > lim || d.ny > lim || d.nz > lim) {
        snprintf(b, sizeof b, "grid %dx%dx%d outside 2..%d per axis", d.nx, d.ny, d.nz, lim);
        why = b;
        return false;
    }
    if (!(d.dt > 0) || !(d.dt < 1.0 / std::sqrt((double)d.ndim))) {
        snprintf(b, sizeof b, "dt = %g violates the Courant limit dt < 1/sqrt(%d)", d.dt, d.ndim);
        why = b;
        return false;
    }
    if (!(d.n_x > 0) || !(d.rho_sp0 > 0) || !std::isfinite(d.n_x) || !std::isfinite(d.rho_sp0)) {
        why = "n_x and rho_sp0 must be positive";
        return false;
    }
    if (d.nspecies < 1 || d.nspecies > PIC_MAX_SPECIES) { why = "nspecies must be 1..4"; return false; }
    for (int s = 0; s < d.nspecies; ++s) {
        const pic_species_desc &sp = d.species[s];
        if (!(sp.q_over_e != 0) || !(sp.m_over_me > 0) || sp.capacity < 0 || sp.capacity > (int64_t)INT32_MAX) {
            snprintf(b, sizeof b, "species %d: q/e must be non-zero, m/m_e positive, capacity 0..2^31-1", s);
            why = b;
            return false;
        }
    }
    for (int a = 0; a < 3; ++a) {
        if (d.bc[a] != PIC_BC_PERIODIC && d.bc[a] != PIC_BC_CONDUCTOR) { why = "unknown boundary kind"; return false; }
        if (a > 0 && d.bc[a] != PIC_BC_PERIODIC) { why = "conducting walls are supported along x only"; return false; }
    }
    if (d.smooth_passes < 0 || d.smooth_passes > 4) { why = "smooth_passes must be 0..4"; return false; }
    if (d.smooth_passes > 0 && d.bc[0] != PIC_BC_PERIODIC) {
        why = "current smoothing is defined for periodic axes only";
        return false;
    }
    return true;
}

TileGeom make_tile_geom(const pic_run_desc &d, const int Tin[3], int H) {
    TileGeom t{};
    const int n3[3] = {d.nx, d.ny, d.ndim == 3 ? d.nz : 1};
    for (int a = 0; a < 3; ++a) {
        const int T = (a < d.ndim) ? std::max(1, std::min(Tin[a], n3[a])) : 1;
        t.T[a] = T;
        t.R[a] = (a < d.ndim) ? T + 2 * H : 1;
        t.ntile[a] = (a < d.ndim) ? (n3[a] + T - 1) / T : 1;
    }
    t.H = H;
    t.ntiles = t.ntile[0] * t.ntile[1] * t.ntile[2];
    t.cells_per_tile = t.T[0] * t.T[1] * t.T[2];
    bool pow2 = true;
    for (int a = 0; a < 3; ++a) {
        int lg = 0;
        while ((1 << lg) < t.T[a]) ++lg;
        t.lg[a] = lg;
        if ((1 << lg) != t.T[a]) pow2 = false;
    }
    if (!pow2) t.lg[0] = t.lg[1] = t.lg[2] = -1;
    return t;
}

// Candidate tile shapes of the autotuner (the first one is the default).
std::vector<std::vector<int>> tile_candidates(int ndim) {
    if (ndim == 2) return {{16, 16, 1}, {32, 16, 1}, {32, 32, 1}, {16, 8, 1}};
    return {{8, 8, 8}, {8, 8, 4}, {16, 8, 4}};
}
std::vector<int> sort_candidates(int ndim) { return ndim == 2 ? std::vector<int>{8, 4, 16} : std::vector<int>{3, 2, 1, 4}; }

void choose_tiles(Run &r, const pic_opts *o, int &max_tiles, long long &max_keys) {
    const pic_run_desc &d = r.d;
    int H = d.ndim == 2 ? 4 : 3;
    int hmax = std::min(d.nx, d.ny);
    if (d.ndim == 3) hmax = std::min(hmax, d.nz);
    H = std::max(1, std::min(H, hmax));
    auto cands = tile_candidates(d.ndim);
    int T[3] = {cands[0][0], cands[0][1], cands[0][2]};
    const bool user_tile = o && (o->tile[0] > 0 || o->tile[1] > 0 || o->tile[2] > 0);
    if (user_tile)
        for (int a = 0; a < 3; ++a)
            if (o->tile[a] > 0) T[a] = o->tile[a];
    r.t = make_tile_geom(d, T, H);
    r.sort_interval = (o && o->sort_interval > 0) ? o->sort_interval : sort_candidates(d.ndim)[0];
    max_tiles = r.t.ntiles;
    max_keys = (long long)r.t.ntiles * r.t.cells_per_tile;
    if (!user_tile) {
        for (auto &c : cands) {
            const int Tc[3] = {c[0], c[1], c[2]};
            const TileGeom t = make_tile_geom(d, Tc, H);
            max_tiles = std::max(max_tiles, t.ntiles);
            max_keys = std::max(max_keys, (long long)t.ntiles * t.cells_per_tile);
        }
    }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to libcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        else
            cudaGetLastError();
    }
    return fn;
}

// cuPointerGetAttribute through the same entry point.
typedef CUresult (*PointerAttrFn)(void *, CUpointer_attribute, CUdeviceptr);
PointerAttrFn pointer_attr() {
    static PointerAttrFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = (PointerAttrFn)p;
        else
            cudaGetLastError();
    }
    return fn;
}

// The host buffer [p, p + bytes) when it lies inside one page-locked allocation
// that the device addresses at the same virtual address (pinned memory under
// unified addressing), so that kernels can read or write it directly over the
// host link; nullptr otherwise (pageable memory, or a range that leaves the
// allocation), in which case the caller stages through device memory.
template <typename T>
T *mapped_host(T *p, size_t bytes) {
    if (!p || bytes == 0) return nullptr;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type != cudaMemoryTypeHost || at.devicePointer != (const void *)p) return nullptr;
    PointerAttrFn f = pointer_attr();
    if (!f) return nullptr;
    CUdeviceptr start = 0;
    size_t size = 0;
    if (f(&start, CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, (CUdeviceptr)p) != CUDA_SUCCESS ||
        f(&size, CU_POINTER_ATTRIBUTE_RANGE_SIZE, (CUdeviceptr)p) != CUDA_SUCCESS)
        return nullptr;
    const uintptr_t a = (uintptr_t)p;
    if (a < (uintptr_t)start || a + bytes > (uintptr_t)start + size) return nullptr;
    return p;
}

// TMA descriptors of the node-field arrays with a box of one tile + halo.  The
// arrays are FP32 planes of 4 (nfA) and 2 (nfB) floats per padded node; a copy
// starts at x = 4 x0 and 2 x0 floats, so the rules (inner box and strides
// multiples of 16 bytes, start x times 4 bytes a multiple of 16) need an even
// tile width and an even padded x extent.  Otherwise r.tma stays false and the
// push stages with coalesced loads.
void node_maps(Run &r) {
    r.tma = false;
    EncodeTiledFn enc = encode_tiled();
    const Geom &g = r.g;
    const TileGeom &t = r.t;
    if (!enc || !r.nfA || (t.T[0] & 1) || (g.px & 1) || t.R[0] * 4 > 256 || t.R[1] > 256 || t.R[2] > 256) return;
    const cuuint32_t rank = g.ndim == 3 ? 3 : 2;
    for (int which = 0; which < 2; ++which) {
        const cuuint64_t per = which == 0 ? 4 : 2;   // floats per node
        const cuuint64_t dims[3] = {per * (cuuint64_t)g.px, (cuuint64_t)g.py, (cuuint64_t)g.pz};
        const cuuint64_t strides[2] = {per * 4 * (cuuint64_t)g.px, per * 4 * (cuuint64_t)g.px * g.py};
        const cuuint32_t box[3] = {(cuuint32_t)(per * t.R[0]), (cuuint32_t)t.R[1], (cuuint32_t)t.R[2]};
        const cuuint32_t estr[3] = {1, 1, 1};
        void *base = which == 0 ? (void *)r.nfA : (void *)r.nfB;
        CUtensorMap *m = which == 0 ? &r.tmA : &r.tmB;
        if (enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, base, dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return;
    }
    r.tma = true;
}

pic_status setup_run(pic_ctx *ctx, Run &r, const pic_opts *o) {
    const pic_run_desc &d = r.d;
    const bool mixed = ctx->precision == PIC_MIXED;
    int max_tiles = 1;
    long long max_keys = 1;
    if (mixed) {
        choose_tiles(r, o, max_tiles, max_keys);
        if (mixed_smem_bytes(r.t, d.ndim) > kMaxPushSmem)
            return fail(ctx, PIC_EINVAL, "tile %dx%dx%d needs more shared memory than a CTA has", r.t.T[0], r.t.T[1],
                        r.t.T[2]);
    }
    const int G = mixed ? r.t.H : 0;
    Geom &g = r.g;
    g.ndim = d.ndim; g.nx = d.nx; g.ny = d.ny; g.nz = d.ndim == 2 ? 1 : d.nz;
    g.G = G; g.Gz = d.ndim == 3 ? G : 0;
    g.px = g.nx + 2 * G; g.py = g.ny + 2 * G; g.pz = g.nz + 2 * g.Gz;
    g.pcells = (long long)g.px * g.py * g.pz;
    g.set_divisors();
    g.bcx = d.bc[0];
    r.inv_alpha_abs = d.n_x * d.n_x * d.rho_sp0 / 2.0;
    const size_t rs = real_size(ctx);
    const long long ncell = (long long)g.nx * g.ny * g.nz;
    const size_t fplanes = mixed ? 9 : 6;   // mixed: e, b and the low-order part of e
    r.F = dev_alloc(ctx, fplanes * rs * g.pcells);
    r.J = dev_alloc(ctx, 6 * 8 * g.pcells);
    if (!r.F || !r.J) return fail(ctx, PIC_ENOMEM, "allocator returned NULL for the field arrays");
    CK(cudaMemsetAsync(r.F, 0, fplanes * rs * g.pcells, ctx->stream));
    CK(cudaMemsetAsync(r.J, 0, 6 * 8 * g.pcells, ctx->stream));
    if (mixed) {
        r.nfA = (float4 *)dev_alloc(ctx, sizeof(float4) * g.pcells);
        r.nfB = (float2 *)dev_alloc(ctx, sizeof(float2) * g.pcells);
        node_maps(r);
        const long long nkeys = max_keys;
        r.offsets = (int *)dev_alloc(ctx, sizeof(int) * (nkeys + 1));
        r.block_sums = (int *)dev_alloc(ctx, sizeof(int) * sort_scan_scratch(nkeys));
        r.max_tiles = max_tiles;
        r.max_keys = max_keys;
        int64_t capmax = 1;
        for (int s = 0; s < d.nspecies; ++s) capmax = std::max<int64_t>(capmax, d.species[s].capacity);
        r.perm = (int *)dev_alloc(ctx, sizeof(int) * capmax);
        if (!r.nfA || !r.nfB || !r.offsets || !r.block_sums || !r.perm)
            return fail(ctx, PIC_ENOMEM, "allocator returned NULL for the tile buffers");
    }
    r.rho_s = (double *)dev_alloc(ctx, sizeof(double) * ncell);
    r.rho_tot = (double *)dev_alloc(ctx, sizeof(double) * ncell);
    r.divb = (double *)dev_alloc(ctx, sizeof(double) * ncell);
    r.acc = (double *)dev_alloc(ctx, sizeof(double) * 64);
    r.hist_cap = kHistCap;
    r.hist = (double *)dev_alloc(ctx, sizeof(double) * 8 * r.hist_cap);
    r.hist_idx = (long long *)dev_alloc(ctx, sizeof(long long));
    if (!r.rho_s || !r.rho_tot || !r.divb || !r.acc || !r.hist || !r.hist_idx)
        return fail(ctx, PIC_ENOMEM, "allocator returned NULL for the diagnostics buffers");
    r.smooth = d.smooth_passes;
    if (r.smooth > 0) {
        for (int b = 0; b < 2; ++b) {
            r.sbuf[b] = dev_alloc(ctx, 8 * 3 * ncell);
            if (!r.sbuf[b]) return fail(ctx, PIC_ENOMEM, "allocator returned NULL for the smoothing buffers");
        }
    }
    CK(cudaMemsetAsync(r.hist, 0, sizeof(double) * 8 * r.hist_cap, ctx->stream));
    CK(cudaMemsetAsync(r.hist_idx, 0, sizeof(long long), ctx->stream));
    for (int s = 0; s < d.nspecies; ++s) {
        SpeciesState &S = r.sp[s];
        S.q_over_e = d.species[s].q_over_e;
        S.m_over_me = d.species[s].m_over_me;
        S.alpha = 2.0 * (S.q_over_e > 0 ? 1.0 : -1.0) / (d.n_x * d.n_x * d.rho_sp0);
        S.h = S.q_over_e / S.m_over_me;
        S.cap = d.species[s].capacity;
        S.n = 0;
        const size_t cap = (size_t)std::max<int64_t>(S.cap, 1);
        if (!mixed) {
            for (int a = 0; a < 3; ++a) {
                S.s64.x[a] = (double *)dev_alloc(ctx, sizeof(double) * cap);
                S.s64.u[a] = (double *)dev_alloc(ctx, sizeof(double) * cap);
                if (!S.s64.x[a] || !S.s64.u[a]) return fail(ctx, PIC_ENOMEM, "allocator returned NULL for particles");
            }
        } else {
            for (int b = 0; b < 2; ++b) {
                SpeciesMixed &m = S.mb[b];
                m.cell = (uint32_t *)dev_alloc(ctx, sizeof(uint32_t) * cap);
                m.id = (int32_t *)dev_alloc(ctx, sizeof(int32_t) * cap);
                for (int a = 0; a < 3; ++a) {
                    m.off[a] = (a < d.ndim) ? (float *)dev_alloc(ctx, sizeof(float) * cap) : nullptr;
                    m.u[a] = (float *)dev_alloc(ctx, sizeof(float) * cap);
                    if ((a < d.ndim && !m.off[a]) || !m.u[a]) return fail(ctx, PIC_ENOMEM, "allocator returned NULL for particles");
                }
                if (!m.cell || !m.id) return fail(ctx, PIC_ENOMEM, "allocator returned NULL for particles");
            }
            S.counts = (int *)dev_alloc(ctx, sizeof(int) * (r.max_keys + 1));
            if (!S.counts) return fail(ctx, PIC_ENOMEM, "allocator returned NULL for the sort counts");
            CK(cudaMemsetAsync(S.counts, 0, sizeof(int) * (r.max_keys + 1), ctx->stream));
            S.tile_start = (int *)dev_alloc(ctx, sizeof(int) * (r.max_tiles + 1));
            S.tile_start_alt = (int *)dev_alloc(ctx, sizeof(int) * (r.max_tiles + 1));
            if (!S.tile_start || !S.tile_start_alt) return fail(ctx, PIC_ENOMEM, "allocator returned NULL for tile offsets");
            CK(cudaMemsetAsync(S.tile_start, 0, sizeof(int) * (r.max_tiles + 1), ctx->stream));
        }
    }
    return PIC_OK;
}

pic_status check_run(pic_ctx *ctx, int run) {
    if (!ctx) return PIC_EINVAL;
    if (run < 0 || run >= (int)ctx->runs.size()) return fail(ctx, PIC_EINVAL, "run index %d out of range", run);
    return PIC_OK;
}

// The transfer stream and its events, created on first use.
pic_status io_ready(pic_ctx *ctx) {
    if (!ctx->io_stream) CK(cudaStreamCreateWithFlags(&ctx->io_stream, cudaStreamNonBlocking));
    for (auto &e : ctx->io_ev)
        if (!e) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return PIC_OK;
}

pic_status read_err(pic_ctx *ctx) {
    int e = 0;
    CK(cudaMemcpyAsync(&e, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (e) {
        CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
        if (e & ERR_TIMEOUT) return fail(ctx, PIC_ETIMEOUT, "a bounded device wait gave up");
        if (e & ERR_FAST_MOVE) return fail(ctx, PIC_ESTATE, "a particle moved more than one cell in one step");
        if (e & ERR_SORT) return fail(ctx, PIC_ESTATE, "particle cell outside the grid during sort");
        if (e & ERR_NONFINITE) return fail(ctx, PIC_ENUMERIC, "non-finite value in the state");
        if (e & ERR_RANGE) return fail(ctx, PIC_EINVAL, "particle position outside the domain");
    }
    return PIC_OK;
}

// ------------------------------------------------------------ stepping

// Invariant: at a push, counts are zero unless counted.  Sorts leave them
// zero, and every other change of the particles or of the tile geometry is
// followed by a sort before the next push.  Counts left by an earlier
// counting push whose sort never came (the sort interval grew in between) no
// longer describe the particles, so they are cleared here.
void prepare_counts(pic_ctx *ctx, Run &r) {
    for (int q = 0; q < r.d.nspecies; ++q) {
        SpeciesState &S = r.sp[q];
        if (!S.counted) continue;
        (void)cudaMemsetAsync(S.counts, 0, sizeof(int) * ((size_t)r.t.ntiles * r.t.cells_per_tile + 1),
                              ctx->stream);   // a failure surfaces at the step's error check
        S.counted = false;
    }
}

SortArgs sort_args(pic_ctx *ctx, Run &r, SpeciesState &S) {
    SortArgs a;
    a.g = r.g;
    a.t = r.t;
    a.n = S.n;
    a.src = S.mb[S.cur];
    a.dst = S.mb[1 - S.cur];
    a.counts = S.counts;
    a.counted = S.counted ? 1 : 0;
    a.offsets = r.offsets;
    a.block_sums = r.block_sums;
    // the old-tile walk is valid only for the tile geometry the layout was sorted with
    a.old_tile_start = (S.tiled && S.tiled_ntiles == r.t.ntiles) ? S.tile_start : nullptr;
    a.tile_start = S.tile_start_alt;
    a.perm = r.perm;
    a.err = ctx->d_err;
    return a;
}

// Host bookkeeping after the sort of S was enqueued: the sorted copy becomes current.
void sort_done(Run &r, SpeciesState &S) {
    S.counted = false;
    S.cur = 1 - S.cur;
    std::swap(S.tile_start, S.tile_start_alt);
    S.tiled = true;
    S.tiled_ntiles = r.t.ntiles;
}

void sort_species(pic_ctx *ctx, Run &r, SpeciesState &S) {
    launch_sort(sort_args(ctx, r, S), ctx->stream);
    sort_done(r, S);
}

HistRef hist_ref(Run &r) { return HistRef{r.hist, r.hist_idx, r.hist_cap}; }

MixedStepArgs mixed_args(pic_ctx *ctx, Run &r) {
    typedef unsigned long long u64;
    MixedStepArgs a;
    a.g = r.g;
    a.t = r.t;
    a.nfA = r.nfA;
    a.nfB = r.nfB;
    for (int c = 0; c < 3; ++c) a.J[c] = jplane<u64>(r, r.jcur, c);
    a.nspecies = r.d.nspecies;
    for (int q = 0; q < r.d.nspecies; ++q) {
        SpeciesState &S = r.sp[q];
        a.sp[q] = S.mb[S.cur];
        a.tile_start[q] = S.tile_start;
        a.h[q] = (float)S.h;
        a.sgn[q] = S.q_over_e > 0 ? 1.f : -1.f;
        a.m_over_me[q] = S.m_over_me;
    }
    a.dt = (float)r.d.dt;
    a.mode = 0;
    a.hist = hist_ref(r);
    a.err = ctx->d_err;
    for (int q = 0; q < 4; ++q) a.key_counts[q] = nullptr;
    a.use_tma = r.tma ? 1 : 0;
    a.tmA = r.tmA;
    a.tmB = r.tmB;
    return a;
}

// energy: record the e^2, b^2 sums (first b half advance); inc: advance the history counter (e advance)
FieldRunF field_run(Run &r, bool energy, bool inc) {
    typedef unsigned long long u64;
    FieldRunF fr;
    fr.g = r.g;
    fr.f = fields_of<float>(r);
    fr.nfA = r.nfA;
    fr.nfB = r.nfB;
    for (int c = 0; c < 3; ++c) {
        fr.J[c] = jplane<u64>(r, r.jcur, c);
        fr.Z[c] = jplane<u64>(r, 1 - r.jcur, c);
    }
    fr.hist = energy ? hist_ref(r) : HistRef{nullptr, nullptr, 0};
    fr.hist_inc = inc ? r.hist_idx : nullptr;
    fr.scale = 2.0 / (r.d.n_x * r.d.n_x * r.d.rho_sp0) * 0x1p-36;
    fr.smooth = r.smooth;
    fr.sbuf[0] = (long long *)r.sbuf[0];
    fr.sbuf[1] = (long long *)r.sbuf[1];
    return fr;
}

// Ints of the step walker's queue tables: prefix [kWalkMaxPhases * nr + 1], base [nr * (kWalkMaxPhases + 1)],
// order [nr].
size_t walk_tab_ints(int nr) { return (size_t)kWalkMaxPhases * nr + 1 + (size_t)nr * (kWalkMaxPhases + 2); }

// Can the step walker run with this push shared memory (cached per context)?
bool walk_ok(pic_ctx *ctx, int ndim, bool walls, bool count, size_t smem) {
    if (smem != ctx->walk_fit_smem) {
        ctx->walk_fit[0][0] = ctx->walk_fit[0][1] = ctx->walk_fit[1][0] = ctx->walk_fit[1][1] = -1;
        ctx->walk_fit_smem = smem;
    }
    int &f = ctx->walk_fit[walls ? 1 : 0][count ? 1 : 0];
    if (f < 0) f = walk_fits(ndim, walls, count, smem) ? 1 : 0;
    return f == 1;
}

// Host source of an argument-table upload: the table itself, or (slot >= 0,
// while a graph is captured) its copy in the pinned region of that step, which
// the captured copy node reads again at every replay.
const void *host_src(pic_ctx *ctx, int slot, size_t &off, const void *data, size_t bytes) {
    if (slot < 0) return data;
    char *dst = ctx->gstage + (size_t)slot * ctx->gstage_stride + off;
    std::memcpy(dst, data, bytes);
    off += (bytes + 255) & ~size_t(255);
    return dst;
}

// One step of every run of a mixed ensemble: per-run sorts when due (one
// batched launch per sort phase), then the step walker (one persistent launch
// for every phase of every run), or with PIC_FLAG_PHASE_LAUNCHES or
// PIC_FLAG_TIMING one batched launch per field phase and one persistent push
// launch for all runs.
pic_status step_multi(pic_ctx *ctx, int slot) {
    size_t soff = 0;
    cudaStream_t s = ctx->stream;
    const int nr = (int)ctx->runs.size();
    int launches = 0;
    // runs whose sort is due
    std::vector<int> due;
    std::vector<char> is_due(nr, 0);
    int maxsp = 0;
    for (int i = 0; i < nr; ++i) {
        Run &r = ctx->runs[i];
        if (!r.sorted || r.since_sort >= r.sort_interval) {
            due.push_back(i);
            is_due[i] = 1;
            maxsp = std::max(maxsp, r.d.nspecies);
        }
    }
    // when the next step sorts every run, this step's push counts their key histograms
    bool count = true;
    for (int i = 0; i < nr; ++i) {
        const Run &r = ctx->runs[i];
        const int since = is_due[i] ? 0 : r.since_sort;
        if (!(since + 1 >= r.sort_interval && r.t.lg[0] >= 0)) count = false;
    }
    const float dt = (float)ctx->runs[0].d.dt;
    int max_smooth = 0;
    for (auto &r : ctx->runs) max_smooth = std::max(max_smooth, r.smooth);
    const int ndim = ctx->runs[0].d.ndim;
    const bool walls = ctx->runs[0].g.bcx == 1;
    const size_t push_smem = mixed_smem_bytes(ctx->runs[0].t, ndim);
    const int nphase = (due.empty() ? 0 : 8 * maxsp) + 5 + (max_smooth > 0 ? 1 + max_smooth : 0);
    const bool walk = !(ctx->flags & (PIC_FLAG_PHASE_LAUNCHES | PIC_FLAG_TIMING)) && nphase <= kWalkMaxPhases &&
                      walk_ok(ctx, ndim, walls, count, push_smem);
    // The walker sorts too unless one run holds more than a quarter of the particles: that run's
    // sort alone then sets the time, and its own launches per phase (more warps per SM for the
    // latency-bound gather and rank) finish it sooner.
    long long most = 0, all = 0;
    for (int i : due) {
        long long n = 0;
        for (int q = 0; q < ctx->runs[i].d.nspecies; ++q) n += ctx->runs[i].sp[q].n;
        most = std::max(most, n);
        all += n;
    }
    const bool walk_sort = walk && most * 4 <= all;
    if (!due.empty() && walk_sort) {
        // the sorts run inside the step walker: record their arguments, book the swap
        for (int i : due) {
            Run &r = ctx->runs[i];
            for (int q = 0; q < r.d.nspecies; ++q) {
                ctx->h_walk_sort[4 * i + q] = sort_args(ctx, r, r.sp[q]);
                sort_done(r, r.sp[q]);
            }
            r.sorted = true;
            r.since_sort = 0;
        }
    } else if (!due.empty()) {
        // species q of every due run is sorted by one launch per sort phase
        KTimer t(ctx, PIC_KERNEL_SORT);
        for (int q = 0; q < maxsp; ++q) {
            int ns = 0;
            for (int i : due) {
                Run &r = ctx->runs[i];
                if (q < r.d.nspecies) ctx->h_sort[ns++] = sort_args(ctx, r, r.sp[q]);
            }
            sort_multi_prefixes(ctx->h_sort.data(), ns, ctx->h_sort_prefix.data());
            CK(cudaMemcpyAsync(ctx->sort_args_dev, host_src(ctx, slot, soff, ctx->h_sort.data(), sizeof(SortArgs) * ns),
                               sizeof(SortArgs) * ns, cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(ctx->sort_prefix_dev,
                               host_src(ctx, slot, soff, ctx->h_sort_prefix.data(), sizeof(int) * 4 * (ns + 1)),
                               sizeof(int) * 4 * (ns + 1), cudaMemcpyHostToDevice, s));
            launch_sort_multi(ctx->sort_args_dev, ctx->sort_prefix_dev, ctx->h_sort_prefix.data(), ns,
                              ctx->runs[0].d.ndim, s);
            for (int i : due) {
                Run &r = ctx->runs[i];
                if (q < r.d.nspecies) sort_done(r, r.sp[q]);
            }
            launches += 8;
        }
        for (int i : due) {
            ctx->runs[i].sorted = true;
            ctx->runs[i].since_sort = 0;
        }
    }
    if (ctx->multi_tiles_dirty) {
        std::vector<int> tp(nr + 1, 0);
        for (int r = 0; r < nr; ++r) tp[r + 1] = tp[r] + ctx->runs[r].t.ntiles;
        CK(cudaMemcpyAsync(ctx->multi_tiles, tp.data(), sizeof(int) * (nr + 1), cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
        ctx->multi_tiles_dirty = false;
    }
    for (auto &r : ctx->runs) prepare_counts(ctx, r);
    for (int i = 0; i < nr; ++i) {
        Run &r = ctx->runs[i];
        ctx->h_args[i] = mixed_args(ctx, r);
        if (count)
            for (int q = 0; q < r.d.nspecies; ++q) ctx->h_args[i].key_counts[q] = r.sp[q].counts;
        ctx->h_fe[i] = field_run(r, true, false);
        ctx->h_fp[i] = field_run(r, false, true);
    }
    CK(cudaMemcpyAsync(ctx->multi_args, host_src(ctx, slot, soff, ctx->h_args.data(), sizeof(MixedStepArgs) * nr),
                       sizeof(MixedStepArgs) * nr, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->multi_fe, host_src(ctx, slot, soff, ctx->h_fe.data(), sizeof(FieldRunF) * nr),
                       sizeof(FieldRunF) * nr, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->multi_fp, host_src(ctx, slot, soff, ctx->h_fp.data(), sizeof(FieldRunF) * nr),
                       sizeof(FieldRunF) * nr, cudaMemcpyHostToDevice, s));
    if (walk) {
        // the whole step in one persistent launch (walk.cu)
        WalkArgs w{};
        int np = 0;
        if (!due.empty() && walk_sort)
            for (int q = 0; q < maxsp; ++q)
                for (int k = S_ZERO; k <= S_GATHER; ++k) {
                    w.species[np] = q;
                    w.kind[np++] = k;
                }
        const int ph_push = np + 2;
        w.kind[np++] = W_B_HALF_E;
        w.kind[np++] = W_NODE;
        w.kind[np++] = W_PUSH;
        if (max_smooth > 0) {
            w.kind[np++] = W_SMOOTH_FOLD;
            for (int p = 0; p < max_smooth; ++p) {
                w.pass[np] = p;
                w.kind[np++] = W_SMOOTH_PASS;
            }
        }
        w.kind[np++] = W_B_HALF;
        w.kind[np++] = W_E_FX;
        const int cpi = walk_cells_per_item(ndim);
        auto items = [&](int ph, int i) -> int {
            const Run &r = ctx->runs[i];
            const long long ncell = (long long)r.g.nx * r.g.ny * r.g.nz;
            if (w.kind[ph] <= S_GATHER)
                return (is_due[i] && w.species[ph] < r.d.nspecies)
                           ? walk_sort_items(ctx->h_walk_sort[4 * i + w.species[ph]], w.kind[ph], cpi) : 0;
            switch (w.kind[ph]) {
            case W_PUSH: return r.t.ntiles;
            case W_SMOOTH_FOLD: return r.smooth > 0 ? (int)((ncell + cpi - 1) / cpi) : 0;
            case W_SMOOTH_PASS: return r.smooth > w.pass[ph] ? (int)((ncell + cpi - 1) / cpi) : 0;
            default: return (int)((r.g.pcells + cpi - 1) / cpi);
            }
        };
        int *prefix = ctx->h_walk.data(), *base = prefix + np * nr + 1, *order = base + nr * (np + 1);
        // slots of a phase: runs by decreasing particles per tile (the longest push items first)
        std::vector<double> load(nr, 0.0);
        for (int i = 0; i < nr; ++i) {
            const Run &r = ctx->runs[i];
            for (int q = 0; q < r.d.nspecies; ++q) load[i] += (double)r.sp[q].n;
            load[i] /= std::max(1, r.t.ntiles);
            order[i] = i;
        }
        std::stable_sort(order, order + nr, [&](int a, int b) { return load[a] > load[b]; });
        int total = 0;
        for (int ph = 0; ph < np; ++ph)
            for (int k = 0; k < nr; ++k) {
                prefix[ph * nr + k] = total;
                total += items(ph, order[k]);
            }
        prefix[np * nr] = total;
        for (int i = 0; i < nr; ++i) {
            base[i * (np + 1)] = 0;
            for (int ph = 0; ph < np; ++ph) base[i * (np + 1) + ph + 1] = base[i * (np + 1) + ph] + items(ph, i);
        }
        // test hook: the push of run 0 waits for an item that does not exist
        if (ctx->flags & PIC_FLAG_INJECT_STALL) base[ph_push] += 1;
        const size_t tab = sizeof(int) * ((size_t)np * nr + 1 + (size_t)nr * (np + 2));
        CK(cudaMemcpyAsync(ctx->walk_tab, host_src(ctx, slot, soff, ctx->h_walk.data(), tab), tab,
                           cudaMemcpyHostToDevice, s));
        if (!due.empty() && walk_sort)
            CK(cudaMemcpyAsync(ctx->walk_sort_dev,
                               host_src(ctx, slot, soff, ctx->h_walk_sort.data(), sizeof(SortArgs) * 4 * nr),
                               sizeof(SortArgs) * 4 * nr, cudaMemcpyHostToDevice, s));
        CK(cudaMemsetAsync(ctx->walk_ctl, 0, sizeof(int) * (2 + nr), s));
        w.sort = ctx->walk_sort_dev;
        w.push = ctx->multi_args;
        w.fe = ctx->multi_fe;
        w.fp = ctx->multi_fp;
        w.prefix = ctx->walk_tab;
        w.base = ctx->walk_tab + np * nr + 1;
        w.order = w.base + nr * (np + 1);
        w.head = ctx->walk_ctl;
        w.abort = ctx->walk_ctl + 1;
        w.done = ctx->walk_ctl + 2;
        w.err = ctx->d_err;
        w.nruns = nr;
        w.nphase = np;
        w.total = total;
        w.cells_per_item = cpi;
        w.h = 0.5f * dt;
        w.dt = dt;
        w.wait_ns = (ctx->flags & PIC_FLAG_INJECT_STALL) ? 20000000LL : 2000000000LL;
        launch_walk(w, ndim, walls, count, push_smem, fixed_tile_code(ctx->runs[0].t, ndim), s);
        CK(cudaGetLastError());
        if (count)
            for (auto &r : ctx->runs)
                for (int q = 0; q < r.d.nspecies; ++q) r.sp[q].counted = true;
        for (auto &r : ctx->runs) {
            r.since_sort++;
            r.jcur = 1 - r.jcur;
            r.step++;
            if (r.hist_n < r.hist_cap) r.hist_n++;
        }
        ctx->launch_total += launches + 1;
        ctx->bytes_per_ps = ndim == 2 ? 48.0 : 56.0;
        return PIC_OK;
    }
    {
        KTimer t(ctx, PIC_KERNEL_FIELD);
        launch_fields_multi(FIELD_B_HALF, ctx->multi_fe, ctx->multi_blocks, ctx->multi_nblocks, nr, 0.5f * dt, dt, s);
        launch_fields_multi(FIELD_NODE, ctx->multi_fp, ctx->multi_blocks, ctx->multi_nblocks, nr, 0.5f * dt, dt, s);
    }
    {
        KTimer t(ctx, PIC_KERNEL_PUSH);
        CK(cudaMemsetAsync(ctx->multi_counter, 0, sizeof(int), s));
        launch_push_mixed_multi(ctx->multi_args, ctx->multi_tiles, nr, ctx->runs[0].d.ndim, ctx->runs[0].t,
                                ctx->runs[0].g.bcx == 1, count, ctx->multi_counter, s);
        if (count)
            for (auto &r : ctx->runs)
                for (int q = 0; q < r.d.nspecies; ++q) r.sp[q].counted = true;
    }
    if (max_smooth > 0) {
        KTimer t(ctx, PIC_KERNEL_SMOOTH);
        launch_smooth_multi(0, 0, ctx->multi_fp, ctx->multi_blocks, ctx->multi_nblocks, nr, s);
        for (int p = 0; p < max_smooth; ++p)
            launch_smooth_multi(1, p, ctx->multi_fp, ctx->multi_blocks, ctx->multi_nblocks, nr, s);
        launches += 1 + max_smooth;
    }
    {
        KTimer t(ctx, PIC_KERNEL_FIELD);
        launch_fields_multi(FIELD_B_HALF, ctx->multi_fp, ctx->multi_blocks, ctx->multi_nblocks, nr, 0.5f * dt, dt, s);
        launch_fields_multi(FIELD_E_FX, ctx->multi_fp, ctx->multi_blocks, ctx->multi_nblocks, nr, 0.5f * dt, dt, s);
    }
    for (auto &r : ctx->runs) {
        r.since_sort++;
        r.jcur = 1 - r.jcur;
        r.step++;
        if (r.hist_n < r.hist_cap) r.hist_n++;
    }
    ctx->launch_total += launches + 5;
    ctx->bytes_per_ps = ctx->runs[0].d.ndim == 2 ? 48.0 : 56.0;
    return PIC_OK;
}

// Current smoothing of one run (main-loop step 10): folds the deposited current
// J into sbuf[0] and applies the passes; returns the smoothed compact current,
// or nullptr when the run does not smooth.
template <typename JT>
const typename SmoothValue<JT>::type *smooth_current(pic_ctx *ctx, Run &r, JT *const J[3]) {
    typedef typename SmoothValue<JT>::type T;
    if (r.smooth <= 0) return nullptr;
    KTimer t(ctx, PIC_KERNEL_SMOOTH);
    T *const buf[2] = {(T *)r.sbuf[0], (T *)r.sbuf[1]};
    return launch_smooth_current<JT>(r.g, J, r.smooth, buf, ctx->stream);
}

void step_run(pic_ctx *ctx, Run &r) {
    cudaStream_t s = ctx->stream;
    double *hslot = (r.hist_n < r.hist_cap) ? r.hist + 8 * r.hist_n : nullptr;
    const int nsp = r.d.nspecies;
    if (ctx->precision == PIC_FP64) {
        FieldPtrs<double> f = fields_of<double>(r);
        {
            KTimer t(ctx, PIC_KERNEL_FIELD);
            launch_b_advance<double>(r.g, f, 0.5 * r.d.dt, HistRef{hslot, nullptr, 0}, s);
        }
        double *J[3] = {jplane<double>(r, r.jcur, 0), jplane<double>(r, r.jcur, 1), jplane<double>(r, r.jcur, 2)};
        {
            KTimer t(ctx, PIC_KERNEL_PUSH);
            for (int q = 0; q < nsp; ++q) {
                SpeciesState &S = r.sp[q];
                launch_push_fp64(r.g, f, J, S.s64, S.n, S.h, S.alpha, r.d.dt, 0, S.m_over_me, hslot, ctx->d_err, s);
            }
        }
        double *Z[3] = {jplane<double>(r, 1 - r.jcur, 0), jplane<double>(r, 1 - r.jcur, 1),
                        jplane<double>(r, 1 - r.jcur, 2)};
        const double *Jc[3] = {J[0], J[1], J[2]};
        const double *Js = smooth_current<double>(ctx, r, J);
        {
            KTimer t(ctx, PIC_KERNEL_FIELD);
            launch_b_advance<double>(r.g, f, 0.5 * r.d.dt, HistRef{nullptr, nullptr, 0}, s);
            if (Js) launch_e_advance_smoothed<double, double, double>(r.g, f, Js, 1.0, Z, r.d.dt, nullptr, s);
            else launch_e_advance<double>(r.g, f, Jc, Z, r.d.dt, s);
        }
        ctx->bytes_per_ps = r.d.ndim == 2 ? 80.0 : 96.0;
        ctx->launch_total += 3 + nsp + (Js ? r.smooth : 0);
    } else {
        int launches = 0;
        if (!r.sorted || r.since_sort >= r.sort_interval) {
            KTimer t(ctx, PIC_KERNEL_SORT);
            for (int q = 0; q < nsp; ++q) {
                launches += r.sp[q].counted ? 6 : 8;
                sort_species(ctx, r, r.sp[q]);
            }
            r.sorted = true;
            r.since_sort = 0;
        }
        FieldPtrs<float> f = fields_of<float>(r);
        {
            KTimer t(ctx, PIC_KERNEL_FIELD);
            launch_b_advance<float>(r.g, f, 0.5f * (float)r.d.dt, hist_ref(r), s);
            launch_node_fields(r.g, f, r.nfA, r.nfB, s);
        }
        typedef unsigned long long u64;
        u64 *J[3] = {jplane<u64>(r, r.jcur, 0), jplane<u64>(r, r.jcur, 1), jplane<u64>(r, r.jcur, 2)};
        {
            KTimer t(ctx, PIC_KERNEL_PUSH);
            MixedStepArgs a;
            a.g = r.g;
            a.t = r.t;
            a.nfA = r.nfA;
            a.nfB = r.nfB;
            for (int c = 0; c < 3; ++c) a.J[c] = J[c];
            a.nspecies = nsp;
            for (int q = 0; q < nsp; ++q) {
                SpeciesState &S = r.sp[q];
                a.sp[q] = S.mb[S.cur];
                a.tile_start[q] = S.tile_start;
                a.h[q] = (float)S.h;
                a.sgn[q] = S.q_over_e > 0 ? 1.f : -1.f;
                a.m_over_me[q] = S.m_over_me;
            }
            a.dt = (float)r.d.dt;
            a.mode = 0;
            a.hist = hist_ref(r);
            a.err = ctx->d_err;
            a.use_tma = r.tma ? 1 : 0;
            a.tmA = r.tmA;
            a.tmB = r.tmB;
            // when the next step sorts, this push counts its key histogram
            const bool count = r.since_sort + 1 >= r.sort_interval && r.t.lg[0] >= 0;
            prepare_counts(ctx, r);
            for (int q = 0; q < 4; ++q) a.key_counts[q] = (count && q < nsp) ? r.sp[q].counts : nullptr;
            launch_push_mixed(a, s);
            if (count)
                for (int q = 0; q < nsp; ++q) r.sp[q].counted = true;
        }
        u64 *Z[3] = {jplane<u64>(r, 1 - r.jcur, 0), jplane<u64>(r, 1 - r.jcur, 1), jplane<u64>(r, 1 - r.jcur, 2)};
        const u64 *Jc[3] = {J[0], J[1], J[2]};
        const long long *Js = smooth_current<u64>(ctx, r, J);
        {
            KTimer t(ctx, PIC_KERNEL_FIELD);
            const double alpha_abs = 2.0 / (r.d.n_x * r.d.n_x * r.d.rho_sp0);
            launch_b_advance<float>(r.g, f, 0.5f * (float)r.d.dt, HistRef{nullptr, nullptr, 0}, s);
            if (Js)
                launch_e_advance_smoothed<float, u64, long long>(r.g, f, Js, alpha_abs * 0x1p-36, Z, (float)r.d.dt,
                                                                 r.hist_idx, s);
            else launch_e_advance_fx(r.g, f, Jc, Z, (float)r.d.dt, alpha_abs, r.hist_idx, s);
        }
        r.since_sort++;
        launches += 5 + (Js ? 1 + r.smooth : 0);   // shell fold + passes
        ctx->launch_total += launches;
        ctx->bytes_per_ps = r.d.ndim == 2 ? 48.0 : 56.0;
    }
    r.jcur = 1 - r.jcur;
    r.step++;
    if (r.hist_n < r.hist_cap) r.hist_n++;
}

}  // namespace

pic_status mlp_load(pic_ctx *ctx, int run, int species, long long n, double theta, const double beta[3], int profile,
                    double L, double x0, int colocate_with, uint64_t seed);

namespace {

pic_status one_step(pic_ctx *ctx, int slot) {
    if (ctx->multi) return step_multi(ctx, slot);
    for (auto &r : ctx->runs) step_run(ctx, r);
    return PIC_OK;
}

int graph_period_of(const pic_ctx *ctx) { return 2 * std::max(1, ctx->runs[0].sort_interval); }

// A period of 2K steps (K = sort interval) starting with a sort brings every
// alternating buffer (current planes, particle buffers, tile offsets) back to
// where it started, so its launches can be replayed as long as each period
// starts in this phase.
bool graph_aligned(const pic_ctx *ctx) {
    if (ctx->multi_tiles_dirty) return false;
    for (const auto &r : ctx->runs) {
        if (!r.sorted || r.since_sort < r.sort_interval || r.sort_interval != ctx->runs[0].sort_interval) return false;
        for (int q = 0; q < r.d.nspecies; ++q)
            if (!r.sp[q].tiled || r.sp[q].tiled_ntiles != r.t.ntiles) return false;
    }
    return true;
}

// Everything the launches of a period depend on.
std::vector<long long> graph_signature(const pic_ctx *ctx) {
    std::vector<long long> v;
    v.push_back((long long)(uintptr_t)ctx->stream);
    v.push_back(ctx->flags & PIC_FLAG_PHASE_LAUNCHES);
    for (const auto &r : ctx->runs) {
        v.push_back(r.jcur);
        v.push_back(r.sort_interval);
        for (int a = 0; a < 3; ++a) v.push_back(r.t.T[a]);
        for (int q = 0; q < r.d.nspecies; ++q) {
            const SpeciesState &S = r.sp[q];
            v.push_back(S.cur);
            v.push_back(S.counted);
            v.push_back(S.n);
            v.push_back((long long)(uintptr_t)S.tile_start);
            v.push_back((long long)(uintptr_t)S.tile_start_alt);
        }
    }
    return v;
}

// Host counters that do not cycle with the period.
void advance_counters(pic_ctx *ctx, int P) {
    for (auto &r : ctx->runs) {
        r.step += P;
        r.hist_n = std::min<int64_t>(r.hist_n + P, r.hist_cap);
    }
}

struct HostSnapshot {
    std::vector<Run> runs;
};

pic_status capture_graph(pic_ctx *ctx) {
    const int P = graph_period_of(ctx);
    if (ctx->graph) { cudaGraphExecDestroy(ctx->graph); ctx->graph = nullptr; }
    if (!ctx->cap_stream && cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return PIC_ECUDA;
    const int nr = (int)ctx->runs.size();
    if (ctx->multi) {
        int maxsp = 0;
        for (auto &r : ctx->runs) maxsp = std::max(maxsp, r.d.nspecies);
        const size_t a = 256;
        auto up = [a](size_t b) { return (b + a - 1) & ~(a - 1); };
        const size_t stride = up(sizeof(MixedStepArgs) * nr) + 2 * up(sizeof(FieldRunF) * nr) +
                              maxsp * (up(sizeof(SortArgs) * nr) + up(sizeof(int) * 4 * (nr + 1))) +
                              up(sizeof(int) * walk_tab_ints(nr)) + up(sizeof(SortArgs) * 4 * nr);
        if (ctx->gstage_bytes < stride * P) {
            if (ctx->gstage) cudaFreeHost(ctx->gstage);
            ctx->gstage = nullptr;
            ctx->gstage_bytes = 0;
            if (cudaMallocHost((void **)&ctx->gstage, stride * P) != cudaSuccess) return PIC_ENOMEM;
            ctx->gstage_bytes = stride * P;
        }
        ctx->gstage_stride = stride;
    }
    // the host bookkeeping of the period is done once, during the capture
    HostSnapshot snap{ctx->runs};
    const std::vector<long long> sig = graph_signature(ctx);
    cudaStream_t user = ctx->stream;
    ctx->stream = ctx->cap_stream;
    ctx->capturing = true;
    const int64_t launches0 = ctx->launch_total;
    pic_status st = PIC_OK;
    if (cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) st = PIC_ECUDA;
    for (int p = 0; p < P && st == PIC_OK; ++p) st = one_step(ctx, p);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(ctx->cap_stream, &g);
    ctx->capturing = false;
    ctx->stream = user;
    if (st == PIC_OK && (ec != cudaSuccess || !g)) st = PIC_ECUDA;
    if (st == PIC_OK && cudaGraphInstantiate(&ctx->graph, g, 0) != cudaSuccess) {
        ctx->graph = nullptr;
        st = PIC_ECUDA;
    }
    if (g) cudaGraphDestroy(g);
    if (st != PIC_OK) {
        cudaGetLastError();   // clear a capture error; nothing was launched
        ctx->runs = snap.runs;
        ctx->graph_sig.clear();
        return st;
    }
    // the host state has cycled back; the signature must match for replays
    if (graph_signature(ctx) != sig) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
        ctx->runs = snap.runs;
        return PIC_ESTATE;
    }
    ctx->graph_sig = sig;
    ctx->graph_period = P;
    ctx->graph_launches = ctx->launch_total - launches0;
    return PIC_OK;
}

}  // namespace

// ================================================================== ABI

extern "C" {

int pic_abi_version(void) { return PIC_ABI_VERSION; }

pic_status pic_init(const pic_run_desc *runs, int nruns, const pic_opts *opts, pic_ctx **out) {
    if (!out) return PIC_EINVAL;
    *out = nullptr;
    if (!runs || nruns < 1) return PIC_EINVAL;
    const int precision = opts ? opts->precision : PIC_FP64;
    if (precision != PIC_FP64 && precision != PIC_MIXED) return PIC_EINVAL;
    for (int r = 0; r < nruns; ++r) {
        std::string why;
        if (!validate(runs[r], precision, why)) return PIC_EINVAL;
    }
    if (opts && opts->allocator && (!opts->allocator->alloc || !opts->allocator->free)) return PIC_EINVAL;
    if (opts && (opts->sort_interval < 0 || opts->tile[0] < 0 || opts->tile[1] < 0 || opts->tile[2] < 0))
        return PIC_EINVAL;
    pic_ctx *ctx = new pic_ctx();
    ctx->precision = precision;
    ctx->flags = opts ? opts->flags : 0;
    ctx->stream = opts ? (cudaStream_t)opts->stream : nullptr;
    if (opts && opts->allocator) { ctx->alloc = *opts->allocator; ctx->have_alloc = true; }
    ctx->runs.resize(nruns);
    ctx->d_err = (int *)dev_alloc(ctx, sizeof(int));
    if (!ctx->d_err) { pic_destroy(ctx); return PIC_ENOMEM; }
    if (cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream) != cudaSuccess) { pic_destroy(ctx); return PIC_ECUDA; }
    size_t stage = 0;
    for (int r = 0; r < nruns; ++r) {
        ctx->runs[r].d = runs[r];
        pic_status st = setup_run(ctx, ctx->runs[r], opts);
        if (st != PIC_OK) { pic_destroy(ctx); return st; }
        const Geom &g = ctx->runs[r].g;
        stage = std::max(stage, sizeof(double) * (size_t)g.nx * g.ny * g.nz);
        int64_t cap = 0;
        for (int s = 0; s < runs[r].nspecies; ++s) cap = std::max<int64_t>(cap, runs[r].species[s].capacity);
        stage = std::max(stage, 6 * sizeof(double) * (size_t)std::min<int64_t>(cap, 1 << 24));
    }
    if (precision == PIC_MIXED && nruns > 1) {
        // one batched step for all runs: they must share ndim and tile geometry
        const Run &r0 = ctx->runs[0];
        for (int r = 1; r < nruns; ++r) {
            const Run &rr = ctx->runs[r];
            if (rr.d.ndim != r0.d.ndim || rr.t.H != r0.t.H || rr.t.T[0] != r0.t.T[0] || rr.t.T[1] != r0.t.T[1] ||
                rr.t.T[2] != r0.t.T[2] || rr.sort_interval != r0.sort_interval || rr.g.bcx != r0.g.bcx) {
                pic_destroy(ctx);
                return PIC_EINVAL;
            }
        }
        ctx->multi = true;
        ctx->multi_args = (MixedStepArgs *)dev_alloc(ctx, sizeof(MixedStepArgs) * nruns);
        ctx->multi_fe = (FieldRunF *)dev_alloc(ctx, sizeof(FieldRunF) * nruns);
        ctx->multi_fp = (FieldRunF *)dev_alloc(ctx, sizeof(FieldRunF) * nruns);
        ctx->multi_tiles = (int *)dev_alloc(ctx, sizeof(int) * (nruns + 1));
        ctx->multi_blocks = (int *)dev_alloc(ctx, sizeof(int) * (nruns + 1));
        ctx->multi_counter = (int *)dev_alloc(ctx, sizeof(int));
        ctx->walk_tab = (int *)dev_alloc(ctx, sizeof(int) * walk_tab_ints(nruns));
        ctx->walk_ctl = (int *)dev_alloc(ctx, sizeof(int) * (2 + nruns));
        ctx->h_walk.resize(walk_tab_ints(nruns));
        ctx->walk_sort_dev = (SortArgs *)dev_alloc(ctx, sizeof(SortArgs) * 4 * nruns);
        ctx->h_walk_sort.assign(4 * (size_t)nruns, SortArgs{});
        ctx->sort_args_dev = (SortArgs *)dev_alloc(ctx, sizeof(SortArgs) * nruns);
        ctx->sort_prefix_dev = (int *)dev_alloc(ctx, sizeof(int) * 4 * (nruns + 1));
        ctx->h_sort.resize(nruns);
        ctx->h_sort_prefix.resize(4 * (nruns + 1));
        if (!ctx->multi_args || !ctx->multi_fe || !ctx->multi_fp || !ctx->multi_tiles || !ctx->multi_blocks ||
            !ctx->multi_counter || !ctx->sort_args_dev || !ctx->sort_prefix_dev || !ctx->walk_tab || !ctx->walk_ctl ||
            !ctx->walk_sort_dev) {
            pic_destroy(ctx);
            return PIC_ENOMEM;
        }
        std::vector<int> tp(nruns + 1, 0), bp(nruns + 1, 0);
        for (int r = 0; r < nruns; ++r) {
            tp[r + 1] = tp[r] + ctx->runs[r].t.ntiles;
            bp[r + 1] = bp[r] + (int)((ctx->runs[r].g.pcells + 255) / 256);
        }
        ctx->multi_nblocks = bp[nruns];
        if (cudaMemcpy(ctx->multi_tiles, tp.data(), sizeof(int) * (nruns + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(ctx->multi_blocks, bp.data(), sizeof(int) * (nruns + 1), cudaMemcpyHostToDevice) != cudaSuccess) {
            pic_destroy(ctx);
            return PIC_ECUDA;
        }
        ctx->h_args.resize(nruns);
        ctx->h_fe.resize(nruns);
        ctx->h_fp.resize(nruns);
    }
    stage = std::max<size_t>(stage, 1 << 16);
    ctx->staging_bytes = stage;
    ctx->staging = dev_alloc(ctx, stage);
    ctx->mj_table = (double *)dev_alloc(ctx, sizeof(double) * (kMjTable + 1));
    const int ncombo = kMlpTheta * kMlpBeta;
    ctx->mlpW = (float *)dev_alloc(ctx, sizeof(float) * kMlpParams);
    ctx->mlpG = (float *)dev_alloc(ctx, sizeof(float) * kMlpParams);
    ctx->mlpM = (float *)dev_alloc(ctx, sizeof(float) * kMlpParams);
    ctx->mlpV = (float *)dev_alloc(ctx, sizeof(float) * kMlpParams);
    ctx->mlpWh = dev_alloc(ctx, 2 * kMlpParams);
    ctx->mlpX = (float *)dev_alloc(ctx, sizeof(float) * 3 * kMlpBatchMax);
    ctx->mlpT = (float *)dev_alloc(ctx, sizeof(float) * kMlpBatchMax);
    ctx->mlpLoss = (double *)dev_alloc(ctx, sizeof(double));
    ctx->mlpF = (double *)dev_alloc(ctx, sizeof(double) * (size_t)ncombo * (kMjTable + 1));
    ctx->mlpPar = (double *)dev_alloc(ctx, sizeof(double) * 8 * ncombo);
    if (!ctx->staging || !ctx->mj_table || !ctx->mlpW || !ctx->mlpG || !ctx->mlpM || !ctx->mlpV || !ctx->mlpWh ||
        !ctx->mlpX || !ctx->mlpT || !ctx->mlpLoss || !ctx->mlpF || !ctx->mlpPar) {
        pic_destroy(ctx);
        return PIC_ENOMEM;
    }
    if (cudaMemsetAsync(ctx->mlpG, 0, sizeof(float) * kMlpParams, ctx->stream) != cudaSuccess) {
        pic_destroy(ctx);
        return PIC_ECUDA;
    }
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) { pic_destroy(ctx); return PIC_ECUDA; }
    *out = ctx;
    return PIC_OK;
}

void pic_destroy(pic_ctx *ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->io_stream) cudaStreamSynchronize(ctx->io_stream), cudaStreamDestroy(ctx->io_stream);
    for (auto e : ctx->io_ev)
        if (e) cudaEventDestroy(e);
    if (ctx->gstage) cudaFreeHost(ctx->gstage);
    for (int k = 0; k < kKernelClasses; ++k)
        for (auto &pr : ctx->ev_pending[k]) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
    for (auto e : ctx->ev_pool) cudaEventDestroy(e);
    for (auto &a : ctx->allocs) {
        if (ctx->have_alloc) ctx->alloc.free(a.first, a.second, ctx->alloc.user);
        else cudaFree(a.first);
    }
    delete ctx;
}

const char *pic_last_error(const pic_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

pic_status pic_set_state(pic_ctx *ctx, int run, const pic_state_view *in) {
    pic_status st = check_run(ctx, run);
    if (st) return st;
    if (!in || !in->fields) return fail(ctx, PIC_EINVAL, "null state view or field buffer");
    Run &r = ctx->runs[run];
    const Geom &g = r.g;
    const long long ncell = (long long)g.nx * g.ny * g.nz;
    // counts and buffers are checked here; every value is checked on the device as it is converted
    for (int s = 0; s < r.d.nspecies; ++s) {
        const int64_t n = in->count[s];
        if (n < 0 || n > r.sp[s].cap) return fail(ctx, PIC_EINVAL, "species %d: count %lld exceeds capacity", s, (long long)n);
        if (n > 0 && !in->particles[s]) return fail(ctx, PIC_EINVAL, "species %d: null particle buffer", s);
    }
    cudaStream_t sm = ctx->stream;
    {
        // errors of earlier calls do not belong to this one
        pic_status st0 = read_err(ctx);
        (void)st0;
    }
    if (ctx->precision == PIC_MIXED && (st = io_ready(ctx)) != PIC_OK) return st;
    double *stg = (double *)ctx->staging;
    // page-locked host buffers are read by the conversion kernels directly
    const double *fmap = mapped_host(in->fields, sizeof(double) * 6 * ncell);
    for (int c = 0; c < 6; ++c) {
        const double *src = fmap ? fmap + c * ncell : stg;
        if (!fmap) CK(cudaMemcpyAsync(stg, in->fields + c * ncell, sizeof(double) * ncell, cudaMemcpyHostToDevice, sm));
        if (ctx->precision == PIC_FP64)
            k_pad_field<double><<<nblk(g.pcells), 256, 0, sm>>>(g, src, (double *)r.F + c * g.pcells, nullptr,
                                                                ctx->d_err);
        else   // e keeps its low-order part (plane 6 + c); b is FP32
            k_pad_field<float><<<nblk(g.pcells), 256, 0, sm>>>(
                g, src, (float *)r.F + c * g.pcells, c < 3 ? (float *)r.F + (6 + c) * g.pcells : nullptr, ctx->d_err);
        CK(cudaGetLastError());
    }
    CK(cudaMemsetAsync(r.J, 0, 6 * 8 * g.pcells, sm));
    r.jcur = 0;
    for (int s = 0; s < r.d.nspecies; ++s) {
        SpeciesState &S = r.sp[s];
        const int64_t n = in->count[s];
        S.n = n;
        const double *P = in->particles[s];
        if (ctx->precision == PIC_FP64) {
            for (int a = 0; a < 3; ++a) {
                if (n == 0) break;
                if (a < g.ndim) CK(cudaMemcpyAsync(S.s64.x[a], P + a * n, sizeof(double) * n, cudaMemcpyHostToDevice, sm));
                else CK(cudaMemsetAsync(S.s64.x[a], 0, sizeof(double) * n, sm));
                CK(cudaMemcpyAsync(S.s64.u[a], P + (3 + a) * n, sizeof(double) * n, cudaMemcpyHostToDevice, sm));
            }
            if (n > 0) k_check64<<<nblk(n), 256, 0, sm>>>(g, S.s64, n, ctx->d_err);
        } else {
            S.cur = 0;
            S.tiled = false;
            S.counted = false;
            if (const double *Pm = mapped_host(P, sizeof(double) * 6 * (size_t)n)) {
                k_upload_mixed<<<nblk(n), 256, 0, sm>>>(g, Pm, n, n, 0, S.mb[0], ctx->d_err);
                CK(cudaGetLastError());
                continue;
            }
            // chunk c is copied into half c % 2 on the transfer stream while the
            // previous chunk is converted on the context stream
            const size_t half = (ctx->staging_bytes / 2) & ~size_t(255);
            double *hb[2] = {stg, (double *)((char *)stg + half)};
            const int64_t chunk = std::max<int64_t>(1, (int64_t)(half / (6 * sizeof(double))));
            cudaStream_t io = ctx->io_stream;
            CK(cudaEventRecord(ctx->io_ev[0], sm));
            CK(cudaStreamWaitEvent(io, ctx->io_ev[0], 0));
            bool used[2] = {false, false};
            int c = 0;
            for (int64_t a0 = 0; a0 < n; a0 += chunk, ++c) {
                const int b = c & 1;
                const int64_t m = std::min(chunk, n - a0);
                if (used[b]) CK(cudaStreamWaitEvent(io, ctx->io_ev[3 + b], 0));   // its last reader is done
                for (int a = 0; a < 6; ++a) {
                    if (a == 2 && g.ndim == 2) continue;
                    CK(cudaMemcpyAsync(hb[b] + a * m, P + a * n + a0, sizeof(double) * m, cudaMemcpyHostToDevice, io));
                }
                CK(cudaEventRecord(ctx->io_ev[1 + b], io));
                CK(cudaStreamWaitEvent(sm, ctx->io_ev[1 + b], 0));
                k_upload_mixed<<<nblk(m), 256, 0, sm>>>(g, hb[b], m, m, a0, S.mb[0], ctx->d_err);
                CK(cudaGetLastError());
                CK(cudaEventRecord(ctx->io_ev[3 + b], sm));
                used[b] = true;
            }
        }
    }
    r.sorted = false;
    r.since_sort = 0;
    r.step = 0;
    r.hist_n = 0;
    CK(cudaMemsetAsync(r.hist, 0, sizeof(double) * 8 * r.hist_cap, sm));
    CK(cudaMemsetAsync(r.hist_idx, 0, sizeof(long long), sm));
    return read_err(ctx);
}

pic_status pic_get_state(pic_ctx *ctx, int run, pic_state_view *out) {
    pic_status st = check_run(ctx, run);
    if (st) return st;
    if (!out || !out->fields) return fail(ctx, PIC_EINVAL, "null state view or field buffer");
    Run &r = ctx->runs[run];
    const Geom &g = r.g;
    const long long ncell = (long long)g.nx * g.ny * g.nz;
    for (int s = 0; s < r.d.nspecies; ++s) {
        if (!out->particles[s]) continue;   // fields only for this species
        if (out->count[s] < r.sp[s].n)
            return fail(ctx, PIC_EINVAL, "species %d: buffer holds %lld particles, %lld needed", s,
                        (long long)out->count[s], (long long)r.sp[s].n);
    }
    cudaStream_t sm = ctx->stream;
    double *stg = (double *)ctx->staging;
    // page-locked host buffers are written by the conversion kernels directly
    double *fmap = mapped_host(out->fields, sizeof(double) * 6 * ncell);
    for (int c = 0; c < 6; ++c) {
        double *dst = fmap ? fmap + c * ncell : stg;
        if (ctx->precision == PIC_FP64)
            k_unpad_field<double><<<nblk(ncell), 256, 0, sm>>>(g, (double *)r.F + c * g.pcells, nullptr, dst);
        else
            k_unpad_field<float><<<nblk(ncell), 256, 0, sm>>>(
                g, (float *)r.F + c * g.pcells, c < 3 ? (float *)r.F + (6 + c) * g.pcells : nullptr, dst);
        if (!fmap)
            CK(cudaMemcpyAsync(out->fields + c * ncell, stg, sizeof(double) * ncell, cudaMemcpyDeviceToHost, sm));
    }
    for (int s = 0; s < r.d.nspecies; ++s) {
        SpeciesState &S = r.sp[s];
        const int64_t n = S.n;
        out->count[s] = n;
        double *P = out->particles[s];
        if (n == 0 || !P) continue;
        if (ctx->precision == PIC_FP64) {
            for (int a = 0; a < 3; ++a) {
                if (a < g.ndim) CK(cudaMemcpyAsync(P + a * n, S.s64.x[a], sizeof(double) * n, cudaMemcpyDeviceToHost, sm));
                CK(cudaMemcpyAsync(P + (3 + a) * n, S.s64.u[a], sizeof(double) * n, cudaMemcpyDeviceToHost, sm));
            }
            if (g.ndim == 2) std::memset(P + 2 * n, 0, sizeof(double) * n);
        } else {
            // conversion and copy in turn on the context stream (a copy stream of
            // its own measured slower here than this serial form); the id -> storage
            // index map lets each chunk touch only its own particles
            k_id_index<<<nblk(n), 256, 0, sm>>>(S.mb[S.cur].id, n, r.perm);
            if (double *Pm = mapped_host(P, sizeof(double) * 6 * (size_t)n)) {
                k_download_by_id<<<nblk(n), 256, 0, sm>>>(g, S.mb[S.cur], r.perm, 0, n, Pm, n);
                CK(cudaGetLastError());
                continue;
            }
            const int64_t chunk = (int64_t)(ctx->staging_bytes / (6 * sizeof(double)));
            for (int64_t a0 = 0; a0 < n; a0 += chunk) {
                const int64_t m = std::min(chunk, n - a0);
                k_download_by_id<<<nblk(m), 256, 0, sm>>>(g, S.mb[S.cur], r.perm, a0, m, stg, m);
                CK(cudaGetLastError());
                for (int a = 0; a < 6; ++a)
                    CK(cudaMemcpyAsync(P + a * n + a0, stg + a * m, sizeof(double) * m, cudaMemcpyDeviceToHost, sm));
            }
        }
    }
    out->step = r.step;
    CK(cudaStreamSynchronize(sm));
    return PIC_OK;
}

pic_status pic_get_particles(pic_ctx *ctx, int run, int species, const int64_t *ids, int64_t nids, double *out) {
    pic_status st = check_run(ctx, run);
    if (st) return st;
    Run &r = ctx->runs[run];
    if (species < 0 || species >= r.d.nspecies) return fail(ctx, PIC_EINVAL, "species %d out of range", species);
    if (nids < 0 || (nids > 0 && (!ids || !out))) return fail(ctx, PIC_EINVAL, "null ids or output");
    SpeciesState &S = r.sp[species];
    for (int64_t q = 0; q < nids; ++q)
        if (ids[q] < 0 || ids[q] >= S.n) return fail(ctx, PIC_EINVAL, "id %lld out of range", (long long)ids[q]);
    cudaStream_t sm = ctx->stream;
    // staging holds 6 doubles per particle for `chunk` particles; the ids of a
    // chunk are copied behind them
    const int64_t chunk = (int64_t)(ctx->staging_bytes / (7 * sizeof(double)));
    double *stg = (double *)ctx->staging;
    if (ctx->precision == PIC_MIXED && S.n > 0)
        k_id_index<<<nblk(S.n), 256, 0, sm>>>(S.mb[S.cur].id, S.n, r.perm);
    for (int64_t a0 = 0; a0 < nids; a0 += chunk) {
        const int64_t m = std::min(chunk, nids - a0);
        long long *dids = reinterpret_cast<long long *>(stg + 6 * m);
        CK(cudaMemcpyAsync(dids, ids + a0, sizeof(long long) * m, cudaMemcpyHostToDevice, sm));
        if (ctx->precision == PIC_MIXED) k_pick_mixed<<<nblk(m), 256, 0, sm>>>(r.g, S.mb[S.cur], r.perm, dids, m, stg);
        else k_pick64<<<nblk(m), 256, 0, sm>>>(S.s64, dids, m, r.d.ndim, stg);
        CK(cudaGetLastError());
        for (int a = 0; a < 6; ++a)
            CK(cudaMemcpyAsync(out + a * nids + a0, stg + a * m, sizeof(double) * m, cudaMemcpyDeviceToHost, sm));
        CK(cudaStreamSynchronize(sm));
    }
    return PIC_OK;
}

pic_status pic_set_uniform_field(pic_ctx *ctx, int run, const double e0[3], const double b0[3]) {
    pic_status st = check_run(ctx, run);
    if (st) return st;
    if (!e0 || !b0) return fail(ctx, PIC_EINVAL, "null field vector");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(e0[a]) || !std::isfinite(b0[a])) return fail(ctx, PIC_ENUMERIC, "non-finite field vector");
    Run &r = ctx->runs[run];
    if (ctx->precision == PIC_FP64) launch_add_uniform<double>(r.g, fields_of<double>(r), e0, b0, ctx->stream);
    else launch_add_uniform<float>(r.g, fields_of<float>(r), e0, b0, ctx->stream);
    CK(cudaGetLastError());
    return PIC_OK;
}

pic_status pic_step(pic_ctx *ctx, int nsteps) {
    if (!ctx) return PIC_EINVAL;
    if (nsteps < 0) return fail(ctx, PIC_EINVAL, "nsteps must be >= 0");
    int n = 0;
    ctx->launch_total = 0;
    const bool graphs = ctx->precision == PIC_MIXED &&
                        !(ctx->flags & (PIC_FLAG_NO_GRAPH | PIC_FLAG_TIMING | PIC_FLAG_INJECT_STALL));
    while (n < nsteps) {
        if (graphs && graph_aligned(ctx) && nsteps - n >= graph_period_of(ctx)) {
            const int P = graph_period_of(ctx);
            if (!ctx->graph || ctx->graph_sig != graph_signature(ctx)) {
                if (capture_graph(ctx) != PIC_OK) {
                    // capture unavailable: launch this period directly
                    for (int q = 0; q < P; ++q) {
                        pic_status st = one_step(ctx, -1);
                        if (st) return st;
                    }
                    n += P;
                    continue;
                }
            } else {
                advance_counters(ctx, P);
                ctx->launch_total += ctx->graph_launches;
            }
            CK(cudaGraphLaunch(ctx->graph, ctx->stream));
            n += P;
            continue;
        }
        pic_status st = one_step(ctx, -1);
        if (st) return st;
        ++n;
    }
    if (nsteps > 0) ctx->launches_per_step = (ctx->launch_total + nsteps / 2) / nsteps;
    CK(cudaGetLastError());
    if (ctx->flags & PIC_FLAG_ASYNC) return PIC_OK;
    return read_err(ctx);
}

pic_status pic_set_flags(pic_ctx *ctx, uint32_t flags) {
    if (!ctx) return PIC_EINVAL;
    if (flags & ~(PIC_FLAG_ASYNC | PIC_FLAG_NO_GRAPH | PIC_FLAG_TIMING | PIC_FLAG_PHASE_LAUNCHES | PIC_FLAG_INJECT_STALL))
        return fail(ctx, PIC_EINVAL, "unknown flag bits");
    ctx->flags = flags;
    return PIC_OK;
}

pic_status pic_sync(pic_ctx *ctx) {
    if (!ctx) return PIC_EINVAL;
    CK(cudaGetLastError());
    return read_err(ctx);
}

pic_status pic_diagnostics(pic_ctx *ctx, int run, pic_diag *out) {
    pic_status st = check_run(ctx, run);
    if (st) return st;
    if (!out) return fail(ctx, PIC_EINVAL, "null output");
    Run &r = ctx->runs[run];
    const Geom &g = r.g;
    cudaStream_t sm = ctx->stream;
    const long long ncell = (long long)g.nx * g.ny * g.nz;
    const int nsp = r.d.nspecies;
    // acc layout: [0..5] field sums, [6 + 6 s ..] particle sums of species s,
    // [40] nonfinite (as long long), [41 + s] max |rho_s|, [48] gauss max
    CK(cudaMemsetAsync(r.acc, 0, sizeof(double) * 64, sm));
    long long *nonfinite = reinterpret_cast<long long *>(r.acc + 40);
    if (ctx->precision == PIC_FP64) launch_field_diag<double>(g, fields_of<double>(r), r.acc, nonfinite, sm);
    else launch_field_diag<float>(g, fields_of<float>(r), r.acc, nonfinite, sm);
    CK(cudaMemsetAsync(r.rho_tot, 0, sizeof(double) * ncell, sm));
    for (int s = 0; s < nsp; ++s) {
        SpeciesState &S = r.sp[s];
        CK(cudaMemsetAsync(r.rho_s, 0, sizeof(double) * ncell, sm));
        if (ctx->precision == PIC_FP64) {
            launch_particle_diag64(g, S.s64, S.n, S.m_over_me, r.acc + 6 + 6 * s, nonfinite, sm);
            launch_rho64(g, S.s64, S.n, S.alpha, r.rho_s, sm);
            launch_rho64(g, S.s64, S.n, S.alpha, r.rho_tot, sm);
        } else {
            launch_particle_diag_mixed(g, S.mb[S.cur], S.n, S.m_over_me, r.acc + 6 + 6 * s, nonfinite, sm);
            launch_rho_mixed(g, S.mb[S.cur], S.n, S.alpha, r.rho_s, sm);
            launch_rho_mixed(g, S.mb[S.cur], S.n, S.alpha, r.rho_tot, sm);
        }
        launch_max_abs_diff(r.rho_s, nullptr, ncell, r.acc + 41 + s, sm);
    }
    if (ctx->precision == PIC_FP64) launch_div_e<double>(g, fields_of<double>(r), r.divb, sm);
    else launch_div_e<float>(g, fields_of<float>(r), r.divb, sm);
    // with smoothing the conserved residual is div e - S rho~: smooth rho~ the
    // same number of times, alternating with rho_s as scratch
    double *rho_cmp = r.rho_tot;
    for (int p = 0; p < r.smooth; ++p) {
        double *other = rho_cmp == r.rho_tot ? r.rho_s : r.rho_tot;
        launch_smooth(g, rho_cmp, other, sm);
        rho_cmp = other;
    }
    launch_max_abs_diff(r.divb, rho_cmp, ncell, r.acc + 48, sm);
    CK(cudaGetLastError());
    double h[64];
    CK(cudaMemcpyAsync(h, r.acc, sizeof h, cudaMemcpyDeviceToHost, sm));
    CK(cudaStreamSynchronize(sm));
    std::memset(out, 0, sizeof *out);
    out->step = r.step;
    out->nspecies = nsp;
    for (int c = 0; c < 3; ++c) {
        out->field_e[c] = 0.5 * h[c] * r.inv_alpha_abs;
        out->field_b[c] = 0.5 * h[3 + c] * r.inv_alpha_abs;
    }
    out->rho_max = 0;
    for (int s = 0; s < nsp; ++s) {
        const double *v = h + 6 + 6 * s;
        out->count[s] = r.sp[s].n;
        out->kinetic[s] = r.sp[s].m_over_me * v[0];
        for (int c = 0; c < 3; ++c) out->sum_u[s][c] = v[1 + c];
        // T in units of m_e c^2: (m_s/m_e) <u . v> / 3 (Sect. 3.1.3)
        out->temperature[s] = r.sp[s].n > 0 ? r.sp[s].m_over_me * v[4] / (3.0 * (double)r.sp[s].n) : 0.0;
        out->rho_max = std::max(out->rho_max, h[41 + s]);
    }
    out->gauss_max = h[48];
    std::memcpy(&out->nonfinite, &h[40], sizeof(long long));
    return out->nonfinite ? fail(ctx, PIC_ENUMERIC, "%lld non-finite values", (long long)out->nonfinite) : PIC_OK;
}

pic_status pic_energy_history(pic_ctx *ctx, int run, double *out, int64_t max_steps, int64_t *nout) {
    pic_status st = check_run(ctx, run);
    if (st) return st;
    if (!nout || (max_steps > 0 && !out)) return fail(ctx, PIC_EINVAL, "null output");
    Run &r = ctx->runs[run];
    const int64_t n = std::min<int64_t>(r.hist_n, std::max<int64_t>(max_steps, 0));
    std::vector<double> h(8 * std::max<int64_t>(n, 1));
    if (n > 0) CK(cudaMemcpyAsync(h.data(), r.hist, sizeof(double) * 8 * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int64_t q = 0; q < n; ++q) {
        const double *v = &h[8 * q];
        out[4 * q + 0] = 0.5 * (v[0] + v[1]);
        out[4 * q + 1] = 0.5 * (v[2] + v[3] + v[4]) * r.inv_alpha_abs;
        out[4 * q + 2] = 0.5 * (v[5] + v[6] + v[7]) * r.inv_alpha_abs;
        out[4 * q + 3] = out[4 * q + 0] + out[4 * q + 1] + out[4 * q + 2];
    }
    *nout = n;
    return PIC_OK;
}

namespace {

struct TuneKey {
    int nruns, ndim;
    long long cells, particles;
    bool operator<(const TuneKey &o) const {
        if (nruns != o.nruns) return nruns < o.nruns;
        if (ndim != o.ndim) return ndim < o.ndim;
        if (cells != o.cells) return cells < o.cells;
        return particles < o.particles;
    }
};
struct TuneVal {
    int T[3];
    int K;
};
std::map<TuneKey, TuneVal> g_tune_cache;
std::mutex g_tune_mutex;

void apply_tuning(pic_ctx *ctx, const int T[3], int K) {
    for (auto &r : ctx->runs) {
        const TileGeom t = make_tile_geom(r.d, T, r.t.H);
        const bool same = t.T[0] == r.t.T[0] && t.T[1] == r.t.T[1] && t.T[2] == r.t.T[2];
        r.t = t;
        r.sort_interval = K;
        node_maps(r);
        if (!same) {
            r.sorted = false;
            for (int q = 0; q < r.d.nspecies; ++q) {
                r.sp[q].tiled = false;
                r.sp[q].counted = false;
            }
        }
    }
    ctx->multi_tiles_dirty = true;
}

}  // namespace

pic_status pic_autotune(pic_ctx *ctx, int max_steps, int tile[3], int *sort_interval, int *steps_taken) {
    if (!ctx) return PIC_EINVAL;
    if (max_steps < 0) return fail(ctx, PIC_EINVAL, "max_steps must be >= 0");
    int taken = 0;
    if (ctx->precision == PIC_MIXED) {
        const int ndim = ctx->runs[0].d.ndim;
        TuneKey key{(int)ctx->runs.size(), ndim, 0, 0};
        for (auto &r : ctx->runs) {
            key.cells += (long long)r.g.nx * r.g.ny * r.g.nz;
            for (int q = 0; q < r.d.nspecies; ++q) key.particles += r.sp[q].n;
        }
        key.particles = key.particles ? (long long)std::llround(std::log2((double)key.particles) * 4) : 0;
        TuneVal best{};
        bool have = false;
        {
            std::lock_guard<std::mutex> lk(g_tune_mutex);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) { best = it->second; have = true; }
        }
        if (!have) {
            double best_rate = -1.0;
            long long parts = 0;
            for (auto &r : ctx->runs)
                for (int q = 0; q < r.d.nspecies; ++q) parts += r.sp[q].n;
            cudaEvent_t e0, e1;
            CK(cudaEventCreate(&e0));
            CK(cudaEventCreate(&e1));
            for (auto &tc : tile_candidates(ndim)) {
                for (int K : sort_candidates(ndim)) {
                    const int n_trial = std::max(2 * K, 4);
                    if (taken + n_trial > max_steps) break;
                    const int T[3] = {tc[0], tc[1], tc[2]};
                    // a candidate whose tiles exceed the allocated tile arrays is skipped
                    bool fits = true;
                    for (auto &r : ctx->runs) {
                        const TileGeom t = make_tile_geom(r.d, T, r.t.H);
                        if (t.ntiles > r.max_tiles) fits = false;
                        if (mixed_smem_bytes(t, ndim) > kMaxPushSmem) fits = false;
                    }
                    if (!fits) continue;
                    apply_tuning(ctx, T, K);
                    CK(cudaEventRecord(e0, ctx->stream));
                    const uint32_t f = ctx->flags;
                    ctx->flags |= PIC_FLAG_ASYNC | PIC_FLAG_NO_GRAPH;
                    pic_status st = pic_step(ctx, n_trial);
                    ctx->flags = f;
                    if (st) return st;
                    CK(cudaEventRecord(e1, ctx->stream));
                    CK(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    CK(cudaEventElapsedTime(&ms, e0, e1));
                    taken += n_trial;
                    const double rate = (double)parts * n_trial / (ms * 1e6);
                    if (rate > best_rate) {
                        best_rate = rate;
                        best = TuneVal{{T[0], T[1], T[2]}, K};
                    }
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (best_rate < 0) {   // no trial fitted in max_steps: keep the current choice
                const Run &r0 = ctx->runs[0];
                best = TuneVal{{r0.t.T[0], r0.t.T[1], r0.t.T[2]}, r0.sort_interval};
            } else {
                std::lock_guard<std::mutex> lk(g_tune_mutex);
                g_tune_cache[key] = best;
            }
        }
        apply_tuning(ctx, best.T, best.K);
        pic_status st = read_err(ctx);
        if (st) return st;
    }
    const Run &r0 = ctx->runs[0];
    if (tile) for (int a = 0; a < 3; ++a) tile[a] = r0.t.T[a];
    if (sort_interval) *sort_interval = r0.sort_interval;
    if (steps_taken) *steps_taken = taken;
    return PIC_OK;
}

pic_status pic_get_tuning(const pic_ctx *ctx, int tile[3], int *sort_interval, int *halo) {
    if (!ctx || ctx->runs.empty()) return PIC_EINVAL;
    const Run &r = ctx->runs[0];
    if (tile) for (int a = 0; a < 3; ++a) tile[a] = r.t.T[a];
    if (sort_interval) *sort_interval = r.sort_interval;
    if (halo) *halo = r.t.H;
    return PIC_OK;
}

pic_status pic_get_counters(const pic_ctx *ctx, int64_t *launches_per_step, double *bytes_per_particle_step) {
    if (!ctx) return PIC_EINVAL;
    if (launches_per_step) *launches_per_step = ctx->launches_per_step;
    if (bytes_per_particle_step) *bytes_per_particle_step = ctx->bytes_per_ps;
    return PIC_OK;
}

pic_status pic_kernel_time(pic_ctx *ctx, int kernel_class, int reset, double *total_ms, int64_t *launches) {
    if (!ctx) return PIC_EINVAL;
    if (kernel_class < 0 || kernel_class >= kKernelClasses) return fail(ctx, PIC_EINVAL, "unknown kernel class");
    CK(cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < kKernelClasses; ++k) {
        for (auto &pr : ctx->ev_pending[k]) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) ctx->ev_ms[k] += ms;
            ctx->ev_n[k]++;
            ctx->ev_pool.push_back(pr.first);
            ctx->ev_pool.push_back(pr.second);
        }
        ctx->ev_pending[k].clear();
    }
    if (total_ms) *total_ms = ctx->ev_ms[kernel_class];
    if (launches) *launches = ctx->ev_n[kernel_class];
    if (reset) {
        for (int k = 0; k < kKernelClasses; ++k) { ctx->ev_ms[k] = 0; ctx->ev_n[k] = 0; }
    }
    return PIC_OK;
}

pic_status pic_load_maxwell_juttner(pic_ctx *ctx, int run, int species, double ppc, double theta, const double beta[3],
                                    int profile, const double *profile_params, int method, int colocate_with,
                                    uint64_t seed) {
    pic_status st = check_run(ctx, run);
    if (st) return st;
    Run &r = ctx->runs[run];
    const Geom &g = r.g;
    if (species < 0 || species >= r.d.nspecies) return fail(ctx, PIC_EINVAL, "species %d out of range", species);
    if (!(ppc > 0) || !std::isfinite(ppc)) return fail(ctx, PIC_EINVAL, "ppc must be positive");
    if (!(theta > 0) || !std::isfinite(theta)) return fail(ctx, PIC_EINVAL, "theta must be positive");
    if (!beta) return fail(ctx, PIC_EINVAL, "null beta");
    const double b2 = beta[0] * beta[0] + beta[1] * beta[1] + beta[2] * beta[2];
    if (!(b2 < 1.0) || !std::isfinite(b2)) return fail(ctx, PIC_EINVAL, "|beta| must be below 1");
    if (method != PIC_MJ_EXACT && method != PIC_MJ_NAIVE_BOOST && method != PIC_MJ_MLP)
        return fail(ctx, PIC_EINVAL, "unknown loader method %d", method);
    double L = 1.0, x0 = 0.0;
    long long n;
    if (profile == PIC_PROFILE_UNIFORM) {
        n = std::llround(ppc * (double)g.nx * g.ny * g.nz);
    } else if (profile == PIC_PROFILE_HARRIS) {
        if (!profile_params) return fail(ctx, PIC_EINVAL, "Harris profile needs L and x0");
        L = profile_params[0];
        x0 = profile_params[1];
        if (!(L > 0) || !(x0 >= 0 && x0 <= g.nx)) return fail(ctx, PIC_EINVAL, "Harris L must be > 0, 0 <= x0 <= nx");
        n = std::llround(ppc * (double)g.ny * g.nz * L * (std::tanh((g.nx - x0) / L) - std::tanh(-x0 / L)));
    } else {
        return fail(ctx, PIC_EINVAL, "unknown density profile %d", profile);
    }
    SpeciesState &S = r.sp[species];
    if (n > S.cap) return fail(ctx, PIC_EINVAL, "species %d: %lld particles exceed capacity %lld", species, n,
                               (long long)S.cap);
    int colocate = 0;
    SpeciesState *C = nullptr;
    if (colocate_with >= 0) {
        if (colocate_with >= r.d.nspecies || colocate_with == species)
            return fail(ctx, PIC_EINVAL, "colocate_with %d is not another species", colocate_with);
        C = &r.sp[colocate_with];
        if (C->n != n) return fail(ctx, PIC_EINVAL, "colocated species holds %lld particles, %lld needed",
                                   (long long)C->n, n);
        colocate = 1;
    }
    if (method == PIC_MJ_MLP) return mlp_load(ctx, run, species, n, theta, beta, profile, L, x0, colocate_with, seed);
    const int naive = method == PIC_MJ_NAIVE_BOOST;
    const double b0 = std::sqrt(b2);
    std::vector<double> F;
    double s0, h, psi, Z;
    build_marginal_table(theta, naive ? 0.0 : b0, kMjTable, F, s0, h, psi, Z);
    cudaStream_t sm = ctx->stream;
    CK(cudaMemcpyAsync(ctx->mj_table, F.data(), sizeof(double) * (kMjTable + 1), cudaMemcpyHostToDevice, sm));
    const bool mixed = ctx->precision == PIC_MIXED;
    if (mixed && C && C->cur != S.cur) {
        // keep both species in the same buffer slot so that positions can be read from the partner
        S.cur = C->cur;
    }
    Species64 d64 = S.s64, c64 = C ? C->s64 : S.s64;
    SpeciesMixed dmx = S.mb[S.cur], cmx = C ? C->mb[C->cur] : S.mb[S.cur];
    launch_load_mj(g, r.d.ndim, n, species, seed, profile, L, x0, theta, beta, naive, ctx->mj_table, s0, h,
                   kMjTable, psi, Z, colocate, d64, c64, dmx, cmx, mixed ? 1 : 0, ctx->d_err, sm);
    CK(cudaGetLastError());
    S.n = n;
    S.tiled = false;
    S.counted = false;
    r.sorted = false;
    r.since_sort = 0;
    // initial staggering of the momenta: one Boris step of -dt/2 (App. A.3.1)
    if (mixed) {
        FieldPtrs<float> f = fields_of<float>(r);
        launch_node_fields(g, f, r.nfA, r.nfB, sm);
        launch_half_back_mixed(g, r.nfA, r.nfB, S.mb[S.cur], n, (float)S.h, (float)r.d.dt, sm);
    } else {
        double *J[3] = {jplane<double>(r, r.jcur, 0), jplane<double>(r, r.jcur, 1), jplane<double>(r, r.jcur, 2)};
        launch_push_fp64(g, fields_of<double>(r), J, S.s64, n, S.h, S.alpha, r.d.dt, 1, S.m_over_me, nullptr,
                         ctx->d_err, sm);
    }
    CK(cudaGetLastError());
    r.step = 0;
    r.hist_n = 0;
    CK(cudaMemsetAsync(r.hist, 0, sizeof(double) * 8 * r.hist_cap, sm));
    CK(cudaMemsetAsync(r.hist_idx, 0, sizeof(long long), sm));
    return read_err(ctx);
}

}  // extern "C"

// ------------------------------------------------------------ learned sampler

namespace {

double mlp_theta(int k) { return std::pow(10.0, -2.0 + 3.0 * k / (kMlpTheta - 1)); }
double mlp_beta(int j) { return 0.95 * j / (kMlpBeta - 1); }

pic_status mlp_build_tables(pic_ctx *ctx) {
    if (ctx->mlp_tables) return PIC_OK;
    const int ncombo = kMlpTheta * kMlpBeta;
    std::vector<double> F((size_t)ncombo * (kMjTable + 1)), par(8 * (size_t)ncombo);
    for (int k = 0; k < kMlpTheta; ++k)
        for (int j = 0; j < kMlpBeta; ++j) {
            const int c = k * kMlpBeta + j;
            std::vector<double> f;
            double s0, h, psi, Z;
            const double th = mlp_theta(k), b0 = mlp_beta(j);
            build_marginal_table(th, b0, kMjTable, f, s0, h, psi, Z);
            std::copy(f.begin(), f.end(), F.begin() + (size_t)c * (kMjTable + 1));
            const double pv[8] = {1.0 / th, 1.0 / std::sqrt(1.0 - b0 * b0), psi, Z, s0, h, th, b0};
            std::copy(pv, pv + 8, par.begin() + 8 * c);
        }
    CK(cudaMemcpyAsync(ctx->mlpF, F.data(), sizeof(double) * F.size(), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->mlpPar, par.data(), sizeof(double) * par.size(), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->mlp_tables = true;
    return PIC_OK;
}

// Xavier-uniform initial weights, zero biases (splitmix64 stream of the seed).
void mlp_init_weights(std::vector<float> &w, uint64_t seed) {
    auto next = [&seed]() {
        uint64_t z = (seed += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * 0x1p-53;
    };
    w.assign(kMlpParams, 0.f);
    const int H = 64;
    auto fill = [&](int off, int fan_in, int fan_out) {
        const double a = std::sqrt(6.0 / (fan_in + fan_out));
        for (int q = 0; q < fan_in * fan_out; ++q) w[off + q] = (float)((2.0 * next() - 1.0) * a);
    };
    fill(0, 3, H);
    fill(H * 3 + H, H, H);
    fill(H * 3 + H + H * H + H, H, H);
    fill(H * 3 + H + 2 * (H * H + H), H, 1);
}

pic_status mlp_upload(pic_ctx *ctx, const float *w) {
    CK(cudaMemcpyAsync(ctx->mlpW, w, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(ctx->mlpM, 0, sizeof(float) * kMlpParams, ctx->stream));
    CK(cudaMemsetAsync(ctx->mlpV, 0, sizeof(float) * kMlpParams, ctx->stream));
    CK(cudaMemsetAsync(ctx->mlpG, 0, sizeof(float) * kMlpParams, ctx->stream));
    launch_mlp_to_half(ctx->mlpW, ctx->mlpWh, ctx->stream);
    CK(cudaGetLastError());
    ctx->mlp_step = 0;
    ctx->mlp_init = true;
    return PIC_OK;
}

}  // namespace

pic_status mlp_load(pic_ctx *ctx, int run, int species, long long n, double theta, const double beta[3], int profile,
                    double L, double x0, int colocate_with, uint64_t seed) {
    if (!ctx->mlp_ready) return fail(ctx, PIC_ESTATE, "the sampler network is not trained (pic_mlp_train or pic_mlp_set_weights)");
    Run &r = ctx->runs[run];
    SpeciesState &S = r.sp[species];
    SpeciesState *C = colocate_with >= 0 ? &r.sp[colocate_with] : nullptr;
    const bool mixed = ctx->precision == PIC_MIXED;
    if (mixed && C && C->cur != S.cur) S.cur = C->cur;
    cudaStream_t sm = ctx->stream;
    launch_load_mj_mlp(r.g, r.d.ndim, n, species, seed, profile, L, x0, theta, beta, ctx->mlpWh, C ? 1 : 0, S.s64,
                       C ? C->s64 : S.s64, S.mb[S.cur], C ? C->mb[C->cur] : S.mb[S.cur], mixed ? 1 : 0, ctx->d_err, sm);
    CK(cudaGetLastError());
    S.n = n;
    S.tiled = false;
    S.counted = false;
    r.sorted = false;
    r.since_sort = 0;
    if (mixed) {
        FieldPtrs<float> f = fields_of<float>(r);
        launch_node_fields(r.g, f, r.nfA, r.nfB, sm);
        launch_half_back_mixed(r.g, r.nfA, r.nfB, S.mb[S.cur], n, (float)S.h, (float)r.d.dt, sm);
    } else {
        double *J[3] = {jplane<double>(r, r.jcur, 0), jplane<double>(r, r.jcur, 1), jplane<double>(r, r.jcur, 2)};
        launch_push_fp64(r.g, fields_of<double>(r), J, S.s64, n, S.h, S.alpha, r.d.dt, 1, S.m_over_me, nullptr,
                         ctx->d_err, sm);
    }
    CK(cudaGetLastError());
    r.step = 0;
    r.hist_n = 0;
    CK(cudaMemsetAsync(r.hist, 0, sizeof(double) * 8 * r.hist_cap, sm));
    CK(cudaMemsetAsync(r.hist_idx, 0, sizeof(long long), sm));
    return read_err(ctx);
}

extern "C" {

pic_status pic_mlp_set_weights(pic_ctx *ctx, const float *w) {
    if (!ctx) return PIC_EINVAL;
    if (!w) return fail(ctx, PIC_EINVAL, "null weights");
    for (int q = 0; q < kMlpParams; ++q)
        if (!std::isfinite(w[q])) return fail(ctx, PIC_ENUMERIC, "non-finite weight %d", q);
    pic_status st = mlp_upload(ctx, w);
    if (st) return st;
    ctx->mlp_ready = true;
    CK(cudaStreamSynchronize(ctx->stream));
    return PIC_OK;
}

pic_status pic_mlp_get_weights(pic_ctx *ctx, float *w) {
    if (!ctx) return PIC_EINVAL;
    if (!w) return fail(ctx, PIC_EINVAL, "null output");
    if (!ctx->mlp_init) return fail(ctx, PIC_ESTATE, "no weights yet");
    CK(cudaMemcpyAsync(w, ctx->mlpW, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return PIC_OK;
}

pic_status pic_mlp_gradients(pic_ctx *ctx, const float *x, const float *target, int n, float *grad, double *loss) {
    if (!ctx) return PIC_EINVAL;
    if (n < 1 || n > kMlpBatchMax || !x || !target || !grad) return fail(ctx, PIC_EINVAL, "batch of 1..%d samples", kMlpBatchMax);
    if (!ctx->mlp_init) return fail(ctx, PIC_ESTATE, "no weights yet");
    cudaStream_t sm = ctx->stream;
    for (int c = 0; c < 3; ++c)
        CK(cudaMemcpyAsync(ctx->mlpX + (size_t)c * n, x + (size_t)c * n, sizeof(float) * n, cudaMemcpyHostToDevice, sm));
    CK(cudaMemcpyAsync(ctx->mlpT, target, sizeof(float) * n, cudaMemcpyHostToDevice, sm));
    CK(cudaMemsetAsync(ctx->mlpG, 0, sizeof(float) * kMlpParams, sm));
    CK(cudaMemsetAsync(ctx->mlpLoss, 0, sizeof(double), sm));
    launch_mlp_fwd_bwd(ctx->mlpW, ctx->mlpX, ctx->mlpT, n, ctx->mlpG, ctx->mlpLoss, sm);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(grad, ctx->mlpG, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, sm));
    double l = 0.0;
    CK(cudaMemcpyAsync(&l, ctx->mlpLoss, sizeof(double), cudaMemcpyDeviceToHost, sm));
    CK(cudaMemsetAsync(ctx->mlpG, 0, sizeof(float) * kMlpParams, sm));
    CK(cudaStreamSynchronize(sm));
    if (loss) *loss = l;
    return PIC_OK;
}

pic_status pic_mlp_train(pic_ctx *ctx, int steps, int batch, double lr, uint64_t seed, double *final_loss) {
    if (!ctx) return PIC_EINVAL;
    if (steps < 1 || batch < 32 || batch > kMlpBatchMax || !(lr > 0))
        return fail(ctx, PIC_EINVAL, "steps >= 1, 32 <= batch <= %d, lr > 0", kMlpBatchMax);
    pic_status st = mlp_build_tables(ctx);
    if (st) return st;
    if (!ctx->mlp_init) {
        std::vector<float> w;
        mlp_init_weights(w, seed);
        st = mlp_upload(ctx, w.data());
        if (st) return st;
    }
    cudaStream_t sm = ctx->stream;
    const int ncombo = kMlpTheta * kMlpBeta;
    const int tail = std::max(1, std::min(100, steps / 10));
    CK(cudaMemsetAsync(ctx->mlpLoss, 0, sizeof(double), sm));
    for (int k = 0; k < steps; ++k) {
        launch_mlp_data(ctx->mlpF, ctx->mlpPar, ncombo, seed, (long long)(ctx->mlp_step + k) * batch, batch, ctx->mlpX,
                        ctx->mlpT, sm);
        launch_mlp_fwd_bwd(ctx->mlpW, ctx->mlpX, ctx->mlpT, batch, ctx->mlpG, ctx->mlpLoss, sm);
        // the reported loss sums the last `tail` steps only
        if (k == steps - tail - 1) CK(cudaMemsetAsync(ctx->mlpLoss, 0, sizeof(double), sm));
        // cosine decay of the learning rate
        const double f = 0.5 * (1.0 + std::cos(M_PI * (double)k / steps));
        launch_adam(ctx->mlpW, ctx->mlpG, ctx->mlpM, ctx->mlpV, ctx->mlp_step + k + 1, (float)(lr * (0.02 + 0.98 * f)), sm);
    }
    ctx->mlp_step += steps;
    launch_mlp_to_half(ctx->mlpW, ctx->mlpWh, sm);
    CK(cudaGetLastError());
    double l = 0.0;
    CK(cudaMemcpyAsync(&l, ctx->mlpLoss, sizeof(double), cudaMemcpyDeviceToHost, sm));
    CK(cudaStreamSynchronize(sm));
    if (final_loss) *final_loss = l / tail;
    ctx->mlp_ready = true;
    return PIC_OK;
}

pic_status pic_mlp_infer(pic_ctx *ctx, const float *x, int64_t n, float *out) {
    if (!ctx) return PIC_EINVAL;
    if (n < 0 || (n > 0 && (!x || !out))) return fail(ctx, PIC_EINVAL, "null input or output");
    if (!ctx->mlp_init) return fail(ctx, PIC_ESTATE, "no weights yet");
    cudaStream_t sm = ctx->stream;
    const int64_t chunk = kMlpBatchMax;
    for (int64_t a0 = 0; a0 < n; a0 += chunk) {
        const int m = (int)std::min(chunk, n - a0);
        for (int c = 0; c < 3; ++c)
            CK(cudaMemcpyAsync(ctx->mlpX + (size_t)c * m, x + (size_t)c * n + a0, sizeof(float) * m,
                               cudaMemcpyHostToDevice, sm));
        launch_mlp_infer(ctx->mlpWh, ctx->mlpX, m, ctx->mlpT, sm);
        CK(cudaMemcpyAsync(out + a0, ctx->mlpT, sizeof(float) * m, cudaMemcpyDeviceToHost, sm));
    }
    CK(cudaStreamSynchronize(sm));
    return PIC_OK;
}

pic_status pic_mj_sample_marginal(pic_ctx *ctx, double theta, double beta0, const double *w, int64_t n, double *y,
                                  int method, double *device_ms) {
    if (!ctx) return PIC_EINVAL;
    if (!(theta > 0) || !(beta0 >= 0 && beta0 < 1) || n < 0 || (n > 0 && (!w || !y)))
        return fail(ctx, PIC_EINVAL, "theta > 0, 0 <= beta0 < 1, non-null buffers");
    if (method != PIC_MJ_EXACT && method != PIC_MJ_MLP) return fail(ctx, PIC_EINVAL, "method EXACT or MLP");
    if (method == PIC_MJ_MLP && !ctx->mlp_ready) return fail(ctx, PIC_ESTATE, "the sampler network is not trained");
    std::vector<double> F;
    double s0, h, psi, Z;
    build_marginal_table(theta, beta0, kMjTable, F, s0, h, psi, Z);
    cudaStream_t sm = ctx->stream;
    CK(cudaMemcpyAsync(ctx->mj_table, F.data(), sizeof(double) * (kMjTable + 1), cudaMemcpyHostToDevice, sm));
    const int64_t chunk = (int64_t)(ctx->staging_bytes / (2 * sizeof(double)));
    double *stg = (double *)ctx->staging;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float total = 0.f;
    for (int64_t a0 = 0; a0 < n; a0 += chunk) {
        const int m = (int)std::min(chunk, n - a0);
        CK(cudaMemcpyAsync(stg, w + a0, sizeof(double) * m, cudaMemcpyHostToDevice, sm));
        CK(cudaEventRecord(e0, sm));
        launch_sample_par(ctx->mj_table, s0, h, psi, Z, ctx->mlpWh, method == PIC_MJ_MLP, theta, beta0, stg, m,
                          stg + m, sm);
        CK(cudaEventRecord(e1, sm));
        CK(cudaMemcpyAsync(y + a0, stg + m, sizeof(double) * m, cudaMemcpyDeviceToHost, sm));
        CK(cudaStreamSynchronize(sm));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        total += ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaGetLastError());
    if (device_ms) *device_ms = total;
    return PIC_OK;
}

}  // extern "C"
