/*
 * pic.h -- C ABI of the GB300 particle-in-cell step library (libpic_gb300.so).
 *
 * The library advances the particle-in-cell scheme of Apar-T (Melzani et al.,
 * arXiv 1308.5892, Sect. 2 and App. A) on one NVIDIA GB300 GPU (sm_103a):
 * field gather from the staggered Yee grid, relativistic Boris push and
 * position update, charge-conserving current deposition by volume change,
 * and the FDTD Maxwell update.  All quantities are in the paper's normalised
 * units (App. A.2): cell size X0 = 1, time in X0/c, velocities in c, fields
 * e and b = cB in m_e c^2/(e X0), momenta u = gamma v / c.
 *
 * General conventions
 *  - Every call returns a pic_status; nothing aborts or throws across the ABI.
 *    On failure pic_last_error(ctx) holds a one-line message.
 *  - Invalid arguments give PIC_EINVAL before any device work is queued.
 *  - Host pointers are borrowed for the duration of the call only.
 *  - Device memory belongs to the context.  It is obtained through the
 *    caller's pic_allocator (or cudaMalloc when none is given) inside
 *    pic_init and returned in pic_destroy; no other call allocates device
 *    memory.
 *  - Device work is queued on the stream given in pic_opts (NULL: the legacy
 *    default stream).  Calls that return data to the host synchronise that
 *    stream; pic_step synchronises it unless PIC_FLAG_ASYNC is set.
 *  - A context is used from one host thread at a time.
 */
#ifndef PIC_GB300_H
#define PIC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_MAX_SPECIES 4
#define PIC_ABI_VERSION 2

typedef enum {
    PIC_OK = 0,
    PIC_EINVAL = 1,    /* invalid argument or descriptor */
    PIC_ENOMEM = 2,    /* the allocator returned NULL */
    PIC_ECUDA = 3,     /* a CUDA runtime call failed (message names it) */
    PIC_ETIMEOUT = 4,  /* a bounded device-side wait gave up */
    PIC_ENUMERIC = 5,  /* a non-finite value was found in the state */
    PIC_ESTATE = 6     /* call not valid in the current state, or a particle
                          moved farther than one cell in one step */
} pic_status;

typedef enum { PIC_FP64 = 0, PIC_MIXED = 1 } pic_precision;
typedef enum { PIC_BC_PERIODIC = 0, PIC_BC_CONDUCTOR = 1 } pic_bc;
typedef enum { PIC_PROFILE_UNIFORM = 0, PIC_PROFILE_HARRIS = 1 } pic_profile;
typedef enum { PIC_MJ_EXACT = 0, PIC_MJ_MLP = 1, PIC_MJ_NAIVE_BOOST = 2 } pic_mj_method;

#define PIC_FLAG_ASYNC 1u      /* pic_step returns without synchronising */
#define PIC_FLAG_NO_GRAPH 2u   /* pic_step launches kernels directly instead of replaying a CUDA graph */
#define PIC_FLAG_TIMING 4u     /* record CUDA events around each kernel class (see pic_kernel_time) */
/* Ensembles of PIC_MIXED runs: one batched launch per phase of the step
 * instead of the persistent step walker (see pic_step). */
#define PIC_FLAG_PHASE_LAUNCHES 8u
/* Test hook of the step walker's bounded waits: the push phase of run 0 waits
 * for one item more than exist, so its wait runs out after 20 ms, the launch
 * ends and pic_step reports PIC_ETIMEOUT; the state of that step is undefined.
 * Nothing faults: every wait is bounded and the kernel returns. */
#define PIC_FLAG_INJECT_STALL 16u

/* Kernel classes timed under PIC_FLAG_TIMING. */
typedef enum { PIC_KERNEL_PUSH = 0, PIC_KERNEL_FIELD = 1, PIC_KERNEL_SORT = 2, PIC_KERNEL_SMOOTH = 3 } pic_kernel_class;

/* Device memory provider.  alloc returns a device pointer of at least `bytes`
 * bytes aligned to 256 bytes, or NULL; free receives the same pointer and size. */
typedef struct {
    void *(*alloc)(size_t bytes, void *user);
    void (*free)(void *ptr, size_t bytes, void *user);
    void *user;
} pic_allocator;

/* One superparticle species (Sect. 2.1): charge and mass of the real particle
 * in units of e and m_e; every superparticle has the same weight.  capacity is
 * the maximum number of superparticles the run will hold. */
typedef struct {
    double q_over_e;
    double m_over_me;
    int64_t capacity;
} pic_species_desc;

/* One simulation (Sect. 2.2.1 and App. A.2).
 *  ndim      2 (2D3V: z ignorable, particles carry u_z) or 3
 *  nx,ny,nz  cells per axis (nz = 1 when ndim = 2); 2..2047 each, nx,ny <= 65535 in 2D
 *  n_x       cells per electron skin depth
 *  rho_sp0   reference superparticles per cell, all species together; with
 *            n_x it fixes the current coupling alpha_s = 2 sgn(q_s)/(n_x^2 rho_sp0) (Eq. alpha)
 *  dt        time step in X0/c; must satisfy dt < 1/sqrt(ndim) (Courant, App. B.1)
 *  bc        per axis: PIC_BC_PERIODIC, or PIC_BC_CONDUCTOR for x only (App. A.4)
 *  smooth_passes
 *            current smoothing (App. A.3.4, main-loop step 10) applied this many
 *            times per step, 0..4 (0: off).  One pass replaces the periodic current
 *            of each cell by the mean of its 3x3x3 neighbourhood weighted 1, 1/2,
 *            1/4, 1/8 by the number of shifted indices (the 1-2-1 stencil per
 *            axis).  Periodic axes only: PIC_EINVAL with a conductor. */
typedef struct {
    int ndim;
    int nx, ny, nz;
    double n_x;
    double rho_sp0;
    double dt;
    int bc[3];
    int nspecies;
    pic_species_desc species[PIC_MAX_SPECIES];
    int smooth_passes;
} pic_run_desc;

/* Options of a context.
 *  precision      PIC_FP64: every quantity in double precision, plain
 *                 one-thread-per-particle kernel with global atomics.
 *                 PIC_MIXED: positions as cell index + FP32 offset (on a
 *                 grid of 2^-24 cells), FP32 momenta and fields, currents
 *                 summed exactly in fixed point (each flux rounded once to
 *                 2^-26 of a particle's volume flux, integer sums), e carried
 *                 as a pair of FP32 words (value and rounding remainder)
 *                 updated in FP64 so that its rounding does not accumulate
 *                 in div e, particles kept sorted by tile; FP64 for
 *                 diagnostics.
 *  sort_interval  steps between re-sorts in PIC_MIXED (0: chosen by the autotuner)
 *  tile           tile shape in cells (0: chosen by the autotuner)
 *  stream         cudaStream_t to queue work on (NULL: default stream)
 *  allocator      device memory provider (NULL: cudaMalloc/cudaFree)
 *  flags          PIC_FLAG_* bits */
typedef struct {
    int precision;
    int sort_interval;
    int tile[3];
    void *stream;
    const pic_allocator *allocator;
    uint32_t flags;
} pic_opts;

typedef struct pic_ctx pic_ctx;

/* Host view of one run's state at the start of a step (App. A.3.1):
 * positions x^t, momenta u^{t-dt/2}, e^t, b^{t-dt/2}.
 *  fields        6 * ncell doubles: planes e_x, e_y, e_z, b_x, b_y, b_z, each
 *                ncell = nz*ny*nx values indexed (k*ny + j)*nx + i, with the
 *                Yee staggering e_x (i+1/2,j,k), e_y (i,j+1/2,k), e_z (i,j,k+1/2),
 *                b_x (i,j+1/2,k+1/2), b_y (i+1/2,j,k+1/2), b_z (i+1/2,j+1/2,k)
 *  count[s]      particles of species s (set: number given; get: in = room in
 *                the buffer, out = number returned)
 *  particles[s]  6 * count[s] doubles: planes x, y, z, u_x, u_y, u_z
 *                (z ignored in 2D); pic_get_state returns particles in the
 *                order they were given to pic_set_state or loaded
 *  step          step counter (get only) */
typedef struct {
    double *fields;
    int64_t count[PIC_MAX_SPECIES];
    double *particles[PIC_MAX_SPECIES];
    int64_t step;
} pic_state_view;

/* FP64 diagnostics of one run (Sect. 3.1, App. A.2 units: p m_e c^2 per superparticle).
 *  kinetic[s]      sum over particles of (m_s/m_e)(gamma - 1), gamma from u^{t-dt/2}
 *  field_e[c]      |alpha|^-1 sum over cells of e_c^2 / 2 at t
 *  field_b[c]      |alpha|^-1 sum over cells of b_c^2 / 2 at t - dt/2
 *  sum_u[s][c]     sum over particles of u_c (= sum gamma v_c, the k = 0
 *                  momentum of Eq. Fourier)
 *  temperature[s]  T_s / (m_e c^2) = (m_s/m_e) <u . v> / 3, the relativistic
 *                  form of T = m <v^2> / 3 (Sect. 3.1.3); equals (m_s/m_e) Theta_s
 *                  for a Maxwell-Juttner population of Theta_s = T / (m_s c^2),
 *                  so species in thermal equilibrium report the same value
 *  gauss_max       max over nodes of |div e - S rho~|, rho~ = sum_s alpha_s W (CIC),
 *                  S the run's current smoothing (identity when off): smoothing the
 *                  current conserves div e - S rho~
 *  rho_max         max over species and nodes of |rho~_s|
 *  nonfinite       number of non-finite values met in fields and particles */
typedef struct {
    int64_t step;
    int nspecies;
    int64_t count[PIC_MAX_SPECIES];
    double kinetic[PIC_MAX_SPECIES];
    double field_e[3];
    double field_b[3];
    double sum_u[PIC_MAX_SPECIES][3];
    double temperature[PIC_MAX_SPECIES];
    double gauss_max;
    double rho_max;
    int64_t nonfinite;
} pic_diag;

/* ABI version of the loaded library (PIC_ABI_VERSION at build time). */
int pic_abi_version(void);

/* Create a context holding nruns independent runs (nruns > 1: a batched
 * ensemble advanced together by pic_step).  Validates every descriptor
 * (Courant limit, sizes, species count and capacities, boundary kinds) and
 * returns PIC_EINVAL without touching the device if one is invalid.  Fields
 * start at zero and every species empty.  *out receives the context, or NULL
 * on failure. */
pic_status pic_init(const pic_run_desc *runs, int nruns, const pic_opts *opts, pic_ctx **out);

/* Free all device memory through the allocator and destroy the context. NULL is a no-op. */
void pic_destroy(pic_ctx *ctx);

/* Message of the last failed call on ctx (empty string if none); valid until the next call. */
const char *pic_last_error(const pic_ctx *ctx);

/* Upload a state (see pic_state_view).  Positions must lie in the domain,
 * [0, n) per periodic axis and [0, nx] between conductor walls; counts must
 * not exceed the capacities (PIC_EINVAL before any device work).  Every value
 * is checked on the device while it is converted: a non-finite value gives
 * PIC_ENUMERIC and a position outside the domain PIC_EINVAL, after which the
 * run's state is undefined until the next successful pic_set_state or load.
 * Host buffers are read during the call only.  A buffer that lies inside one
 * page-locked allocation (cudaHostAlloc, cudaHostRegister) is read by the
 * conversion kernels directly over the host link; other buffers are staged
 * through device memory.  Both give the same state. */
pic_status pic_set_state(pic_ctx *ctx, int run, const pic_state_view *in);

/* Download the state into caller buffers (converted to FP64).  A NULL
 * particles[s] skips species s (count[s] still receives its size).  As for
 * pic_set_state, page-locked buffers are written by the kernels directly. */
pic_status pic_get_state(pic_ctx *ctx, int run, pic_state_view *out);

/* Copy chosen particles of one species by id (ids as returned in load/set
 * order, 0 <= id < count): out holds 6 * nids doubles, planes x, y, z, u_x,
 * u_y, u_z, in the order of ids.  Synchronises. */
pic_status pic_get_particles(pic_ctx *ctx, int run, int species, const int64_t *ids, int64_t nids, double *out);

/* Add uniform fields e0 to e and b0 to b of one run (tests; background field). */
pic_status pic_set_uniform_field(pic_ctx *ctx, int run, const double e0[3], const double b0[3]);

/* Load `ppc` superparticles per cell of one species with a drifting
 * Maxwell-Juttner distribution (Sect. 4.3, Eq. Jutt, App. D) of temperature
 * theta = T/(m c^2) and bulk velocity beta (in c; |beta| < 1), replacing the
 * species' particles.  profile: PIC_PROFILE_UNIFORM (uniform density), or
 * PIC_PROFILE_HARRIS with profile_params[0] = L, [1] = x0: comoving density
 * proportional to sech^2((x - x0)/L) along x with ppc the value at x0
 * (App. C).  method: PIC_MJ_EXACT (inverse CDF of the marginal of p along
 * beta, Eq. distr_y, then the conditional of Eq. finding_u), PIC_MJ_MLP (the
 * learned inverse CDF, see pic_mlp_*), PIC_MJ_NAIVE_BOOST (rest-frame
 * sample boosted particle by particle, Sect. 4.2; wrong for relativistic
 * theta and beta, kept as a control).  colocate_with >= 0 copies the
 * positions of that species (pairs on top of each other, rho = 0, Sect. 2.1).
 * The momenta are then integrated back by -dt/2 (App. A.3.1).  seed selects
 * the counter-based random stream (Philox-4x32-10). */
pic_status pic_load_maxwell_juttner(pic_ctx *ctx, int run, int species, double ppc, double theta,
                                    const double beta[3], int profile, const double *profile_params,
                                    int method, int colocate_with, uint64_t seed);

/* Advance every run by nsteps steps of the main loop (App. A.3.1).  Queued
 * on the context stream; unless PIC_FLAG_ASYNC, synchronises and reports a
 * device-side error flag (PIC_ESTATE when a particle moved more than one cell
 * in a step, PIC_ETIMEOUT when a bounded wait gave up).
 * PIC_MIXED without PIC_FLAG_NO_GRAPH or PIC_FLAG_TIMING: once the runs are
 * sorted and a sort is due, one period of 2K steps (K = sort interval) is
 * captured as a CUDA graph (on a stream of the context's own; the capture
 * does not run the steps) and launched on the context stream; later periods
 * replay it while the state it was captured from is unchanged, so results
 * are bitwise those of direct launches.  A failed capture falls back to
 * direct launches.
 * Ensembles (nruns > 1, PIC_MIXED): unless PIC_FLAG_PHASE_LAUNCHES or
 * PIC_FLAG_TIMING, each step is one persistent launch (the step walker: a work
 * queue of (phase, run, item) items with per-run dependencies and bounded
 * waits, covering the re-sorts that are due, the field updates, the push and
 * the current smoothing); the fields and particles are bitwise those of the
 * launches per phase. */
pic_status pic_step(pic_ctx *ctx, int nsteps);

/* Wait for queued work and report the device-side error flag. */
pic_status pic_sync(pic_ctx *ctx);

/* FP64 diagnostics of one run (see pic_diag); synchronises. */
pic_status pic_diagnostics(pic_ctx *ctx, int run, pic_diag *out);

/* Per-step energy history recorded by the step kernels at no extra pass
 * (units of p m_e c^2, App. A.2): for each step n taken since the last
 * pic_set_state or load (at most 65536 steps are recorded, up to max_steps
 * are returned), out[4n + 0] = kinetic energy at t_n (mean of gamma - 1 over
 * u^{t-dt/2} and u^{t+dt/2}, all species), out[4n + 1] = electric energy of
 * e^t, out[4n + 2] = magnetic energy of b^t, out[4n + 3] = their sum.
 * *nout receives the number of steps written.  Synchronises. */
pic_status pic_energy_history(pic_ctx *ctx, int run, double *out, int64_t max_steps, int64_t *nout);

/* Autotuner of the mixed path: advances every run by real steps (at most
 * max_steps) under each candidate (tile shape, sort interval), keeps the one
 * with the highest particle-steps per second, and caches it in the process
 * for contexts of the same shape (a cached choice costs no steps).  The
 * physical result does not depend on the choice: every particle is advanced
 * by the same arithmetic and the current is an exact fixed-point sum.
 * tile, sort_interval (nullable) receive the choice, *steps_taken the number
 * of steps the trials used.  No-op for PIC_FP64. */
pic_status pic_autotune(pic_ctx *ctx, int max_steps, int tile[3], int *sort_interval, int *steps_taken);

/* Replace the PIC_FLAG_* bits of a context, e.g. to time a window with
 * PIC_FLAG_TIMING (which replays no CUDA graph) and another without it.
 * Takes effect at the next call; PIC_EINVAL for unknown bits. */
pic_status pic_set_flags(pic_ctx *ctx, uint32_t flags);

/* Tuning actually used by a context: tile shape, sort interval, halo. */
pic_status pic_get_tuning(const pic_ctx *ctx, int tile[3], int *sort_interval, int *halo);

/* Counters of the last pic_step, for benchmarks: kernel launches queued per
 * step (all runs, averaged over the call) and algorithmic bytes moved per
 * particle-step by the push/deposit kernel (particle state read + written). */
pic_status pic_get_counters(const pic_ctx *ctx, int64_t *launches_per_step, double *bytes_per_particle_step);

/* With PIC_FLAG_TIMING: total device time (ms, CUDA events on the context
 * stream) and number of launches of one kernel class since the last call to
 * pic_kernel_time with reset != 0.  Synchronises. */
pic_status pic_kernel_time(pic_ctx *ctx, int kernel_class, int reset, double *total_ms, int64_t *launches);

/* ---- learned sampler of the loader (method PIC_MJ_MLP) ----
 * A small network p_par = f(theta, beta0, w) replaces the inversion of the
 * cumulative marginal of Eq. distr_y: 3 -> 64 -> 64 -> 64 -> 1, tanh hidden
 * layers, inputs (log10 theta + 0.5)/1.5, 2 beta0/0.95 - 1, probit(w)/3,
 * output o with asinh(p_par) = atanh(beta0) + asinh(sqrt(theta)) o; valid for
 * 0.01 <= theta <= 10 and 0 <= beta0 <= 0.95.  PIC_MLP_PARAMS FP32 parameters
 * in the order W1[64][3] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[64] b4. */
#define PIC_MLP_PARAMS 8641

/* Train the context's network on the GPU: each of `steps` Adam steps (cosine
 * decay from lr) draws `batch` fresh samples (32..8192) from the exact
 * sampler on a 16 x 12 grid of (theta, beta0) and minimises the mean squared
 * error of o.  Starts from Xavier-uniform weights of `seed` unless weights
 * were set.  *final_loss receives the mean loss of the last steps. */
pic_status pic_mlp_train(pic_ctx *ctx, int steps, int batch, double lr, uint64_t seed, double *final_loss);
pic_status pic_mlp_set_weights(pic_ctx *ctx, const float *w);
pic_status pic_mlp_get_weights(pic_ctx *ctx, float *w);
/* One forward and backward pass of the FP32 training kernel on a host batch:
 * x holds 3 planes of n inputs, target n outputs (1 <= n <= 8192); grad
 * receives d(loss)/d(parameters) of loss = mean (o - target)^2. */
pic_status pic_mlp_gradients(pic_ctx *ctx, const float *x, const float *target, int n, float *grad, double *loss);
/* FP16 inference (FP32 accumulation) of n host inputs (3 planes) into out. */
pic_status pic_mlp_infer(pic_ctx *ctx, const float *x, int64_t n, float *out);
/* Drift component p_par of given uniforms w (host, n values) for one
 * (theta, beta0), by method PIC_MJ_EXACT or PIC_MJ_MLP, into y (host);
 * *device_ms receives the kernel time. */
pic_status pic_mj_sample_marginal(pic_ctx *ctx, double theta, double beta0, const double *w, int64_t n, double *y,
                                  int method, double *device_ms);

/* Gauss-law check for callers that must not allocate device memory.
 *
 * The paper has no counterpart of this entry point: it is a library service.
 * It computes, for a caller-owned FP64 state on the current device, the same
 * two numbers as pic_diagnostics: out[0] = max over nodes of |div e - rho~|
 * and out[1] = max over species and nodes of |rho~_s|, rho~_s = alpha_s times
 * the CIC weights of the positions.  It exists for callers that cannot call
 * cudaMalloc (or any allocating routine) where they need the check: a step
 * loop whose memory pool is fixed up front, a host framework that owns the
 * device allocator, or code that must not enter the allocator and its
 * implicit synchronisation.  No context is needed and nothing is allocated:
 * the only scratch is a static device array of 2^20 doubles inside the
 * library, which every GPU that loads the library keeps for the life of the
 * process.
 *  ndim, nx,ny,nz  grid (nz = 1 when ndim = 2); nx*ny*nz at most 1048576,
 *                  larger grids return PIC_EINVAL with a message on stderr
 *  e               device pointer, 3 planes of nz*ny*nx doubles (e_x, e_y,
 *                  e_z), plain layout indexed (k*ny + j)*nx + i, periodic
 *  nspecies        0..PIC_MAX_SPECIES
 *  counts, alpha   host arrays: particles and alpha_s per species
 *  pos             host array of device pointers, each 3*counts[s] doubles
 *                  (planes x, y, z; z ignored in 2D), positions in [0, n)
 *  out             device pointer to 2 doubles, written by the call
 *  stream          cudaStream_t the work is queued on (NULL: default stream)
 * The call is asynchronous on `stream`.  The first call on a device looks up
 * the scratch array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  The address is
 * kept for the life of the process: after cudaDeviceReset the array moves,
 * so do not call this entry point after a reset.  Every call on a
 * device shares the one scratch array and clears it before use: calls whose
 * work overlaps on the GPU (other streams, other host threads) race and must
 * be serialised by the caller.  Returns PIC_EINVAL for invalid arguments and
 * PIC_ECUDA when a CUDA call fails. */
pic_status pic_gauss_residual_static(int ndim, int nx, int ny, int nz, const double *e, int nspecies,
                                     const int64_t *counts, const double *const *pos, const double *alpha,
                                     double *out, void *stream);

/* Measured fused multiply-add throughput of the current device, the ALU
 * denominators of the rooflines (the FP64 path is bound by the FP64 pipe).
 *  kind    PIC_PEAK_FP32_FMA or PIC_PEAK_FP64_FMA
 *  tflops  out: TFLOP/s, 2 flops per FMA, from CUDA events around one launch of
 *          8 blocks of 256 threads per SM, each thread running 8 independent
 *          FMA chains (after one warm-up launch)
 *  ms      out (nullable): duration of the timed launch
 * Needs no context; allocates and frees a few bytes of device memory;
 * synchronous on the legacy default stream (about 20 ms).  Returns PIC_EINVAL
 * for an unknown kind or a null tflops, PIC_ECUDA when a CUDA call fails. */
#define PIC_PEAK_FP32_FMA 0
#define PIC_PEAK_FP64_FMA 1
pic_status pic_alu_peak(int kind, double *tflops, double *ms);

#ifdef __cplusplus
}
#endif
#endif /* PIC_GB300_H */
