/*
 * pic_oracle.c -- plain, slow, FP64 CPU oracle of one particle-in-cell step
 * of Apar-T (Melzani et al., "Apar-T: code, validation, and physical
 * interpretation of particle-in-cell results", arXiv 1308.5892).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file.  It shares no source with
 * the CUDA library and never calls it.
 *
 * Everything is written in the paper's normalised units (App. A.2): lengths
 * in cells X0 = 1, times in X0/c, velocities in c, fields e and b = cB in
 * m_e c^2/(e X0), momenta u = gamma v / c.  Every operation is evaluated one
 * at a time in double precision, in the order the paper states it, with no
 * blocking, fusion or reordering.
 *
 * Grid (App. A.3.2, Fig. Yee): nx*ny*nz cells, arrays indexed (k*ny + j)*nx + i
 * with i fastest.  Staggering of component c at array index (i,j,k):
 *   e_x (i+1/2, j, k)      e_y (i, j+1/2, k)      e_z (i, j, k+1/2)
 *   b_x (i, j+1/2, k+1/2)  b_y (i+1/2, j, k+1/2)  b_z (i+1/2, j+1/2, k)
 * A field block is 3 planes of ncell doubles (x, y, z components).
 * In 2D3V (ndim = 2) nz = 1, z is ignorable, particles carry u_z but no z.
 *
 * Readings of points the paper leaves open (each is listed with its reason in
 * the design notes of the repository):
 *  - Boris rotation: the standard t/s form, the exact solution of the implicit
 *    rotation equation of App. A.3.3 (the printed closed form is garbled).
 *  - Position update: x^{t+dt} = x^t + dt u/gamma (Eq. mover2 prints u^t).
 *  - Deposit (App. A.3.4, Eq. current_dep) is applied per straight segment;
 *    the path x^t -> x^{t+dt} is split at every integer (node) plane it
 *    crosses, segments taken in the order of their crossing parameter, ties
 *    in axis order x, y, z.
 *  - Conductor walls in x sit on the node planes x = 0 and x = nx (App. A.4):
 *    e_y = e_z = b_x = 0 on the wall, staggered values outside the domain
 *    read as zero in the gather, particles are reflected specularly and the
 *    deposit follows the path to the wall and the mirrored remainder.
 *  - Current smoothing (App. A.3.4) acts on the periodic current, i.e. after
 *    the images of a periodic grid have been summed; one call of the paper's
 *    step 10 is one pass.  It is defined here for periodic axes only.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_BC_PERIODIC 0
#define ORC_BC_CONDUCTOR 1

typedef struct {
    int ndim;          /* 2 (2D3V, z ignorable) or 3 */
    int nx, ny, nz;    /* cells; nz = 1 when ndim = 2 */
    double dt;         /* time step in X0/c */
    int bc_x;          /* ORC_BC_PERIODIC or ORC_BC_CONDUCTOR (walls at x = 0, nx) */
    int smooth_passes; /* current smoothing of App. A.3.4 applied this many times (0: off; periodic grids) */
} orc_grid;

typedef struct {
    int64_t n;         /* number of superparticles */
    double *pos;       /* 3*n: planes x, y, z (z unused in 2D) */
    double *u;         /* 3*n: planes u_x, u_y, u_z, u = gamma v / c */
    double q_over_e;   /* q_s / e */
    double m_over_me;  /* m_s / m_e */
    double alpha;      /* current coupling alpha_s = 2 sgn(q_s) / (n_x^2 rho_sp0), Eq. alpha */
} orc_species;

int orc_abi_version(void) { return 5; }

static long wrapi(long i, long n) { long r = i % n; return r < 0 ? r + n : r; }

static long cidx(const orc_grid *g, long i, long j, long k) {
    return (wrapi(k, g->nz) * g->ny + wrapi(j, g->ny)) * g->nx + wrapi(i, g->nx);
}

static long ncell(const orc_grid *g) { return (long)g->nx * g->ny * g->nz; }

/* ---------------------------------------------------------------- fields */

/* Conductor walls (App. A.4): tangential e and normal b vanish on the wall
 * plane i = 0 (which, in the wrapped storage, is also the plane i = nx). */
static void wall_b(const orc_grid *g, double *b) {
    if (g->bc_x != ORC_BC_CONDUCTOR) return;
    long nc = ncell(g);
    for (long k = 0; k < g->nz; ++k)
        for (long j = 0; j < g->ny; ++j) b[0 * nc + cidx(g, 0, j, k)] = 0.0;
}

static void wall_e(const orc_grid *g, double *e) {
    if (g->bc_x != ORC_BC_CONDUCTOR) return;
    long nc = ncell(g);
    for (long k = 0; k < g->nz; ++k)
        for (long j = 0; j < g->ny; ++j) {
            e[1 * nc + cidx(g, 0, j, k)] = 0.0;
            e[2 * nc + cidx(g, 0, j, k)] = 0.0;
        }
}

/* Faraday, Eq. dyn3 discretised on the Yee lattice (App. A.3.2):
 * b <- b - h curl e, with h = dt/2 for the two half advances of the loop. */
void orc_b_advance(const orc_grid *g, const double *e, double *b, double h) {
    long nc = ncell(g);
    const double *ex = e, *ey = e + nc, *ez = e + 2 * nc;
    double *bx = b, *by = b + nc, *bz = b + 2 * nc;
    for (long k = 0; k < g->nz; ++k)
        for (long j = 0; j < g->ny; ++j)
            for (long i = 0; i < g->nx; ++i) {
                long c = cidx(g, i, j, k);
                double curl_x = (ez[cidx(g, i, j + 1, k)] - ez[c]) - (ey[cidx(g, i, j, k + 1)] - ey[c]);
                double curl_y = (ex[cidx(g, i, j, k + 1)] - ex[c]) - (ez[cidx(g, i + 1, j, k)] - ez[c]);
                double curl_z = (ey[cidx(g, i + 1, j, k)] - ey[c]) - (ex[cidx(g, i, j + 1, k)] - ex[c]);
                bx[c] = bx[c] - h * curl_x;
                by[c] = by[c] - h * curl_y;
                bz[c] = bz[c] - h * curl_z;
            }
    wall_b(g, b);
}

/* Ampere without current, Eq. dyn4 with c = 1 (App. A.3.2): e <- e + h curl b. */
void orc_e_advance(const orc_grid *g, double *e, const double *b, double h) {
    long nc = ncell(g);
    double *ex = e, *ey = e + nc, *ez = e + 2 * nc;
    const double *bx = b, *by = b + nc, *bz = b + 2 * nc;
    for (long k = 0; k < g->nz; ++k)
        for (long j = 0; j < g->ny; ++j)
            for (long i = 0; i < g->nx; ++i) {
                long c = cidx(g, i, j, k);
                double curl_x = (bz[c] - bz[cidx(g, i, j - 1, k)]) - (by[c] - by[cidx(g, i, j, k - 1)]);
                double curl_y = (bx[c] - bx[cidx(g, i, j, k - 1)]) - (bz[c] - bz[cidx(g, i - 1, j, k)]);
                double curl_z = (by[c] - by[cidx(g, i - 1, j, k)]) - (bx[c] - bx[cidx(g, i, j - 1, k)]);
                ex[c] = ex[c] + h * curl_x;
                ey[c] = ey[c] + h * curl_y;
                ez[c] = ez[c] + h * curl_z;
            }
    wall_e(g, e);
}

/* Staggered value read by the gather.  With conductor walls, a value whose
 * location lies outside [0, nx] (inside the conductor) or on the wall plane
 * for a tangential e / normal b component reads as zero (App. A.4). */
static double sval(const orc_grid *g, const double *f, int comp_kind, long i, long j, long k) {
    if (g->bc_x == ORC_BC_CONDUCTOR) {
        if (comp_kind == 1) {          /* located at x = i + 1/2 */
            if (i < 0 || i > g->nx - 1) return 0.0;
        } else {                       /* located at x = i (node plane) */
            if (i <= 0 || i >= g->nx) return 0.0;
        }
    }
    return f[cidx(g, i, j, k)];
}

/* Node values (App. A.3.3): e averaged over its 2 edge neighbours, b over its
 * 4 face neighbours, e.g. E_x(i,j,k) = (e_x(i-1,j,k) + e_x(i,j,k))/2 and
 * B_z(i,j,k) = (b_z(i,j,k) + b_z(i-1,j,k) + b_z(i-1,j-1,k) + b_z(i,j-1,k))/4. */
static void node_fields(const orc_grid *g, const double *e, const double *b,
                        long i, long j, long k, double EB[6]) {
    long nc = ncell(g);
    const double *ex = e, *ey = e + nc, *ez = e + 2 * nc;
    const double *bx = b, *by = b + nc, *bz = b + 2 * nc;
    /* kind 1: x-staggered (e_x, b_y, b_z); kind 0: x on nodes (e_y, e_z, b_x) */
    EB[0] = 0.5 * (sval(g, ex, 1, i - 1, j, k) + sval(g, ex, 1, i, j, k));
    EB[1] = 0.5 * (sval(g, ey, 0, i, j - 1, k) + sval(g, ey, 0, i, j, k));
    EB[2] = 0.5 * (sval(g, ez, 0, i, j, k - 1) + sval(g, ez, 0, i, j, k));
    EB[3] = 0.25 * (sval(g, bx, 0, i, j, k) + sval(g, bx, 0, i, j - 1, k) +
                    sval(g, bx, 0, i, j, k - 1) + sval(g, bx, 0, i, j - 1, k - 1));
    EB[4] = 0.25 * (sval(g, by, 1, i, j, k) + sval(g, by, 1, i - 1, j, k) +
                    sval(g, by, 1, i, j, k - 1) + sval(g, by, 1, i - 1, j, k - 1));
    EB[5] = 0.25 * (sval(g, bz, 1, i, j, k) + sval(g, bz, 1, i - 1, j, k) +
                    sval(g, bz, 1, i - 1, j - 1, k) + sval(g, bz, 1, i, j - 1, k));
}

/* Exported for tests: 6 planes (E_x..B_z) of node-averaged fields. */
void orc_node_fields(const orc_grid *g, const double *e, const double *b, double *out) {
    long nc = ncell(g);
    for (long k = 0; k < g->nz; ++k)
        for (long j = 0; j < g->ny; ++j)
            for (long i = 0; i < g->nx; ++i) {
                double EB[6];
                node_fields(g, e, b, i, j, k, EB);
                for (int c = 0; c < 6; ++c) out[c * nc + cidx(g, i, j, k)] = EB[c];
            }
}

/* Cell index and offset along one axis: x = i + delta, i = floor(x). */
static void split_coord(double x, long n, int conductor, long *i, double *d) {
    double f = floor(x);
    long ii = (long)f;
    double dd = x - f;
    if (conductor && ii >= n) { ii = n - 1; dd = 1.0; }   /* particle exactly on the far wall */
    *i = ii;
    *d = dd;
}

/* Trilinear (CIC) gather (App. A.3.3): node (i+eps, j+eta, k+xi) has weight
 * prod over axes of (delta if the offset is 1 else 1 - delta). */
static void gather_one(const orc_grid *g, const double *e, const double *b,
                       double x, double y, double z, double EB[6]) {
    long i, j, k = 0;
    double dx, dy, dz = 0.0;
    split_coord(x, g->nx, g->bc_x == ORC_BC_CONDUCTOR, &i, &dx);
    split_coord(y, g->ny, 0, &j, &dy);
    if (g->ndim == 3) split_coord(z, g->nz, 0, &k, &dz);
    for (int c = 0; c < 6; ++c) EB[c] = 0.0;
    int nzn = (g->ndim == 3) ? 2 : 1;
    for (int xi = 0; xi < nzn; ++xi)
        for (int eta = 0; eta < 2; ++eta)
            for (int eps = 0; eps < 2; ++eps) {
                double w = (eps ? dx : 1.0 - dx) * (eta ? dy : 1.0 - dy);
                if (g->ndim == 3) w *= (xi ? dz : 1.0 - dz);
                double node[6];
                node_fields(g, e, b, i + eps, j + eta, k + xi, node);
                for (int c = 0; c < 6; ++c) EB[c] += w * node[c];
            }
}

void orc_gather(const orc_grid *g, const double *e, const double *b, int64_t n,
                const double *pos, double *out) {
    for (int64_t p = 0; p < n; ++p) {
        double EB[6];
        gather_one(g, e, b, pos[p], pos[n + p], pos[2 * n + p], EB);
        for (int c = 0; c < 6; ++c) out[c * n + p] = EB[c];
    }
}

/* ------------------------------------------------------------- particles */

/* Relativistic Boris step (App. A.3.3, Eq. mover1, Birdsall & Langdon 15.4):
 *   u- = u + h e dt/2,  gamma = sqrt(1 + u-^2),  t = h b dt / (2 gamma),
 *   s = 2 t / (1 + t^2),  u' = u- + u- x t,  u+ = u- + u' x s,
 *   u_new = u+ + h e dt/2,   with h = (q/e)(m_e/m). */
static void boris_one(double u[3], const double EB[6], double h, double dt) {
    double um[3], t[3], s[3], up[3], uprime[3];
    for (int a = 0; a < 3; ++a) um[a] = u[a] + h * EB[a] * dt * 0.5;
    double gam = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    for (int a = 0; a < 3; ++a) t[a] = h * EB[3 + a] * dt / (2.0 * gam);
    double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    for (int a = 0; a < 3; ++a) s[a] = 2.0 * t[a] / (1.0 + t2);
    uprime[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
    uprime[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
    uprime[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
    up[0] = um[0] + (uprime[1] * s[2] - uprime[2] * s[1]);
    up[1] = um[1] + (uprime[2] * s[0] - uprime[0] * s[2]);
    up[2] = um[2] + (uprime[0] * s[1] - uprime[1] * s[0]);
    for (int a = 0; a < 3; ++a) u[a] = up[a] + h * EB[a] * dt * 0.5;
}

/* Exported: u (3*n planes) advanced by one Boris step with given fields EB (6*n planes). */
void orc_boris(int64_t n, double *u, const double *EB, double h, double dt) {
    for (int64_t p = 0; p < n; ++p) {
        double uu[3] = {u[p], u[n + p], u[2 * n + p]};
        double f[6];
        for (int c = 0; c < 6; ++c) f[c] = EB[c * n + p];
        boris_one(uu, f, h, dt);
        u[p] = uu[0]; u[n + p] = uu[1]; u[2 * n + p] = uu[2];
    }
}

/* ---------------------------------------------------------------- deposit */

/* One straight segment inside one cell of the main grid (App. A.1 and A.3.4,
 * Eq. current_dep).  The particle, a cube of volume X0^3, starts at offset
 * delta inside cell (i,j,k) and moves by D.  With d = delta + D/2 and the
 * mid-point weights W^0 = 1 - d, W^1 = d, the part of the volume change of the
 * grid-B cells proportional to D_x is the flux through the x face at
 * (i+1/2, j+eta, k+xi):  F = D_x [W_y^eta W_z^xi + (-1)^(eta+xi) D_y D_z / 12].
 * It enters Ampere's law (Eq. max2bis) as e_x(i, j+eta, k+xi) += -alpha F;
 * y and z follow by cyclic permutation.
 * In 2D3V the cube is uniform along z: the in-plane fluxes are
 * D_x W_y^eta and D_y W_x^eps, and the out-of-plane flux through the cell is
 * D_z [W_x^eps W_y^eta + (-1)^(eps+eta) D_x D_y / 12], D_z = dt u_z / gamma
 * for this segment.  J receives -alpha F. */
static void deposit_segment(const orc_grid *g, double *J, long i, long j, long k,
                            const double delta[3], const double D[3], double alpha) {
    long nc = ncell(g);
    double *Jx = J, *Jy = J + nc, *Jz = J + 2 * nc;
    double W[3][2];
    for (int a = 0; a < 3; ++a) {
        double d = delta[a] + 0.5 * D[a];
        W[a][0] = 1.0 - d;
        W[a][1] = d;
    }
    if (g->ndim == 3) {
        for (int p = 0; p < 2; ++p)
            for (int q = 0; q < 2; ++q) {
                double sgn = ((p + q) & 1) ? -1.0 : 1.0;
                /* x faces: (i+1/2, j+p, k+q) */
                double Fx = D[0] * (W[1][p] * W[2][q] + sgn * D[1] * D[2] / 12.0);
                /* y faces: (i+q, j+1/2, k+p)  -- eta over z (p), eps over x (q) */
                double Fy = D[1] * (W[2][p] * W[0][q] + sgn * D[2] * D[0] / 12.0);
                /* z faces: (i+p, j+q, k+1/2) */
                double Fz = D[2] * (W[0][p] * W[1][q] + sgn * D[0] * D[1] / 12.0);
                Jx[cidx(g, i, j + p, k + q)] += -alpha * Fx;
                Jy[cidx(g, i + q, j, k + p)] += -alpha * Fy;
                Jz[cidx(g, i + p, j + q, k)] += -alpha * Fz;
            }
    } else {
        for (int p = 0; p < 2; ++p) {
            double Fx = D[0] * W[1][p];          /* face (i+1/2, j+p) */
            double Fy = D[1] * W[0][p];          /* face (i+p, j+1/2) */
            Jx[cidx(g, i, j + p, 0)] += -alpha * Fx;
            Jy[cidx(g, i + p, j, 0)] += -alpha * Fy;
            for (int q = 0; q < 2; ++q) {
                double sgn = ((p + q) & 1) ? -1.0 : 1.0;
                double Fz = D[2] * (W[0][p] * W[1][q] + sgn * D[0] * D[1] / 12.0);
                Jz[cidx(g, i + p, j + q, 0)] += -alpha * Fz;   /* node (i+p, j+q) */
            }
        }
    }
}

/* Deposit of the straight path from x0 (unwrapped start) by displacement dx.
 * The path is split at each integer plane it crosses (at most one per axis
 * because |dx_a| < 1); segments are taken in increasing crossing parameter,
 * ties in axis order.  In 2D3V dx[2] is the out-of-plane displacement, shared
 * between segments in proportion to their parameter length. */
static void deposit_path(const orc_grid *g, double *J, const double x0[3],
                         const double dx[3], double alpha) {
    int nd = g->ndim;
    double tc[3] = {2.0, 2.0, 2.0};
    double plane[3] = {0, 0, 0};
    for (int a = 0; a < nd; ++a) {
        double c0 = floor(x0[a]), c1 = floor(x0[a] + dx[a]);
        if (c1 != c0 && dx[a] != 0.0) {
            plane[a] = (c1 > c0) ? c1 : c0;
            tc[a] = (plane[a] - x0[a]) / dx[a];
        }
    }
    /* order crossing axes by t, stable in axis order */
    int order[3] = {0, 1, 2};
    for (int a = 0; a < 3; ++a)
        for (int b2 = 0; b2 < 2 - a; ++b2)
            if (tc[order[b2 + 1]] < tc[order[b2]]) {
                int tmp = order[b2]; order[b2] = order[b2 + 1]; order[b2 + 1] = tmp;
            }
    double p[3] = {x0[0], x0[1], nd == 3 ? x0[2] : 0.0};
    long cell[3];
    for (int a = 0; a < nd; ++a) cell[a] = (long)floor(x0[a]);
    if (nd == 2) cell[2] = 0;
    double tprev = 0.0;
    for (int s = 0; s <= 3; ++s) {
        int ax = (s < 3) ? order[s] : -1;
        double t = 1.0;
        if (ax >= 0) {
            if (ax >= nd || tc[ax] > 1.0) continue;
            t = tc[ax];
        }
        double q[3], D[3], delta[3];
        for (int a = 0; a < nd; ++a) q[a] = x0[a] + dx[a] * t;
        if (ax >= 0) q[ax] = plane[ax];
        for (int a = 0; a < nd; ++a) {
            D[a] = q[a] - p[a];
            delta[a] = p[a] - (double)cell[a];
        }
        if (nd == 2) {
            D[2] = dx[2] * (t - tprev);
            delta[2] = 0.0;
        }
        deposit_segment(g, J, cell[0], cell[1], cell[2], delta, D, alpha);
        for (int a = 0; a < nd; ++a) p[a] = q[a];
        if (ax >= 0) cell[ax] += (dx[ax] > 0.0) ? 1 : -1;
        tprev = t;
        if (ax < 0) break;
    }
}

/* Periodic wrap of a coordinate into [0, n). */
static double wrap_coord(double x, double n) {
    while (x < 0.0) x += n;
    while (x >= n) x -= n;
    return x;
}

/* Move (Eq. mover2 read as x^{t+dt} = x^t + dt u/gamma) with boundary handling
 * and deposit of the path.  u is u^{t+dt/2}; it is flipped on reflection. */
static void move_and_deposit(const orc_grid *g, double *J, double pos[3], double u[3],
                             double alpha, int deposit) {
    double gam = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    double dx[3];
    for (int a = 0; a < 3; ++a) dx[a] = g->dt * u[a] / gam;
    int nd = g->ndim;
    double x0[3] = {pos[0], pos[1], nd == 3 ? pos[2] : 0.0};
    double xn = x0[0] + dx[0];
    if (g->bc_x == ORC_BC_CONDUCTOR && (xn < 0.0 || xn > (double)g->nx)) {
        /* Specular reflection on the wall (App. A.4): path to the wall, then
         * the mirrored remainder, sharing the other components by parameter. */
        double wall = (xn < 0.0) ? 0.0 : (double)g->nx;
        double t = (wall - x0[0]) / dx[0];
        double d1[3] = {wall - x0[0], dx[1] * t, dx[2] * t};
        if (deposit) deposit_path(g, J, x0, d1, alpha);
        double x1[3] = {wall, x0[1] + d1[1], nd == 3 ? x0[2] + d1[2] : 0.0};
        double d2[3] = {-(dx[0] - d1[0]), dx[1] - d1[1], dx[2] - d1[2]};
        /* the mirrored remainder starts on the wall plane moving inwards */
        if (deposit) deposit_path(g, J, x1, d2, alpha);
        pos[0] = wall + d2[0];
        pos[1] = x1[1] + d2[1];
        if (nd == 3) pos[2] = x1[2] + d2[2];
        u[0] = -u[0];
    } else {
        if (deposit) deposit_path(g, J, x0, dx, alpha);
        pos[0] = x0[0] + dx[0];
        pos[1] = x0[1] + dx[1];
        if (nd == 3) pos[2] = x0[2] + dx[2];
    }
    if (g->bc_x == ORC_BC_PERIODIC) pos[0] = wrap_coord(pos[0], g->nx);
    pos[1] = wrap_coord(pos[1], g->ny);
    if (nd == 3) pos[2] = wrap_coord(pos[2], g->nz);
}

/* Exported for tests: deposit n straight paths (pos0 3*n planes, disp 3*n
 * planes) into J (3 planes), no boundary handling beyond periodic indices. */
void orc_deposit(const orc_grid *g, double *J, int64_t n, const double *pos0,
                 const double *disp, double alpha) {
    for (int64_t p = 0; p < n; ++p) {
        double x0[3] = {pos0[p], pos0[n + p], pos0[2 * n + p]};
        double dx[3] = {disp[p], disp[n + p], disp[2 * n + p]};
        deposit_path(g, J, x0, dx, alpha);
    }
}

/* Charge density at the nodes: rho~(node) = sum_p alpha_s W_node(x_p), the
 * CIC weight of App. A.3.3 (the overlap of the particle cube with the grid-B
 * cell of that node).  With conductor walls the nodes x = 0 and x = nx share
 * storage, as for the fields. */
void orc_rho(const orc_grid *g, int64_t n, const double *pos, double alpha, double *rho) {
    for (int64_t p = 0; p < n; ++p) {
        long i, j, k = 0;
        double dx, dy, dz = 0.0;
        split_coord(pos[p], g->nx, g->bc_x == ORC_BC_CONDUCTOR, &i, &dx);
        split_coord(pos[n + p], g->ny, 0, &j, &dy);
        if (g->ndim == 3) split_coord(pos[2 * n + p], g->nz, 0, &k, &dz);
        int nzn = (g->ndim == 3) ? 2 : 1;
        for (int xi = 0; xi < nzn; ++xi)
            for (int eta = 0; eta < 2; ++eta)
                for (int eps = 0; eps < 2; ++eps) {
                    double w = (eps ? dx : 1.0 - dx) * (eta ? dy : 1.0 - dy);
                    if (g->ndim == 3) w *= (xi ? dz : 1.0 - dz);
                    rho[cidx(g, i + eps, j + eta, k + xi)] += alpha * w;
                }
    }
}

/* Discrete divergence of e at the nodes. */
void orc_div_e(const orc_grid *g, const double *e, double *div) {
    long nc = ncell(g);
    const double *ex = e, *ey = e + nc, *ez = e + 2 * nc;
    for (long k = 0; k < g->nz; ++k)
        for (long j = 0; j < g->ny; ++j)
            for (long i = 0; i < g->nx; ++i) {
                long c = cidx(g, i, j, k);
                div[c] = (ex[c] - ex[cidx(g, i - 1, j, k)]) + (ey[c] - ey[cidx(g, i, j - 1, k)]) +
                         (ez[c] - ez[cidx(g, i, j, k - 1)]);
            }
}

/* Current smoothing (App. A.3.4, main-loop step 10), applied `passes` times
 * to each of `nplanes` grid planes.  One pass replaces the value of cell
 * (i,j,k) by the weighted mean of its 3x3x3 neighbourhood: weight 1 for the
 * cell itself, 1/2 for the six cells that differ in one index, 1/4 for the
 * twelve that differ in two and 1/8 for the eight that differ in three, the
 * sum divided by the total weight.  Neighbour indices wrap periodically; in
 * 2D3V (nz = 1) the z neighbours are the cell itself, which is the same
 * smoothing of a z-independent field.  Every pass reads a copy of the
 * previous values, so the result does not depend on the sweep order. */
void orc_smooth(const orc_grid *g, double *a, int nplanes, int passes) {
    long nc = ncell(g);
    double *prev = (double *)malloc(sizeof(double) * nc);
    for (int q = 0; q < nplanes; ++q) {
        double *v = a + q * nc;
        for (int pass = 0; pass < passes; ++pass) {
            memcpy(prev, v, sizeof(double) * nc);
            for (long k = 0; k < g->nz; ++k)
                for (long j = 0; j < g->ny; ++j)
                    for (long i = 0; i < g->nx; ++i) {
                        double sum = 0.0, wsum = 0.0;
                        for (int dk = -1; dk <= 1; ++dk)
                            for (int dj = -1; dj <= 1; ++dj)
                                for (int di = -1; di <= 1; ++di) {
                                    int shifted = (di != 0) + (dj != 0) + (dk != 0);
                                    double w = 1.0;
                                    for (int m = 0; m < shifted; ++m) w *= 0.5;
                                    sum += w * prev[cidx(g, i + di, j + dj, k + dk)];
                                    wsum += w;
                                }
                        v[cidx(g, i, j, k)] = sum / wsum;
                    }
        }
    }
    free(prev);
}

/* ------------------------------------------------------------ main loop */

/* One step of the main loop of App. A.3.1.  State on entry: x^t, u^{t-dt/2},
 * e^t, b^{t-dt/2}; on exit x^{t+dt}, u^{t+dt/2}, e^{t+dt}, b^{t+dt/2}.
 *  1  b half advance with curl e^t           (b at t)
 *  2  u update with e^t, b^t gathered at x^t (u at t+dt/2)
 *  3  x update                                (x at t+dt)
 *  4  b half advance with curl e^t            (b at t+dt/2)
 *  5  boundary for b
 *  6  e full advance with curl b^{t+dt/2}     (e at t+dt, no current yet)
 *  7  boundary for e
 *  8  boundary for particles
 *  9  currents from the displacement x^t -> x^{t+dt}
 * 10  smoothing of the currents, g->smooth_passes times (App. A.3.4)
 * 11  boundary for the currents (periodic indices fold them)
 * 12  e += currents, e boundary again
 * J is caller-provided scratch of 3 planes; on exit it holds what was added to e:
 * the step's -alpha*flux sums, smoothed when smoothing is on. */
/* Steps 2, 3, 8 and 9 for particles p0 <= p < p1 of species S, currents into J. */
static void push_particles(const orc_grid *g, const double *e, const double *b, double *J, const orc_species *S,
                           int64_t p0, int64_t p1) {
    double h = S->q_over_e / S->m_over_me;
    int64_t n = S->n;
    for (int64_t p = p0; p < p1; ++p) {
        double pos[3] = {S->pos[p], S->pos[n + p], S->pos[2 * n + p]};
        double u[3] = {S->u[p], S->u[n + p], S->u[2 * n + p]};
        double EB[6];
        gather_one(g, e, b, pos[0], pos[1], pos[2], EB);       /* 2 */
        boris_one(u, EB, h, g->dt);
        move_and_deposit(g, J, pos, u, S->alpha, 1);           /* 3, 8, 9 */
        S->pos[p] = pos[0]; S->pos[n + p] = pos[1];
        if (g->ndim == 3) S->pos[2 * n + p] = pos[2];
        S->u[p] = u[0]; S->u[n + p] = u[1]; S->u[2 * n + p] = u[2];
    }
}

/* Number of threads the particle loop uses: 1 in the plain build; in the
 * OpenMP build (the all-cores timing of the benchmark only) n > 0 sets it. */
int orc_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

void orc_step(const orc_grid *g, double *e, double *b, double *J, int nsp, const orc_species *sp) {
    long nc = ncell(g);
    memset(J, 0, sizeof(double) * 3 * nc);
    orc_b_advance(g, e, b, 0.5 * g->dt);                          /* 1 */
#ifndef _OPENMP
    for (int s = 0; s < nsp; ++s) push_particles(g, e, b, J, &sp[s], 0, sp[s].n);
#else
    /* OpenMP build: each thread pushes a contiguous share of every species and
     * deposits into its own current grid; the grids are added in thread order.
     * Only the order of the FP64 current sums differs from the plain build. */
    {
        int nt = omp_get_max_threads();
        double *Jt = (double *)calloc((size_t)nt * 3 * nc, sizeof(double));
#pragma omp parallel num_threads(nt)
        {
            int t = omp_get_thread_num(), m = omp_get_num_threads();
            double *Jm = Jt + (size_t)t * 3 * nc;
            for (int s = 0; s < nsp; ++s) {
                int64_t n = sp[s].n;
                push_particles(g, e, b, Jm, &sp[s], n * t / m, n * (t + 1) / m);
            }
        }
        for (int t = 0; t < nt; ++t)
            for (long c = 0; c < 3 * nc; ++c) J[c] += Jt[(size_t)t * 3 * nc + c];
        free(Jt);
    }
#endif
    orc_b_advance(g, e, b, 0.5 * g->dt);                          /* 4, 5 */
    orc_e_advance(g, e, b, g->dt);                                /* 6, 7 */
    if (g->smooth_passes > 0) orc_smooth(g, J, 3, g->smooth_passes);   /* 10 */
    for (long c = 0; c < 3 * nc; ++c) e[c] += J[c];               /* 11, 12 */
    wall_e(g, e);
}

/* Initial staggering (App. A.3.1): momenta are integrated back by -dt/2 with
 * one Boris step of length -dt/2 using e^0 and b^0 at x^0.  (b^{-dt/2} =
 * b^0 + (dt/2) curl e^0 is applied by the caller with orc_b_advance(-dt/2).) */
void orc_stagger_back(const orc_grid *g, const double *e, const double *b, int nsp, const orc_species *sp) {
    for (int s = 0; s < nsp; ++s) {
        const orc_species *S = &sp[s];
        double h = S->q_over_e / S->m_over_me;
        int64_t n = S->n;
        for (int64_t p = 0; p < n; ++p) {
            double EB[6];
            gather_one(g, e, b, S->pos[p], S->pos[n + p], S->pos[2 * n + p], EB);
            double u[3] = {S->u[p], S->u[n + p], S->u[2 * n + p]};
            boris_one(u, EB, h, -0.5 * g->dt);
            S->u[p] = u[0]; S->u[n + p] = u[1]; S->u[2 * n + p] = u[2];
        }
    }
}

/* Multi-step driver for timing and long runs. */
void orc_run(const orc_grid *g, double *e, double *b, double *J, int nsp, const orc_species *sp, int nsteps) {
    for (int n = 0; n < nsteps; ++n) orc_step(g, e, b, J, nsp, sp);
}

/* -------------------------------------------------------- diagnostics */

/* Energies in units of p m_e c^2 per superparticle (App. A.2):
 * kinetic sum (m_s/m_e)(gamma - 1); field |alpha|^-1 sum c^2 / 2 per component.
 * out: [0..nsp) kinetic per species, then 6 field components (e_x..b_z). */
void orc_energies(const orc_grid *g, const double *e, const double *b, int nsp, const orc_species *sp,
                  double inv_alpha_abs, double *out) {
    long nc = ncell(g);
    for (int s = 0; s < nsp; ++s) {
        const orc_species *S = &sp[s];
        double acc = 0.0;
        for (int64_t p = 0; p < S->n; ++p) {
            double ux = S->u[p], uy = S->u[S->n + p], uz = S->u[2 * S->n + p];
            double u2 = ux * ux + uy * uy + uz * uz;
            acc += S->m_over_me * (sqrt(1.0 + u2) - 1.0);
        }
        out[s] = acc;
    }
    for (int c = 0; c < 3; ++c) {
        double ae = 0.0, ab = 0.0;
        for (long q = 0; q < nc; ++q) {
            ae += e[c * nc + q] * e[c * nc + q];
            ab += b[c * nc + q] * b[c * nc + q];
        }
        out[nsp + c] = 0.5 * ae * inv_alpha_abs;
        out[nsp + 3 + c] = 0.5 * ab * inv_alpha_abs;
    }
}

/* Temperature of each species in units of m_e c^2 (Sect. 3.1.3 measures
 * T = m <v^2> / 3; relativistically the mean is that of u . v, u = gamma v, so
 * that a Maxwell-Juttner population of temperature Theta = T / (m_s c^2) gives
 * exactly (m_s/m_e) Theta): out[s] = (m_s/m_e) (1/n) sum |u|^2 / gamma / 3,
 * 0 for an empty species. */
void orc_temperature(int nsp, const orc_species *sp, double *out) {
    for (int s = 0; s < nsp; ++s) {
        const orc_species *S = &sp[s];
        double acc = 0.0;
        for (int64_t p = 0; p < S->n; ++p) {
            double ux = S->u[p], uy = S->u[S->n + p], uz = S->u[2 * S->n + p];
            double u2 = ux * ux + uy * uy + uz * uz;
            double gamma = sqrt(1.0 + u2);
            acc += u2 / gamma;   /* u . v with v = u / gamma */
        }
        out[s] = S->n > 0 ? S->m_over_me * acc / (3.0 * (double)S->n) : 0.0;
    }
}
