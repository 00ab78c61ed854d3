/*
 * FP64 CPU oracle for one time step of the DPRI urban-flow LES.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference for the
 * CUDA library; only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark may load it.  It shares no code, header, table or constant
 * generator with the CUDA path.
 *
 * Plain, slow loops in the order of the paper's LES routines
 * (Sec. 2.1 "LES Code Structure -- Functional"):
 *   bondv1 (boundary conditions), les (Smagorinsky eddy viscosity),
 *   velfg (advection + diffusion "body force", Sec. 2.5 "Pre-computing
 *   Neighboring Points"), les (SGS stress divergence), adam (Adams-Bashforth),
 *   feedbf (building forcing), press (Poisson equation by red-black SOR,
 *   Sec. 2.6 "SOR Algorithm Implementation"), velnw (velocity update).
 * velnw is run last in each call so that every step ends with a projected,
 * divergence-free velocity.
 *
 * Staggered grid, 1-based interior indices like the paper's Fortran:
 *   cells i=1..nx, j=1..ny, k=1..nz; one ghost layer (index 0 and n+1);
 *   u(i,j,k) on the east face of cell i (face 0 = x=0 inflow plane),
 *   v(i,j,k) on the north face of cell j, w(i,j,k) on the top face of cell k;
 *   p, nut, rhs, solid at cell centres.
 * Every array is stored (nz+2) x (ny+2) x (nx+2), i fastest.
 *
 * Where the paper gives no formula (everything except the u-component of
 * velfg and the SOR update) the discretisation is the stated reading, written
 * out in full in the comment of each routine.  Parity of those readings is
 * pinned only by the invariants and closed forms in the test-suite
 * (polynomial exactness, Taylor-Green decay, symmetry, dissipation sign).
 *
 * Threads.  The same source builds twice: sequential, and with -fopenmp for
 * timing the CPU baseline on every host core.  Only loops over k whose
 * iterations write disjoint cells carry a parallel-for (the cells of one SOR
 * colour read only the other colour, so a half-sweep is order-independent);
 * every FP64 sum is formed per k-plane into its own slot and the planes are
 * added in k order afterwards, so both builds give bit-identical results.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define BC_INOUT 0
#define BC_FREESLIP 1
#define BC_WALL 2
#define BC_PERIODIC 3

typedef struct {
    int32_t nx, ny, nz;
    int32_t bc_x, bc_y, bc_z;
    double dx, dy;
    double dt, cs, nu, omega, tol;
    int32_t max_sweeps, check_every, fixed_sweeps;
    int32_t pad_;
    double turb;
    uint64_t seed;
} orc_params;

typedef struct {
    int32_t sweeps, status;
    double rel_residual, rhs_norm, rhs_mean, mass_factor, p_mean, q_in, q_out;
} orc_stats;

typedef struct {
    orc_params P;
    int sx, sy, sz;
    double *dz, *dzs, *inflow;
    unsigned char* solid;
    double *u, *v, *w, *p, *rhs, *nut;
    double *p_twin;           /* second copy of p for the twinned double buffer (on first use) */
    double *us, *vs, *ws;     /* u* (after AB2 + forcing) */
    double *fu, *fv, *fw;     /* F_old: previous tendency (AB2 history) */
    int64_t step;
    orc_stats st;
    /* inflow profile series in time (the LES side of the coupling to a
     * mesoscale model, Sec. 4): n profiles U_m(z_k) at times t_m */
    int nseries;
    double *series_t, *series_p;   /* [n], [n][nz+2] */
    double *plane_a, *plane_b;     /* [nz+2] per-plane partial sums (added in k order) */
} orc_t;

#define IX(o, i, j, k) (((size_t)(k) * (o)->sy + (size_t)(j)) * (o)->sx + (size_t)(i))

/* ------------------------------------------------------------------------ */
/* counter-based normal variates for the turbulent inflow:
 * splitmix64 (Steele, Lea & Flood 2014) as a hash of (seed, counter),
 * then the Box-Muller transform.                                            */
static uint64_t splitmix64_at(uint64_t seed, uint64_t ctr) {
    uint64_t z = seed + (ctr + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double unit_open(uint64_t x) { return ((double)(x >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
static double gauss_at(uint64_t seed, uint64_t c) {
    double u1 = unit_open(splitmix64_at(seed, 2u * c));
    double u2 = unit_open(splitmix64_at(seed, 2u * c + 1u));
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}
/* one normal variate per (step, component, padded j, padded k) */
static double inflow_noise(const orc_t* o, int comp, int j, int k) {
    uint64_t c = ((uint64_t)o->step * 3u + (uint64_t)comp);
    c = (c * (uint64_t)o->sy + (uint64_t)j) * (uint64_t)o->sz + (uint64_t)k;
    return gauss_at(o->P.seed, c);
}

/* ------------------------------------------------------------------------ */
/* geometry helpers                                                          */

static int wrap(int i, int n) { return i < 1 ? i + n : (i > n ? i - n : i); }

static int is_fluid(const orc_t* o, int i, int j, int k) {
    const orc_params* P = &o->P;
    if (P->bc_x == BC_PERIODIC) i = wrap(i, P->nx);
    if (P->bc_y == BC_PERIODIC) j = wrap(j, P->ny);
    if (P->bc_z == BC_PERIODIC) k = wrap(k, P->nz);
    if (i < 1 || i > P->nx || j < 1 || j > P->ny || k < 1 || k > P->nz) return 0;
    return o->solid[IX(o, i, j, k)] == 0;
}

/* A face is "open" when it is an interior face (or a periodic face) whose two
 * neighbouring cells are both fluid.  Face f along an axis sits between
 * cells f and f+1 (f = 0..n).  Domain-boundary faces of a non-periodic axis
 * are never open: p is Neumann there and the face velocity is set by bondv1. */
static int open_x(const orc_t* o, int f, int j, int k) {
    if (o->P.bc_x != BC_PERIODIC && (f <= 0 || f >= o->P.nx)) return 0;
    return is_fluid(o, f, j, k) && is_fluid(o, f + 1, j, k);
}
static int open_y(const orc_t* o, int i, int f, int k) {
    if (o->P.bc_y != BC_PERIODIC && (f <= 0 || f >= o->P.ny)) return 0;
    return is_fluid(o, i, f, k) && is_fluid(o, i, f + 1, k);
}
static int open_z(const orc_t* o, int i, int j, int f) {
    if (o->P.bc_z != BC_PERIODIC && (f <= 0 || f >= o->P.nz)) return 0;
    return is_fluid(o, i, j, f) && is_fluid(o, i, j, f + 1);
}

/* range of faces advanced by the momentum equation along an axis:
 * 1..n-1 for a bounded axis, 1..n for a periodic one (face 0 == face n). */
static int face_hi(int bc, int n) { return bc == BC_PERIODIC ? n : n - 1; }

/* ------------------------------------------------------------------------ */
/* bondv1: boundary conditions (Sec. 2.1; the boundary range idea of Sec. 2.4)
 *
 * Reading (the paper lists "initial wind profile, inflow, outflow" only):
 *  x inflow/outflow: u(0) = U(z_k) (1 + I xi_u); v,w ghosts at i=0 carry
 *    I U(z_k) xi (zero when I = 0); outflow zero gradient u(nx) = u(nx-1),
 *    ghosts u(nx+1) = u(nx), v(nx+1) = v(nx), w(nx+1) = w(nx).
 *  y free-slip: v(0) = v(ny) = 0, v(ny+1) = -v(ny-1); u, w mirror.
 *  z wall: no-slip ground (w(0) = 0, u(0) = -u(1), v(0) = -v(1)),
 *    free-slip lid (w(nz) = 0, w(nz+1) = -w(nz-1), u, v mirror).
 *  periodic: a(0) = a(n), a(n+1) = a(1) for every array.
 * The passes run x, then y over all i, then z over all i and j, so corner
 * ghosts take the composition of the rules in that order.                   */
/* inflow profile at level k for the current step: the fixed profile, or the
 * series interpolated linearly in time t = step * dt between the two
 * bracketing profiles (held constant before the first and after the last) */
static double inflow_at(const orc_t* o, int k) {
    if (o->nseries <= 0) return o->inflow[k];
    const int n = o->nseries, sk = o->P.nz + 2;
    const double t = (double)o->step * o->P.dt;
    if (n == 1 || t <= o->series_t[0]) return o->series_p[k];
    if (t >= o->series_t[n - 1]) return o->series_p[(size_t)(n - 1) * sk + k];
    int m = 0;
    while (m + 1 < n - 1 && o->series_t[m + 1] <= t) ++m;
    const double w = (t - o->series_t[m]) / (o->series_t[m + 1] - o->series_t[m]);
    return (1.0 - w) * o->series_p[(size_t)m * sk + k] + w * o->series_p[(size_t)(m + 1) * sk + k];
}

static void bc_fill(orc_t* o) {
    const orc_params* P = &o->P;
    const int nx = P->nx, ny = P->ny, nz = P->nz;
    double* A[3] = {o->u, o->v, o->w};
    for (int k = 1; k <= nz; ++k)
        for (int j = 1; j <= ny; ++j) {
            if (P->bc_x == BC_PERIODIC) {
                for (int a = 0; a < 3; ++a) {
                    A[a][IX(o, 0, j, k)] = A[a][IX(o, nx, j, k)];
                    A[a][IX(o, nx + 1, j, k)] = A[a][IX(o, 1, j, k)];
                }
            } else {
                double U = inflow_at(o, k);
                double xu = 0.0, xv = 0.0, xw = 0.0;
                if (P->turb != 0.0) {
                    xu = inflow_noise(o, 0, j, k);
                    xv = inflow_noise(o, 1, j, k);
                    xw = inflow_noise(o, 2, j, k);
                }
                o->u[IX(o, 0, j, k)] = U * (1.0 + P->turb * xu);
                o->v[IX(o, 0, j, k)] = P->turb * U * xv;
                o->w[IX(o, 0, j, k)] = P->turb * U * xw;
                o->u[IX(o, nx, j, k)] = o->u[IX(o, nx - 1, j, k)];
                o->u[IX(o, nx + 1, j, k)] = o->u[IX(o, nx, j, k)];
                o->v[IX(o, nx + 1, j, k)] = o->v[IX(o, nx, j, k)];
                o->w[IX(o, nx + 1, j, k)] = o->w[IX(o, nx, j, k)];
            }
        }
    for (int k = 1; k <= nz; ++k)
        for (int i = 0; i <= nx + 1; ++i) {
            if (P->bc_y == BC_PERIODIC) {
                for (int a = 0; a < 3; ++a) {
                    A[a][IX(o, i, 0, k)] = A[a][IX(o, i, ny, k)];
                    A[a][IX(o, i, ny + 1, k)] = A[a][IX(o, i, 1, k)];
                }
            } else {
                o->v[IX(o, i, 0, k)] = 0.0;
                o->v[IX(o, i, ny, k)] = 0.0;
                o->v[IX(o, i, ny + 1, k)] = -o->v[IX(o, i, ny - 1, k)];
                o->u[IX(o, i, 0, k)] = o->u[IX(o, i, 1, k)];
                o->u[IX(o, i, ny + 1, k)] = o->u[IX(o, i, ny, k)];
                o->w[IX(o, i, 0, k)] = o->w[IX(o, i, 1, k)];
                o->w[IX(o, i, ny + 1, k)] = o->w[IX(o, i, ny, k)];
            }
        }
    for (int j = 0; j <= ny + 1; ++j)
        for (int i = 0; i <= nx + 1; ++i) {
            if (P->bc_z == BC_PERIODIC) {
                for (int a = 0; a < 3; ++a) {
                    A[a][IX(o, i, j, 0)] = A[a][IX(o, i, j, nz)];
                    A[a][IX(o, i, j, nz + 1)] = A[a][IX(o, i, j, 1)];
                }
            } else {
                o->w[IX(o, i, j, 0)] = 0.0;
                o->w[IX(o, i, j, nz)] = 0.0;
                o->w[IX(o, i, j, nz + 1)] = -o->w[IX(o, i, j, nz - 1)];
                o->u[IX(o, i, j, 0)] = -o->u[IX(o, i, j, 1)];
                o->u[IX(o, i, j, nz + 1)] = o->u[IX(o, i, j, nz)];
                o->v[IX(o, i, j, 0)] = -o->v[IX(o, i, j, 1)];
                o->v[IX(o, i, j, nz + 1)] = o->v[IX(o, i, j, nz)];
            }
        }
}

/* ghosts of a cell-centred scalar: zero gradient, or periodic wrap */
static void scalar_ghosts(orc_t* o, double* a) {
    const orc_params* P = &o->P;
    const int nx = P->nx, ny = P->ny, nz = P->nz;
    for (int k = 1; k <= nz; ++k)
        for (int j = 1; j <= ny; ++j) {
            int per = P->bc_x == BC_PERIODIC;
            a[IX(o, 0, j, k)] = a[IX(o, per ? nx : 1, j, k)];
            a[IX(o, nx + 1, j, k)] = a[IX(o, per ? 1 : nx, j, k)];
        }
    for (int k = 1; k <= nz; ++k)
        for (int i = 0; i <= nx + 1; ++i) {
            int per = P->bc_y == BC_PERIODIC;
            a[IX(o, i, 0, k)] = a[IX(o, i, per ? ny : 1, k)];
            a[IX(o, i, ny + 1, k)] = a[IX(o, i, per ? 1 : ny, k)];
        }
    for (int j = 0; j <= ny + 1; ++j)
        for (int i = 0; i <= nx + 1; ++i) {
            int per = P->bc_z == BC_PERIODIC;
            a[IX(o, i, j, 0)] = a[IX(o, i, j, per ? nz : 1)];
            a[IX(o, i, j, nz + 1)] = a[IX(o, i, j, per ? 1 : nz)];
        }
}

/* ------------------------------------------------------------------------ */
/* les (part 1): Smagorinsky eddy viscosity (Sec. 2.1, routine les)
 *
 * Reading: nu_t = (Cs Delta)^2 |S| at cell centres, Delta = (dx dy dz_k)^(1/3),
 * |S| = sqrt(2 S_ij S_ij) = sqrt(2 (S11^2+S22^2+S33^2) + 4 (S12^2+S13^2+S23^2)),
 * normal rates at the centre, each shear rate on its cell edges and averaged
 * over the four edges around the centre.  nu_t = 0 in building cells.       */
static double s12_edge(const orc_t* o, int i, int j, int k) {  /* edge (x_i face, y_j face) */
    return 0.5 * ((o->u[IX(o, i, j + 1, k)] - o->u[IX(o, i, j, k)]) / o->P.dy +
                  (o->v[IX(o, i + 1, j, k)] - o->v[IX(o, i, j, k)]) / o->P.dx);
}
static double s13_edge(const orc_t* o, int i, int j, int k) {  /* edge (x_i face, z_k face) */
    return 0.5 * ((o->u[IX(o, i, j, k + 1)] - o->u[IX(o, i, j, k)]) / o->dzs[k] +
                  (o->w[IX(o, i + 1, j, k)] - o->w[IX(o, i, j, k)]) / o->P.dx);
}
static double s23_edge(const orc_t* o, int i, int j, int k) {  /* edge (y_j face, z_k face) */
    return 0.5 * ((o->v[IX(o, i, j, k + 1)] - o->v[IX(o, i, j, k)]) / o->dzs[k] +
                  (o->w[IX(o, i, j + 1, k)] - o->w[IX(o, i, j, k)]) / o->P.dy);
}

static void les_nut(orc_t* o) {
    const orc_params* P = &o->P;
#pragma omp parallel for schedule(static)
    for (int k = 1; k <= P->nz; ++k)
        for (int j = 1; j <= P->ny; ++j)
            for (int i = 1; i <= P->nx; ++i) {
                size_t c = IX(o, i, j, k);
                if (o->solid[c]) { o->nut[c] = 0.0; continue; }
                double s11 = (o->u[c] - o->u[IX(o, i - 1, j, k)]) / P->dx;
                double s22 = (o->v[c] - o->v[IX(o, i, j - 1, k)]) / P->dy;
                double s33 = (o->w[c] - o->w[IX(o, i, j, k - 1)]) / o->dz[k];
                double s12 = 0.25 * (s12_edge(o, i - 1, j - 1, k) + s12_edge(o, i, j - 1, k) +
                                     s12_edge(o, i - 1, j, k) + s12_edge(o, i, j, k));
                double s13 = 0.25 * (s13_edge(o, i - 1, j, k - 1) + s13_edge(o, i, j, k - 1) +
                                     s13_edge(o, i - 1, j, k) + s13_edge(o, i, j, k));
                double s23 = 0.25 * (s23_edge(o, i, j - 1, k - 1) + s23_edge(o, i, j, k - 1) +
                                     s23_edge(o, i, j - 1, k) + s23_edge(o, i, j, k));
                double smag = sqrt(2.0 * (s11 * s11 + s22 * s22 + s33 * s33) +
                                   4.0 * (s12 * s12 + s13 * s13 + s23 * s23));
                double delta = cbrt(P->dx * P->dy * o->dz[k]);
                double l = P->cs * delta;
                o->nut[c] = l * l * smag;
            }
    scalar_ghosts(o, o->nut);
}

/* ------------------------------------------------------------------------ */
/* velfg: advection + molecular diffusion ("body force"), Sec. 2.5.
 *
 * u follows the paper's printed u-component exactly:
 *   cov1 at cell centre c  = 1/2 (u_{c-1}+u_c) (u_c-u_{c-1})/dx,
 *   covx = (dx_{i+1} cov1_i + dx_i cov1_{i+1}) / (dx_i + dx_{i+1}),
 *   cov2 on the (x_i, y_{j+1/2}) edge = vbar (u_{j+1}-u_j)/dy, covy = mean of
 *   the two edges, cov3 likewise with wbar and dzs,
 *   dfu = 2 (diu1_{i+1}-diu1_i)/(dx_i+dx_{i+1}) + (diu2_{j+1/2}-diu2_{j-1/2})/dy
 *         + (diu3_{k+1/2}-diu3_{k-1/2})/dz_k,
 *   f = -(covx+covy+covz) + nu dfu.
 * v is the symmetric analogue.  For w the control volume spans the centres
 * k and k+1 (height dzs_k): centre values are interpolated to the face with
 * dz weights like covx, and the in-plane advecting velocities u, v are
 * interpolated from heights z_k, z_{k+1} to z_w(k) the same way.            */
static double velfg_u(const orc_t* o, int i, int j, int k) {
    const double dx = o->P.dx, dy = o->P.dy;
    const double* u = o->u;
    const double* v = o->v;
    const double* w = o->w;
    double um = u[IX(o, i - 1, j, k)], uc = u[IX(o, i, j, k)], up = u[IX(o, i + 1, j, k)];
    double cov1_i = 0.5 * (um + uc) * (uc - um) / dx;
    double cov1_ip = 0.5 * (uc + up) * (up - uc) / dx;
    double covx = (dx * cov1_i + dx * cov1_ip) / (dx + dx);
    double vn = 0.5 * (v[IX(o, i, j, k)] + v[IX(o, i + 1, j, k)]);
    double vs = 0.5 * (v[IX(o, i, j - 1, k)] + v[IX(o, i + 1, j - 1, k)]);
    double cov2_n = vn * (u[IX(o, i, j + 1, k)] - uc) / dy;
    double cov2_s = vs * (uc - u[IX(o, i, j - 1, k)]) / dy;
    double covy = (cov2_s + cov2_n) / 2.0;
    double wt = 0.5 * (w[IX(o, i, j, k)] + w[IX(o, i + 1, j, k)]);
    double wb = 0.5 * (w[IX(o, i, j, k - 1)] + w[IX(o, i + 1, j, k - 1)]);
    double cov3_t = wt * (u[IX(o, i, j, k + 1)] - uc) / o->dzs[k];
    double cov3_b = wb * (uc - u[IX(o, i, j, k - 1)]) / o->dzs[k - 1];
    double covz = (cov3_b + cov3_t) / 2.0;
    double diu1_i = (uc - um) / dx, diu1_ip = (up - uc) / dx;
    double diu2_n = (u[IX(o, i, j + 1, k)] - uc) / dy, diu2_s = (uc - u[IX(o, i, j - 1, k)]) / dy;
    double diu3_t = (u[IX(o, i, j, k + 1)] - uc) / o->dzs[k];
    double diu3_b = (uc - u[IX(o, i, j, k - 1)]) / o->dzs[k - 1];
    double dfu = 2.0 * (diu1_ip - diu1_i) / (dx + dx) + (diu2_n - diu2_s) / dy +
                 (diu3_t - diu3_b) / o->dz[k];
    return -(covx + covy + covz) + o->P.nu * dfu;
}

static double velfg_v(const orc_t* o, int i, int j, int k) {
    const double dx = o->P.dx, dy = o->P.dy;
    const double* u = o->u;
    const double* v = o->v;
    const double* w = o->w;
    double vm = v[IX(o, i, j - 1, k)], vc = v[IX(o, i, j, k)], vp = v[IX(o, i, j + 1, k)];
    double cov_j = 0.5 * (vm + vc) * (vc - vm) / dy;
    double cov_jp = 0.5 * (vc + vp) * (vp - vc) / dy;
    double covy = (dy * cov_j + dy * cov_jp) / (dy + dy);
    double ue = 0.5 * (u[IX(o, i, j, k)] + u[IX(o, i, j + 1, k)]);
    double uw = 0.5 * (u[IX(o, i - 1, j, k)] + u[IX(o, i - 1, j + 1, k)]);
    double cov_e = ue * (v[IX(o, i + 1, j, k)] - vc) / dx;
    double cov_w = uw * (vc - v[IX(o, i - 1, j, k)]) / dx;
    double covx = (cov_w + cov_e) / 2.0;
    double wt = 0.5 * (w[IX(o, i, j, k)] + w[IX(o, i, j + 1, k)]);
    double wb = 0.5 * (w[IX(o, i, j, k - 1)] + w[IX(o, i, j + 1, k - 1)]);
    double cov_t = wt * (v[IX(o, i, j, k + 1)] - vc) / o->dzs[k];
    double cov_b = wb * (vc - v[IX(o, i, j, k - 1)]) / o->dzs[k - 1];
    double covz = (cov_b + cov_t) / 2.0;
    double dv_e = (v[IX(o, i + 1, j, k)] - vc) / dx, dv_w = (vc - v[IX(o, i - 1, j, k)]) / dx;
    double dv_j = (vc - vm) / dy, dv_jp = (vp - vc) / dy;
    double dv_t = (v[IX(o, i, j, k + 1)] - vc) / o->dzs[k];
    double dv_b = (vc - v[IX(o, i, j, k - 1)]) / o->dzs[k - 1];
    double dfv = (dv_e - dv_w) / dx + 2.0 * (dv_jp - dv_j) / (dy + dy) + (dv_t - dv_b) / o->dz[k];
    return -(covx + covy + covz) + o->P.nu * dfv;
}

static double velfg_w(const orc_t* o, int i, int j, int k) {
    const double dx = o->P.dx, dy = o->P.dy;
    const double* u = o->u;
    const double* v = o->v;
    const double* w = o->w;
    const double dzk = o->dz[k], dzp = o->dz[k + 1];
    double wm = w[IX(o, i, j, k - 1)], wc = w[IX(o, i, j, k)], wp = w[IX(o, i, j, k + 1)];
    double cov_k = 0.5 * (wm + wc) * (wc - wm) / dzk;
    double cov_kp = 0.5 * (wc + wp) * (wp - wc) / dzp;
    double covz = (dzp * cov_k + dzk * cov_kp) / (dzk + dzp);
    double ue = (dzp * u[IX(o, i, j, k)] + dzk * u[IX(o, i, j, k + 1)]) / (dzk + dzp);
    double uw = (dzp * u[IX(o, i - 1, j, k)] + dzk * u[IX(o, i - 1, j, k + 1)]) / (dzk + dzp);
    double cov_e = ue * (w[IX(o, i + 1, j, k)] - wc) / dx;
    double cov_w = uw * (wc - w[IX(o, i - 1, j, k)]) / dx;
    double covx = (cov_w + cov_e) / 2.0;
    double vn = (dzp * v[IX(o, i, j, k)] + dzk * v[IX(o, i, j, k + 1)]) / (dzk + dzp);
    double vs = (dzp * v[IX(o, i, j - 1, k)] + dzk * v[IX(o, i, j - 1, k + 1)]) / (dzk + dzp);
    double cov_n = vn * (w[IX(o, i, j + 1, k)] - wc) / dy;
    double cov_s = vs * (wc - w[IX(o, i, j - 1, k)]) / dy;
    double covy = (cov_s + cov_n) / 2.0;
    double dw_e = (w[IX(o, i + 1, j, k)] - wc) / dx, dw_w = (wc - w[IX(o, i - 1, j, k)]) / dx;
    double dw_n = (w[IX(o, i, j + 1, k)] - wc) / dy, dw_s = (wc - w[IX(o, i, j - 1, k)]) / dy;
    double dw_k = (wc - wm) / dzk, dw_kp = (wp - wc) / dzp;
    double dfw = (dw_e - dw_w) / dx + (dw_n - dw_s) / dy + 2.0 * (dw_kp - dw_k) / (dzk + dzp);
    return -(covx + covy + covz) + o->P.nu * dfw;
}

/* ------------------------------------------------------------------------ */
/* les (part 2): divergence of the SGS stress tau_ij = 2 nu_t S_ij.
 * Reading: normal stresses at centres, shear stresses on the edges where the
 * shear rates live, with nu_t averaged over the four cells around the edge. */
static double nut_avg_xy(const orc_t* o, int i, int j, int k) {  /* z-edge (i,j) */
    return 0.25 * (o->nut[IX(o, i, j, k)] + o->nut[IX(o, i + 1, j, k)] +
                   o->nut[IX(o, i, j + 1, k)] + o->nut[IX(o, i + 1, j + 1, k)]);
}
static double nut_avg_xz(const orc_t* o, int i, int j, int k) {  /* y-edge (i,k) */
    return 0.25 * (o->nut[IX(o, i, j, k)] + o->nut[IX(o, i + 1, j, k)] +
                   o->nut[IX(o, i, j, k + 1)] + o->nut[IX(o, i + 1, j, k + 1)]);
}
static double nut_avg_yz(const orc_t* o, int i, int j, int k) {  /* x-edge (j,k) */
    return 0.25 * (o->nut[IX(o, i, j, k)] + o->nut[IX(o, i, j + 1, k)] +
                   o->nut[IX(o, i, j, k + 1)] + o->nut[IX(o, i, j + 1, k + 1)]);
}

static double sgs_u(const orc_t* o, int i, int j, int k) {
    const double dx = o->P.dx, dy = o->P.dy;
    double t11_i = 2.0 * o->nut[IX(o, i, j, k)] * (o->u[IX(o, i, j, k)] - o->u[IX(o, i - 1, j, k)]) / dx;
    double t11_ip = 2.0 * o->nut[IX(o, i + 1, j, k)] * (o->u[IX(o, i + 1, j, k)] - o->u[IX(o, i, j, k)]) / dx;
    double t12_n = 2.0 * nut_avg_xy(o, i, j, k) * s12_edge(o, i, j, k);
    double t12_s = 2.0 * nut_avg_xy(o, i, j - 1, k) * s12_edge(o, i, j - 1, k);
    double t13_t = 2.0 * nut_avg_xz(o, i, j, k) * s13_edge(o, i, j, k);
    double t13_b = 2.0 * nut_avg_xz(o, i, j, k - 1) * s13_edge(o, i, j, k - 1);
    return (t11_ip - t11_i) / dx + (t12_n - t12_s) / dy + (t13_t - t13_b) / o->dz[k];
}
static double sgs_v(const orc_t* o, int i, int j, int k) {
    const double dx = o->P.dx, dy = o->P.dy;
    double t22_j = 2.0 * o->nut[IX(o, i, j, k)] * (o->v[IX(o, i, j, k)] - o->v[IX(o, i, j - 1, k)]) / dy;
    double t22_jp = 2.0 * o->nut[IX(o, i, j + 1, k)] * (o->v[IX(o, i, j + 1, k)] - o->v[IX(o, i, j, k)]) / dy;
    double t12_e = 2.0 * nut_avg_xy(o, i, j, k) * s12_edge(o, i, j, k);
    double t12_w = 2.0 * nut_avg_xy(o, i - 1, j, k) * s12_edge(o, i - 1, j, k);
    double t23_t = 2.0 * nut_avg_yz(o, i, j, k) * s23_edge(o, i, j, k);
    double t23_b = 2.0 * nut_avg_yz(o, i, j, k - 1) * s23_edge(o, i, j, k - 1);
    return (t12_e - t12_w) / dx + (t22_jp - t22_j) / dy + (t23_t - t23_b) / o->dz[k];
}
static double sgs_w(const orc_t* o, int i, int j, int k) {
    const double dx = o->P.dx, dy = o->P.dy;
    double t33_k = 2.0 * o->nut[IX(o, i, j, k)] * (o->w[IX(o, i, j, k)] - o->w[IX(o, i, j, k - 1)]) / o->dz[k];
    double t33_kp = 2.0 * o->nut[IX(o, i, j, k + 1)] * (o->w[IX(o, i, j, k + 1)] - o->w[IX(o, i, j, k)]) / o->dz[k + 1];
    double t13_e = 2.0 * nut_avg_xz(o, i, j, k) * s13_edge(o, i, j, k);
    double t13_w = 2.0 * nut_avg_xz(o, i - 1, j, k) * s13_edge(o, i - 1, j, k);
    double t23_n = 2.0 * nut_avg_yz(o, i, j, k) * s23_edge(o, i, j, k);
    double t23_s = 2.0 * nut_avg_yz(o, i, j - 1, k) * s23_edge(o, i, j - 1, k);
    return (t13_e - t13_w) / dx + (t23_n - t23_s) / dy + (t33_kp - t33_k) / o->dzs[k];
}

/* ------------------------------------------------------------------------ */
/* velfg + les + adam + feedbf over the faces advanced by the momentum equation.
 *
 * adam (Sec. 2.1/2.3, adam(fgh, fgh_old, ...)): second-order Adams-Bashforth
 * on the raw tendency, Fhat = 3/2 F^n - 1/2 F^{n-1}; the first step is
 * forward Euler.  F_old keeps the raw tendency.
 * feedbf (Sec. 2.1, "building effects"), reading: direct forcing, u* = u +
 * dt Fhat on open faces and u* = 0 on faces touching a building cell.
 * Faces not advanced (inflow, outflow, walls) are copied from u.            */
static void momentum(orc_t* o) {
    const orc_params* P = &o->P;
    const int nx = P->nx, ny = P->ny, nz = P->nz;
    const int first = (o->step == 0);
    size_t n = (size_t)o->sx * o->sy * o->sz;
    memcpy(o->us, o->u, n * sizeof(double));
    memcpy(o->vs, o->v, n * sizeof(double));
    memcpy(o->ws, o->w, n * sizeof(double));
#pragma omp parallel for schedule(static)
    for (int k = 1; k <= nz; ++k)
        for (int j = 1; j <= ny; ++j)
            for (int i = 1; i <= face_hi(P->bc_x, nx); ++i) {
                size_t c = IX(o, i, j, k);
                double F = velfg_u(o, i, j, k) + sgs_u(o, i, j, k);
                double Fh = first ? F : 1.5 * F - 0.5 * o->fu[c];
                o->fu[c] = F;
                o->us[c] = open_x(o, i, j, k) ? o->u[c] + P->dt * Fh : 0.0;
            }
#pragma omp parallel for schedule(static)
    for (int k = 1; k <= nz; ++k)
        for (int j = 1; j <= face_hi(P->bc_y, ny); ++j)
            for (int i = 1; i <= nx; ++i) {
                size_t c = IX(o, i, j, k);
                double F = velfg_v(o, i, j, k) + sgs_v(o, i, j, k);
                double Fh = first ? F : 1.5 * F - 0.5 * o->fv[c];
                o->fv[c] = F;
                o->vs[c] = open_y(o, i, j, k) ? o->v[c] + P->dt * Fh : 0.0;
            }
#pragma omp parallel for schedule(static)
    for (int k = 1; k <= face_hi(P->bc_z, nz); ++k)
        for (int j = 1; j <= ny; ++j)
            for (int i = 1; i <= nx; ++i) {
                size_t c = IX(o, i, j, k);
                double F = velfg_w(o, i, j, k) + sgs_w(o, i, j, k);
                double Fh = first ? F : 1.5 * F - 0.5 * o->fw[c];
                o->fw[c] = F;
                o->ws[c] = open_z(o, i, j, k) ? o->w[c] + P->dt * Fh : 0.0;
            }
}

/* bondv1 (outflow part) on u*: zero-gradient outflow face, then the FP64
 * mass-flux correction u*(nx) *= Q_in/Q_out with Q = sum u dy dz_k over the
 * plane; periodic axes copy face n into face 0.                             */
static void outflow_fix(orc_t* o) {
    const orc_params* P = &o->P;
    const int nx = P->nx, ny = P->ny, nz = P->nz;
    o->st.mass_factor = 1.0;
    o->st.q_in = o->st.q_out = 0.0;
    if (P->bc_x == BC_PERIODIC) {
        for (int k = 1; k <= nz; ++k)
            for (int j = 1; j <= ny; ++j) o->us[IX(o, 0, j, k)] = o->us[IX(o, nx, j, k)];
    } else {
        double qin = 0.0, qout = 0.0;
        for (int k = 1; k <= nz; ++k)
            for (int j = 1; j <= ny; ++j) {
                o->us[IX(o, nx, j, k)] = o->us[IX(o, nx - 1, j, k)];
                qin += o->us[IX(o, 0, j, k)] * P->dy * o->dz[k];
                qout += o->us[IX(o, nx, j, k)] * P->dy * o->dz[k];
            }
        double f = (fabs(qout) > 1e-300) ? qin / qout : 1.0;
        for (int k = 1; k <= nz; ++k)
            for (int j = 1; j <= ny; ++j) o->us[IX(o, nx, j, k)] *= f;
        o->st.mass_factor = f;
        o->st.q_in = qin;
        o->st.q_out = qout * f;
    }
    if (P->bc_y == BC_PERIODIC)
        for (int k = 1; k <= nz; ++k)
            for (int i = 1; i <= nx; ++i) o->vs[IX(o, i, 0, k)] = o->vs[IX(o, i, ny, k)];
    if (P->bc_z == BC_PERIODIC)
        for (int j = 1; j <= ny; ++j)
            for (int i = 1; i <= nx; ++i) o->ws[IX(o, i, j, 0)] = o->ws[IX(o, i, j, nz)];
}

/* ------------------------------------------------------------------------ */
/* press: Poisson equation for the kinematic pressure.
 *
 * Reading of the coefficient arrays of the printed SOR code (Sec. 2.6):
 *   cn2l = cn2s = 1/dx^2, cn3l = cn3s = 1/dy^2,
 *   cn4l_k = 1/(dz_k dzs_k), cn4s_k = 1/(dz_k dzs_{k-1}),
 * each multiplied by the open-face indicator (so building faces and
 * non-periodic domain faces are Neumann), and cn1 = 1 / (sum of the six).
 * rhs = div(u*)/dt on fluid cells with its dz-weighted fluid mean removed
 * (the solvability condition of the pure-Neumann problem).                  */
typedef struct { double e, w, n, s, t, b, cn1; int ie, iw, jn, js, kt, kb; } coef_t;

static int coefs(const orc_t* o, int i, int j, int k, coef_t* c) {
    const orc_params* P = &o->P;
    if (!is_fluid(o, i, j, k)) return 0;
    c->e = open_x(o, i, j, k) / (P->dx * P->dx);
    c->w = open_x(o, i - 1, j, k) / (P->dx * P->dx);
    c->n = open_y(o, i, j, k) / (P->dy * P->dy);
    c->s = open_y(o, i, j - 1, k) / (P->dy * P->dy);
    c->t = open_z(o, i, j, k) / (o->dz[k] * o->dzs[k]);
    c->b = open_z(o, i, j, k - 1) / (o->dz[k] * o->dzs[k - 1]);
    double sum = c->e + c->w + c->n + c->s + c->t + c->b;
    if (sum == 0.0) return 0;
    c->cn1 = 1.0 / sum;
    /* neighbour indices (wrapped on periodic axes; unused when closed) */
    c->ie = P->bc_x == BC_PERIODIC ? wrap(i + 1, P->nx) : i + 1;
    c->iw = P->bc_x == BC_PERIODIC ? wrap(i - 1, P->nx) : i - 1;
    c->jn = P->bc_y == BC_PERIODIC ? wrap(j + 1, P->ny) : j + 1;
    c->js = P->bc_y == BC_PERIODIC ? wrap(j - 1, P->ny) : j - 1;
    c->kt = P->bc_z == BC_PERIODIC ? wrap(k + 1, P->nz) : k + 1;
    c->kb = P->bc_z == BC_PERIODIC ? wrap(k - 1, P->nz) : k - 1;
    return 1;
}

/* sum over neighbours a_nb p_nb, with closed faces contributing nothing */
static double nb_sum(const orc_t* o, const double* p, int i, int j, int k, const coef_t* c) {
    double s = 0.0;
    if (c->e != 0.0) s += c->e * p[IX(o, c->ie, j, k)];
    if (c->w != 0.0) s += c->w * p[IX(o, c->iw, j, k)];
    if (c->n != 0.0) s += c->n * p[IX(o, i, c->jn, k)];
    if (c->s != 0.0) s += c->s * p[IX(o, i, c->js, k)];
    if (c->t != 0.0) s += c->t * p[IX(o, i, j, c->kt)];
    if (c->b != 0.0) s += c->b * p[IX(o, i, j, c->kb)];
    return s;
}

static void make_rhs(orc_t* o) {
    const orc_params* P = &o->P;
#pragma omp parallel for schedule(static)
    for (int k = 1; k <= P->nz; ++k) {
        double num = 0.0, den = 0.0;
        for (int j = 1; j <= P->ny; ++j)
            for (int i = 1; i <= P->nx; ++i) {
                size_t c = IX(o, i, j, k);
                if (!is_fluid(o, i, j, k)) { o->rhs[c] = 0.0; continue; }
                double div = (o->us[c] - o->us[IX(o, i - 1, j, k)]) / P->dx +
                             (o->vs[c] - o->vs[IX(o, i, j - 1, k)]) / P->dy +
                             (o->ws[c] - o->ws[IX(o, i, j, k - 1)]) / o->dz[k];
                o->rhs[c] = div / P->dt;
                num += o->dz[k] * o->rhs[c];
                den += o->dz[k];
            }
        o->plane_a[k] = num;
        o->plane_b[k] = den;
    }
    double num = 0.0, den = 0.0;
    for (int k = 1; k <= P->nz; ++k) {
        num += o->plane_a[k];
        den += o->plane_b[k];
    }
    double mean = den > 0.0 ? num / den : 0.0;
#pragma omp parallel for schedule(static)
    for (int k = 1; k <= P->nz; ++k)
        for (int j = 1; j <= P->ny; ++j)
            for (int i = 1; i <= P->nx; ++i)
                if (is_fluid(o, i, j, k)) o->rhs[IX(o, i, j, k)] -= mean;
    o->st.rhs_mean = mean;
}

/* one half-sweep of the red-black SOR of Sec. 2.6: colour nrd = 0 first
 * (cells with i+j+k odd, from i = 1 + mod(k+j+nrd, 2)), then nrd = 1.       */
static void sor_half(orc_t* o, int nrd) {
    const orc_params* P = &o->P;
#pragma omp parallel for schedule(static)
    for (int k = 1; k <= P->nz; ++k)
        for (int j = 1; j <= P->ny; ++j)
            for (int i = 1 + (k + j + nrd) % 2; i <= P->nx; i += 2) {
                coef_t c;
                if (!coefs(o, i, j, k, &c)) continue;
                size_t ix = IX(o, i, j, k);
                double reltmp = P->omega * (c.cn1 * (nb_sum(o, o->p, i, j, k, &c) - o->rhs[ix]) - o->p[ix]);
                o->p[ix] += reltmp;
            }
}

static void sor_sweep(orc_t* o) {
    sor_half(o, 0);
    sor_half(o, 1);
}

/* "Twinned double buffering" (Sec. 2.6): two copies of p.  For nrd = 0 every
 * unknown of the second copy takes the printed update with its own value and
 * all its neighbours from the first copy; for nrd = 1 the first copy from the
 * second.  Every cell of a half-sweep reads only the other copy (a weighted
 * Jacobi iteration with relaxation omega).                                 */
static void twin_half(orc_t* o, int nrd, double omega) {
    const orc_params* P = &o->P;
    const double* src = nrd == 0 ? o->p : o->p_twin;
    double* dst = nrd == 0 ? o->p_twin : o->p;
#pragma omp parallel for schedule(static)
    for (int k = 1; k <= P->nz; ++k)
        for (int j = 1; j <= P->ny; ++j)
            for (int i = 1; i <= P->nx; ++i) {
                coef_t c;
                if (!coefs(o, i, j, k, &c)) continue;
                size_t ix = IX(o, i, j, k);
                double reltmp = omega * (c.cn1 * (nb_sum(o, src, i, j, k, &c) - o->rhs[ix]) - src[ix]);
                dst[ix] = src[ix] + reltmp;
            }
}

/* (A p)_c = sum_nb a_nb (p_nb - p_c) on fluid cells, 0 elsewhere */
static double apply_A_cell(const orc_t* o, const double* p, int i, int j, int k) {
    coef_t c;
    if (!coefs(o, i, j, k, &c)) return 0.0;
    double diag = c.e + c.w + c.n + c.s + c.t + c.b;
    return nb_sum(o, p, i, j, k, &c) - diag * p[IX(o, i, j, k)];
}

/* relative residual ||rhs - A p||_2 / ||rhs||_2 over the fluid cells (FP64) */
static double residual(orc_t* o) {
    const orc_params* P = &o->P;
#pragma omp parallel for schedule(static)
    for (int k = 1; k <= P->nz; ++k) {
        double rn = 0.0, bn = 0.0;
        for (int j = 1; j <= P->ny; ++j)
            for (int i = 1; i <= P->nx; ++i) {
                coef_t c;
                if (!coefs(o, i, j, k, &c)) continue;
                size_t ix = IX(o, i, j, k);
                double r = o->rhs[ix] - apply_A_cell(o, o->p, i, j, k);
                rn += r * r;
                bn += o->rhs[ix] * o->rhs[ix];
            }
        o->plane_a[k] = rn;
        o->plane_b[k] = bn;
    }
    double rn = 0.0, bn = 0.0;
    for (int k = 1; k <= P->nz; ++k) {
        rn += o->plane_a[k];
        bn += o->plane_b[k];
    }
    o->st.rhs_norm = sqrt(bn);
    if (bn == 0.0) return sqrt(rn);
    return sqrt(rn / bn);
}

static void gauge(orc_t* o) {
    const orc_params* P = &o->P;
#pragma omp parallel for schedule(static)
    for (int k = 1; k <= P->nz; ++k) {
        double num = 0.0, den = 0.0;
        for (int j = 1; j <= P->ny; ++j)
            for (int i = 1; i <= P->nx; ++i)
                if (is_fluid(o, i, j, k)) {
                    num += o->dz[k] * o->p[IX(o, i, j, k)];
                    den += o->dz[k];
                }
        o->plane_a[k] = num;
        o->plane_b[k] = den;
    }
    double num = 0.0, den = 0.0;
    for (int k = 1; k <= P->nz; ++k) {
        num += o->plane_a[k];
        den += o->plane_b[k];
    }
    double m = den > 0.0 ? num / den : 0.0;
#pragma omp parallel for schedule(static)
    for (int k = 1; k <= P->nz; ++k)
        for (int j = 1; j <= P->ny; ++j)
            for (int i = 1; i <= P->nx; ++i)
                if (is_fluid(o, i, j, k)) o->p[IX(o, i, j, k)] -= m;
    o->st.p_mean = m;
}

/* SOR iterations with the stop rule: exactly max_sweeps sweeps when
 * fixed_sweeps is set; otherwise stop at the first check (every check_every
 * sweeps, and at max_sweeps) whose FP64 relative residual is <= tol.        */
static void sor_solve(orc_t* o) {
    const orc_params* P = &o->P;
    int s = 0;
    double rel = 0.0;
    if (P->fixed_sweeps) {
        for (s = 1; s <= P->max_sweeps; ++s) sor_sweep(o);
        s = P->max_sweeps;
        rel = residual(o);
    } else {
        for (s = 1; s <= P->max_sweeps; ++s) {
            sor_sweep(o);
            if (s % P->check_every == 0 || s == P->max_sweeps) {
                rel = residual(o);
                if (rel <= P->tol) break;
            }
        }
        if (s > P->max_sweeps) s = P->max_sweeps;
    }
    o->st.sweeps = s;
    o->st.rel_residual = rel;
    o->st.status = (!P->fixed_sweeps && !(rel <= P->tol)) ? 1 : 0;
    gauge(o);
}

/* ------------------------------------------------------------------------ */
/* velnw: u^{n+1} = u* - dt grad p on open advanced faces (0 on closed
 * faces); boundary faces keep u*.  Periodic axes copy face n into face 0.   */
static void project(orc_t* o) {
    const orc_params* P = &o->P;
    const int nx = P->nx, ny = P->ny, nz = P->nz;
    size_t n = (size_t)o->sx * o->sy * o->sz;
    memcpy(o->u, o->us, n * sizeof(double));
    memcpy(o->v, o->vs, n * sizeof(double));
    memcpy(o->w, o->ws, n * sizeof(double));
#pragma omp parallel for schedule(static)
    for (int k = 1; k <= nz; ++k)
        for (int j = 1; j <= ny; ++j)
            for (int i = 1; i <= face_hi(P->bc_x, nx); ++i) {
                size_t c = IX(o, i, j, k);
                int ie = P->bc_x == BC_PERIODIC ? wrap(i + 1, nx) : i + 1;
                o->u[c] = open_x(o, i, j, k)
                              ? o->us[c] - P->dt * (o->p[IX(o, ie, j, k)] - o->p[c]) / P->dx
                              : 0.0;
            }
#pragma omp parallel for schedule(static)
    for (int k = 1; k <= nz; ++k)
        for (int j = 1; j <= face_hi(P->bc_y, ny); ++j)
            for (int i = 1; i <= nx; ++i) {
                size_t c = IX(o, i, j, k);
                int jn = P->bc_y == BC_PERIODIC ? wrap(j + 1, ny) : j + 1;
                o->v[c] = open_y(o, i, j, k)
                              ? o->vs[c] - P->dt * (o->p[IX(o, i, jn, k)] - o->p[c]) / P->dy
                              : 0.0;
            }
#pragma omp parallel for schedule(static)
    for (int k = 1; k <= face_hi(P->bc_z, nz); ++k)
        for (int j = 1; j <= ny; ++j)
            for (int i = 1; i <= nx; ++i) {
                size_t c = IX(o, i, j, k);
                int kt = P->bc_z == BC_PERIODIC ? wrap(k + 1, nz) : k + 1;
                o->w[c] = open_z(o, i, j, k)
                              ? o->ws[c] - P->dt * (o->p[IX(o, i, j, kt)] - o->p[c]) / o->dzs[k]
                              : 0.0;
            }
    if (P->bc_x == BC_PERIODIC)
        for (int k = 1; k <= nz; ++k)
            for (int j = 1; j <= ny; ++j) o->u[IX(o, 0, j, k)] = o->u[IX(o, nx, j, k)];
    if (P->bc_y == BC_PERIODIC)
        for (int k = 1; k <= nz; ++k)
            for (int i = 1; i <= nx; ++i) o->v[IX(o, i, 0, k)] = o->v[IX(o, i, ny, k)];
    if (P->bc_z == BC_PERIODIC)
        for (int j = 1; j <= ny; ++j)
            for (int i = 1; i <= nx; ++i) o->w[IX(o, i, j, 0)] = o->w[IX(o, i, j, nz)];
}

/* ======================================================================== */
/* exported entry points (ctypes)                                            */

orc_t* orc_create(const orc_params* P, const double* dz, const unsigned char* solid,
                  const double* inflow) {
    if (P->nx < 2 || P->ny < 2 || P->nz < 2) return NULL;
    orc_t* o = (orc_t*)calloc(1, sizeof(orc_t));
    o->P = *P;
    o->sx = P->nx + 2;
    o->sy = P->ny + 2;
    o->sz = P->nz + 2;
    size_t n = (size_t)o->sx * o->sy * o->sz;
    o->dz = (double*)calloc(o->sz, sizeof(double));
    o->dzs = (double*)calloc(o->sz, sizeof(double));
    o->inflow = (double*)calloc(o->sz, sizeof(double));
    o->plane_a = (double*)calloc(o->sz, sizeof(double));
    o->plane_b = (double*)calloc(o->sz, sizeof(double));
    for (int k = 1; k <= P->nz; ++k) {
        o->dz[k] = dz[k - 1];
        o->inflow[k] = inflow[k - 1];
    }
    if (P->bc_z == BC_PERIODIC) {
        o->dz[0] = o->dz[P->nz];
        o->dz[P->nz + 1] = o->dz[1];
    } else {
        o->dz[0] = o->dz[1];
        o->dz[P->nz + 1] = o->dz[P->nz];
    }
    for (int k = 0; k <= P->nz; ++k) o->dzs[k] = 0.5 * (o->dz[k] + o->dz[k + 1]);
    o->dzs[P->nz + 1] = o->dz[P->nz + 1];
    o->solid = (unsigned char*)calloc(n, 1);
    for (int k = 1; k <= P->nz; ++k)
        for (int j = 1; j <= P->ny; ++j)
            for (int i = 1; i <= P->nx; ++i)
                o->solid[IX(o, i, j, k)] =
                    solid[((size_t)(k - 1) * P->ny + (j - 1)) * P->nx + (i - 1)] ? 1 : 0;
    double** arrs[] = {&o->u, &o->v, &o->w, &o->p, &o->rhs, &o->nut, &o->us,
                       &o->vs, &o->ws, &o->fu, &o->fv, &o->fw};
    for (size_t a = 0; a < sizeof(arrs) / sizeof(arrs[0]); ++a)
        *arrs[a] = (double*)calloc(n, sizeof(double));
    return o;
}

void orc_destroy(orc_t* o) {
    if (!o) return;
    double* arrs[] = {o->u, o->v, o->w, o->p, o->rhs, o->nut, o->us, o->vs, o->ws,
                      o->fu, o->fv, o->fw, o->dz, o->dzs, o->inflow, o->p_twin,
                      o->plane_a, o->plane_b};
    for (size_t a = 0; a < sizeof(arrs) / sizeof(arrs[0]); ++a) free(arrs[a]);
    free(o->series_t);
    free(o->series_p);
    free(o->solid);
    free(o);
}

/* n profiles [n][nz] at increasing times [n]; n = 0 returns to the fixed profile */
int orc_set_inflow_series(orc_t* o, int n, const double* times, const double* profiles) {
    if (n < 0) return -1;
    for (int m = 1; m < n; ++m)
        if (!(times[m] > times[m - 1])) return -1;
    free(o->series_t);
    free(o->series_p);
    o->series_t = NULL;
    o->series_p = NULL;
    o->nseries = 0;
    if (n == 0) return 0;
    const int sk = o->P.nz + 2;
    o->series_t = (double*)calloc((size_t)n, sizeof(double));
    o->series_p = (double*)calloc((size_t)n * sk, sizeof(double));
    for (int m = 0; m < n; ++m) {
        o->series_t[m] = times[m];
        for (int k = 1; k <= o->P.nz; ++k) o->series_p[(size_t)m * sk + k] = profiles[(size_t)m * o->P.nz + k - 1];
    }
    o->nseries = n;
    return 0;
}

/* the inflow profile the next step will use (for pinning the interpolation) */
void orc_inflow_profile(const orc_t* o, double* out) {
    for (int k = 1; k <= o->P.nz; ++k) out[k - 1] = inflow_at(o, k);
}

/* I/O layout: u (nz, ny, nx+1) faces i=0..nx; v (nz, ny+1, nx) faces j=0..ny;
 * w (nz+1, ny, nx) faces k=0..nz; cell arrays (nz, ny, nx).                  */
enum { A_U = 0, A_V, A_W, A_P, A_RHS, A_NUT, A_US, A_VS, A_WS, A_FU, A_FV, A_FW };

static double* arr(orc_t* o, int which) {
    switch (which) {
        case A_U: return o->u;
        case A_V: return o->v;
        case A_W: return o->w;
        case A_P: return o->p;
        case A_RHS: return o->rhs;
        case A_NUT: return o->nut;
        case A_US: return o->us;
        case A_VS: return o->vs;
        case A_WS: return o->ws;
        case A_FU: return o->fu;
        case A_FV: return o->fv;
        case A_FW: return o->fw;
    }
    return NULL;
}
/* staggering of an array: 0 = cell, 1 = x face, 2 = y face, 3 = z face */
static int stag(int which) {
    switch (which) {
        case A_U: case A_US: case A_FU: return 1;
        case A_V: case A_VS: case A_FV: return 2;
        case A_W: case A_WS: case A_FW: return 3;
    }
    return 0;
}

static void io_dims(const orc_t* o, int which, int* i0, int* j0, int* k0, int* ni, int* nj, int* nk) {
    int s = stag(which);
    *ni = o->P.nx + (s == 1);
    *nj = o->P.ny + (s == 2);
    *nk = o->P.nz + (s == 3);
    *i0 = (s == 1) ? 0 : 1;
    *j0 = (s == 2) ? 0 : 1;
    *k0 = (s == 3) ? 0 : 1;
}

int orc_get(orc_t* o, int which, double* out) {
    double* a = arr(o, which);
    if (!a) return -1;
    int i0, j0, k0, ni, nj, nk;
    io_dims(o, which, &i0, &j0, &k0, &ni, &nj, &nk);
    size_t q = 0;
    for (int k = 0; k < nk; ++k)
        for (int j = 0; j < nj; ++j)
            for (int i = 0; i < ni; ++i) out[q++] = a[IX(o, i0 + i, j0 + j, k0 + k)];
    return 0;
}

int orc_set(orc_t* o, int which, const double* in) {
    double* a = arr(o, which);
    if (!a) return -1;
    int i0, j0, k0, ni, nj, nk;
    io_dims(o, which, &i0, &j0, &k0, &ni, &nj, &nk);
    size_t q = 0;
    for (int k = 0; k < nk; ++k)
        for (int j = 0; j < nj; ++j)
            for (int i = 0; i < ni; ++i) a[IX(o, i0 + i, j0 + j, k0 + k)] = in[q++];
    return 0;
}

/* raw padded array (nz+2, ny+2, nx+2) for operator tests that set ghosts */
double* orc_raw(orc_t* o, int which) { return arr(o, which); }
void orc_dims(const orc_t* o, int32_t* d) { d[0] = o->sx; d[1] = o->sy; d[2] = o->sz; }
void orc_stats_get(const orc_t* o, orc_stats* s) { *s = o->st; }
int64_t orc_step_index(const orc_t* o) { return o->step; }
void orc_set_step_index(orc_t* o, int64_t s) { o->step = s; }

/* phases, exposed one by one for the operator tests */
void orc_bc_fill(orc_t* o) { bc_fill(o); }
void orc_les_nut(orc_t* o) { les_nut(o); }
void orc_momentum(orc_t* o) { momentum(o); }
void orc_outflow_fix(orc_t* o) { outflow_fix(o); }
void orc_make_rhs(orc_t* o) { make_rhs(o); }
void orc_sor_half(orc_t* o, int nrd) { sor_half(o, nrd); }
void orc_sor_sweeps(orc_t* o, int n) { for (int s = 0; s < n; ++s) sor_sweep(o); }
/* n twinned sweeps (nrd = 0 then 1) starting with both copies equal to p */
int orc_twin_sweeps(orc_t* o, int n, double omega) {
    const size_t cells = (size_t)o->sx * o->sy * o->sz;
    if (!o->p_twin && !(o->p_twin = (double*)malloc(cells * sizeof(double)))) return -1;
    memcpy(o->p_twin, o->p, cells * sizeof(double));
    for (int s = 0; s < n; ++s) {
        twin_half(o, 0, omega);
        twin_half(o, 1, omega);
    }
    return 0;
}
double orc_residual(orc_t* o) { return residual(o); }
void orc_sor_solve(orc_t* o) { sor_solve(o); }
void orc_gauge(orc_t* o) { gauge(o); }
void orc_project(orc_t* o) { project(o); }

/* tendency only (velfg + les part 2, no AB2, no forcing) into the F arrays,
 * over the advanced faces; used by the operator tests                       */
void orc_tendency(orc_t* o, int with_sgs) {
    const orc_params* P = &o->P;
    for (int k = 1; k <= P->nz; ++k)
        for (int j = 1; j <= P->ny; ++j)
            for (int i = 1; i <= face_hi(P->bc_x, P->nx); ++i)
                o->fu[IX(o, i, j, k)] = velfg_u(o, i, j, k) + (with_sgs ? sgs_u(o, i, j, k) : 0.0);
    for (int k = 1; k <= P->nz; ++k)
        for (int j = 1; j <= face_hi(P->bc_y, P->ny); ++j)
            for (int i = 1; i <= P->nx; ++i)
                o->fv[IX(o, i, j, k)] = velfg_v(o, i, j, k) + (with_sgs ? sgs_v(o, i, j, k) : 0.0);
    for (int k = 1; k <= face_hi(P->bc_z, P->nz); ++k)
        for (int j = 1; j <= P->ny; ++j)
            for (int i = 1; i <= P->nx; ++i)
                o->fw[IX(o, i, j, k)] = velfg_w(o, i, j, k) + (with_sgs ? sgs_w(o, i, j, k) : 0.0);
}

/* out = A p for a cell array p in I/O layout (nz, ny, nx) */
void orc_apply_A(orc_t* o, const double* p_io, double* out_io) {
    const orc_params* P = &o->P;
    size_t n = (size_t)o->sx * o->sy * o->sz;
    double* tmp = (double*)calloc(n, sizeof(double));
    size_t q = 0;
    for (int k = 1; k <= P->nz; ++k)
        for (int j = 1; j <= P->ny; ++j)
            for (int i = 1; i <= P->nx; ++i) tmp[IX(o, i, j, k)] = p_io[q++];
    q = 0;
    for (int k = 1; k <= P->nz; ++k)
        for (int j = 1; j <= P->ny; ++j)
            for (int i = 1; i <= P->nx; ++i) out_io[q++] = apply_A_cell(o, tmp, i, j, k);
    free(tmp);
}

/* divergence of the current (u, v, w) at cell centres, I/O layout */
void orc_divergence(orc_t* o, double* out_io) {
    const orc_params* P = &o->P;
    size_t q = 0;
    for (int k = 1; k <= P->nz; ++k)
        for (int j = 1; j <= P->ny; ++j)
            for (int i = 1; i <= P->nx; ++i) {
                size_t c = IX(o, i, j, k);
                out_io[q++] = is_fluid(o, i, j, k)
                                  ? (o->u[c] - o->u[IX(o, i - 1, j, k)]) / P->dx +
                                        (o->v[c] - o->v[IX(o, i, j - 1, k)]) / P->dy +
                                        (o->w[c] - o->w[IX(o, i, j, k - 1)]) / o->dz[k]
                                  : 0.0;
            }
}

/* Poisson solve for a given rhs (I/O layout; NULL keeps the current rhs):
 * remove the dz-weighted fluid mean, iterate SOR from the current p, gauge. */
void orc_pressure_solve(orc_t* o, const double* rhs_io) {
    const orc_params* P = &o->P;
    if (rhs_io) {
        double num = 0.0, den = 0.0;
        size_t q = 0;
        for (int k = 1; k <= P->nz; ++k)
            for (int j = 1; j <= P->ny; ++j)
                for (int i = 1; i <= P->nx; ++i) {
                    size_t c = IX(o, i, j, k);
                    double r = rhs_io[q++];
                    if (!is_fluid(o, i, j, k)) { o->rhs[c] = 0.0; continue; }
                    o->rhs[c] = r;
                    num += o->dz[k] * r;
                    den += o->dz[k];
                }
        double mean = den > 0.0 ? num / den : 0.0;
        for (int k = 1; k <= P->nz; ++k)
            for (int j = 1; j <= P->ny; ++j)
                for (int i = 1; i <= P->nx; ++i)
                    if (is_fluid(o, i, j, k)) o->rhs[IX(o, i, j, k)] -= mean;
        o->st.rhs_mean = mean;
    }
    sor_solve(o);
}

/* one full time step: bondv1, les, velfg, les, adam, feedbf, bondv1 (outflow),
 * press, velnw                                                               */
void orc_step(orc_t* o, int nsteps) {
    for (int s = 0; s < nsteps; ++s) {
        bc_fill(o);
        les_nut(o);
        momentum(o);
        outflow_fix(o);
        make_rhs(o);
        sor_solve(o);
        project(o);
        o->step += 1;
    }
}

/* threads of the OpenMP build (the sequential build always reports 1) */
int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* raw inflow noise, for pinning the generator to its published definition */
double orc_gauss(uint64_t seed, uint64_t ctr) { return gauss_at(seed, ctr); }
uint64_t orc_splitmix64(uint64_t seed, uint64_t ctr) { return splitmix64_at(seed, ctr); }
