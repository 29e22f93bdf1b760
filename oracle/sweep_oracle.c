/*
 * sweep_oracle.c -- CPU reference for the two-dimensional swept rule
 * (Walker & Niemeyer, "The Two-Dimensional Swept Rule Applied on
 * Heterogeneous Architectures").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, fp64 reference
 * that the CUDA path is checked against.  Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark may load it; the product path never
 * does.  It shares no code, header, table or constant with the CUDA library.
 *
 * What it computes (each function cites the passage it follows):
 *   - heat diffusion, App. A: 5-point Laplacian, periodic unit square, with
 *     the explicit midpoint (RK2) rule or the forward-Euler rule of App. A;
 *   - compressible Euler, App. B: conservative form Q_t + F_x + G_y = 0,
 *     ideal-gas EOS, pressure-ratio minmod reconstruction, Rusanov-form flux
 *     (the flux formula of App. B), RK2 midpoint in time;
 *   - a replay of the swept phase schedule of Sec. 3.3 (Up-Pyramid, X/Y
 *     Bridges, Octahedron, Down-Pyramid) that computes every (cell, level)
 *     one at a time and checks that every value it reads was produced by an
 *     earlier phase or by the same shape, and that every value is produced
 *     exactly once.
 *
 * Rounding order is pinned (the paper states none): every a*b+c that is
 * meant to be fused is an explicit fma(); everything else must stay unfused,
 * so this file is compiled with -ffp-contract=off.  Division and sqrt are
 * the IEEE-rounded C operators.
 *
 * Readings where the paper is silent or garbled are listed beside the code
 * that takes them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ENOMEM 2
#define ORACLE_EDEP 3   /* replay: a read of a value that was not available */
#define ORACLE_EDUP 4   /* replay: a value computed twice                    */
#define ORACLE_EGAP 5   /* replay: a value never computed                    */

static inline int64_t wrapi(int64_t i, int64_t n)
{
    int64_t r = i % n;
    return r < 0 ? r + n : r;
}

/* ======================================================================
 * Heat diffusion -- App. A.
 * Update of App. A with r_x = r_y = r = alpha*dt/dx^2 (dx = dy):
 *   T' = T + r[(T_{i+1} - 2T + T_{i-1}) + (T_{j+1} - 2T + T_{j-1})]
 * Pinned order (reading: the sum of the four neighbours first, then the
 * centre term, then the scaled increment):
 *   s = (T_{i-1} + T_{i+1}) + (T_{j-1} + T_{j+1})
 *   t = fma(-4, T, s)
 *   T' = fma(c, t, T_own)
 * RK2 midpoint (the time rule of the configuration; App. A itself uses
 * forward Euler, kept as scheme 1):
 *   stage 1: T* = fma(r/2, t(T^n), T^n)
 *   stage 2: T^{n+1} = fma(r, t(T*), T^n)
 * ====================================================================== */

static double heat_t(const double *u, int64_t nx, int64_t ny, int64_t i, int64_t j)
{
    const double uc = u[j * nx + i];
    const double uw = u[j * nx + wrapi(i - 1, nx)];
    const double ue = u[j * nx + wrapi(i + 1, nx)];
    const double us = u[wrapi(j - 1, ny) * nx + i];
    const double un = u[wrapi(j + 1, ny) * nx + i];
    const double s = (uw + ue) + (us + un);
    return fma(-4.0, uc, s);
}

/* one stage: out = fma(c, t(src), own) on every cell */
static void heat_stage(int64_t nx, int64_t ny, double c, const double *src,
                       const double *own, double *out)
{
    int64_t j;
#pragma omp parallel for schedule(static)
    for (j = 0; j < ny; ++j)
        for (int64_t i = 0; i < nx; ++i)
            out[j * nx + i] = fma(c, heat_t(src, nx, ny, i, j), own[j * nx + i]);
}

/* The mesh ratio of App. A, r = alpha dt / dx^2 (dy = dx, so r_x = r_y = r),
 * evaluated as written: the product alpha dt over the square dx dx. */
double oracle_heat_r(double alpha, double dt, double dx)
{
    return (alpha * dt) / (dx * dx);
}

/* scheme 0: RK2 midpoint; scheme 1: forward Euler (App. A update).  The
 * coefficient r comes from the physical inputs (alpha, dt, dx) of App. A. */
int oracle_heat_run(int64_t nx, int64_t ny, double alpha, double dt, double dx, int scheme,
                    double *u, int64_t nsteps)
{
    if (nx < 3 || ny < 3 || nsteps < 0 || (scheme != 0 && scheme != 1) || !(dx > 0.0) ||
        !(alpha > 0.0) || !(dt > 0.0))
        return ORACLE_EINVAL;
    const double r = oracle_heat_r(alpha, dt, dx);
    double *a = (double *)malloc(sizeof(double) * (size_t)(nx * ny));
    double *b = (double *)malloc(sizeof(double) * (size_t)(nx * ny));
    if (!a || !b) {
        free(a);
        free(b);
        return ORACLE_ENOMEM;
    }
    const double c1 = 0.5 * r;
    for (int64_t n = 0; n < nsteps; ++n) {
        if (scheme == 0) {
            heat_stage(nx, ny, c1, u, u, a); /* T*      */
            heat_stage(nx, ny, r, a, u, b);  /* T^{n+1} */
        } else {
            heat_stage(nx, ny, r, u, u, b);
        }
        memcpy(u, b, sizeof(double) * (size_t)(nx * ny));
    }
    free(a);
    free(b);
    return ORACLE_OK;
}

/* ======================================================================
 * Compressible Euler -- App. B.
 * Q = (rho, rho u, rho v, E), F = (rho u, rho u^2 + p, rho u v, (E+p) u),
 * G = (rho v, rho u v, rho v^2 + p, (E+p) v), E = p/(gamma-1) + rho(u^2+v^2)/2.
 * Signs: the conservative form Q_t + F_x + G_y = 0 of App. B (the
 * component-wise PDE lines printed above it are garbled; the conservative
 * form governs).
 * ====================================================================== */

/* Cell pressure used by the limiter (EOS of App. B), symmetric in x and y:
 *   inv = 1/rho; u = m_x*inv; v = m_y*inv; p = (gamma-1)*fma(-1/2, m_x u + m_y v, E) */
static double cell_pressure(double rho, double mx, double my, double E, double gamma)
{
    const double inv = 1.0 / rho;
    const double u = mx * inv;
    const double v = my * inv;
    const double ke2 = mx * u + my * v;
    return (gamma - 1.0) * fma(-0.5, ke2, E);
}

/* Pressure-ratio minmod of App. B.  With dm = P_i - P_{i-1} and
 * dp = P_{i+1} - P_i, the factor for the reconstruction of cell i towards
 * its + face is phi = min(dm/dp, 1) and towards its - face phi' =
 * min(dp/dm, 1), both only where the ratio lies strictly between 0 and
 * infinity, else 0.  Reading: the printed ratio and the exponents on it are
 * garbled; the orientation taken is the textbook minmod one (the limited
 * slope equals minmod(dm, dp)).  "0 < ratio < infinity" is read in exact
 * arithmetic: both differences nonzero with the same sign. */
static void minmod_pair(double dm, double dp, double *phi_plus, double *phi_minus)
{
    if ((dm > 0.0 && dp > 0.0) || (dm < 0.0 && dp < 0.0)) {
        const double th = dm / dp;
        const double thp = dp / dm;
        *phi_plus = th < 1.0 ? th : 1.0;
        *phi_minus = thp < 1.0 ? thp : 1.0;
    } else {
        *phi_plus = 0.0;
        *phi_minus = 0.0;
    }
}

/* Paper-literal orientation (variant): the ratio printed in App. B is
 * P_r,i = (P_{i+1}-P_i)/(P_i-P_{i-1}); the reconstruction of cell i towards
 * i+1/2 uses min(P_r,i, 1) and that of cell i+1 towards i+1/2 uses
 * min(1/P_r,i+1, 1) (reading the garbled exponent "1" as +1). */
static void literal_pair(double dm, double dp, double *phi_plus, double *phi_minus)
{
    if ((dm > 0.0 && dp > 0.0) || (dm < 0.0 && dp < 0.0)) {
        const double pr = dp / dm;  /* P_r,i         */
        const double pri = dm / dp; /* 1 / P_r,i     */
        *phi_plus = pr < 1.0 ? pr : 1.0;
        *phi_minus = pri < 1.0 ? pri : 1.0;
    } else {
        *phi_plus = 0.0;
        *phi_minus = 0.0;
    }
}

/* Flux of one reconstructed state in the face-normal frame q = (rho, m_n,
 * m_t, E): inv = 1/rho, u_n = m_n inv, u_t = m_t inv,
 * p = (gamma-1) fma(-1/2, fma(m_n, u_n, m_t u_t), E), c = sqrt((gamma p) inv),
 * f = (m_n, fma(m_n, u_n, p), m_t u_n, (E + p) u_n), lam = |u_n| + c. */
static void state_flux(const double q[4], double gamma, double f[4], double *lam)
{
    const double inv = 1.0 / q[0];
    const double un = q[1] * inv;
    const double ut = q[2] * inv;
    const double ke2 = fma(q[1], un, q[2] * ut);
    const double p = (gamma - 1.0) * fma(-0.5, ke2, q[3]);
    const double c = sqrt((gamma * p) * inv);
    f[0] = q[1];
    f[1] = fma(q[1], un, p);
    f[2] = q[2] * un;
    f[3] = (q[3] + p) * un;
    *lam = fabs(un) + c;
}

/* Numerical flux at the face between cells "0" and "1" of a line of four
 * cells (-1, 0, 1, 2), states in the face-normal frame, P the cell
 * pressures.  Reconstruction (App. B):
 *   Q_L = Q_0 + (phi_0/2)(Q_1 - Q_0),  Q_R = Q_1 - (phi'_1/2)(Q_1 - Q_0)
 * flux (App. B, the formula is the Rusanov / local Lax-Friedrichs one; the
 * text calls it Roe):
 *   Fh = 1/2 (F(Q_R) + F(Q_L) + r (Q_L - Q_R)),  r = max(|u_n|+c) over L, R
 * Reading: the spectral radius is taken as the larger of the two
 * reconstructed states' |u_n| + c (the paper does not say where). */
/* limiter 0: pressure minmod (textbook orientation); 1: paper-literal
 * orientation; 2: no limiting (phi = 1: the face value is the average of the
 * two cells).  Mode 2 is not a scheme of the paper: it exists so that a test
 * can pin the order of the flux, update and time rule without the limiter. */
static void limiter_pair(int limiter, double dm, double dp, double *phi_plus, double *phi_minus)
{
    if (limiter == 0) {
        minmod_pair(dm, dp, phi_plus, phi_minus);
    } else if (limiter == 1) {
        literal_pair(dm, dp, phi_plus, phi_minus);
    } else {
        *phi_plus = 1.0;
        *phi_minus = 1.0;
    }
}

static void face_flux(const double *qm1, const double *q0, const double *q1, const double *q2,
                      double pm1, double p0, double p1, double p2, double gamma, int limiter,
                      double fh[4])
{
    double phi0p, phi0m, phi1p, phi1m;
    limiter_pair(limiter, p0 - pm1, p1 - p0, &phi0p, &phi0m);
    limiter_pair(limiter, p1 - p0, p2 - p1, &phi1p, &phi1m);
    (void)qm1;
    (void)q2;
    (void)phi0m;
    (void)phi1p;
    const double hl = 0.5 * phi0p;
    const double hr = 0.5 * phi1m;
    double ql[4], qr[4], fl[4], fr[4], laml, lamr;
    for (int k = 0; k < 4; ++k) {
        const double dq = q1[k] - q0[k];
        ql[k] = fma(hl, dq, q0[k]);
        qr[k] = fma(-hr, dq, q1[k]);
    }
    state_flux(ql, gamma, fl, &laml);
    state_flux(qr, gamma, fr, &lamr);
    const double r = laml > lamr ? laml : lamr;
    for (int k = 0; k < 4; ++k)
        fh[k] = 0.5 * fma(r, ql[k] - qr[k], fl[k] + fr[k]);
}

/* state of cell (i, j) of SoA array q[4][ny][nx] in the x-normal frame
 * (rho, m_x, m_y, E) or the y-normal frame (rho, m_y, m_x, E) */
static void load_cell(const double *q, int64_t nx, int64_t ny, int64_t i, int64_t j, int ynormal,
                      double s[4])
{
    const int64_t ii = wrapi(i, nx), jj = wrapi(j, ny);
    const int64_t plane = nx * ny, c = jj * nx + ii;
    s[0] = q[c];
    s[1] = q[(ynormal ? 2 : 1) * plane + c];
    s[2] = q[(ynormal ? 1 : 2) * plane + c];
    s[3] = q[3 * plane + c];
}

static double pressure_at(const double *q, int64_t nx, int64_t ny, int64_t i, int64_t j,
                          double gamma)
{
    double s[4];
    load_cell(q, nx, ny, i, j, 0, s);
    return cell_pressure(s[0], s[1], s[2], s[3], gamma);
}

/* face flux through the face at i+1/2 (axis 0) or j+1/2 (axis 1), returned in
 * the (rho, m_x, m_y, E) ordering */
static void flux_at(const double *q, int64_t nx, int64_t ny, int64_t i, int64_t j, int axis,
                    double gamma, int limiter, double out[4])
{
    double c[4][4], p[4], fh[4];
    for (int m = 0; m < 4; ++m) {
        const int64_t ii = axis == 0 ? i - 1 + m : i;
        const int64_t jj = axis == 1 ? j - 1 + m : j;
        load_cell(q, nx, ny, ii, jj, axis, c[m]);
        p[m] = pressure_at(q, nx, ny, ii, jj, gamma);
    }
    face_flux(c[0], c[1], c[2], c[3], p[0], p[1], p[2], p[3], gamma, limiter, fh);
    out[0] = fh[0];
    out[1] = axis == 0 ? fh[1] : fh[2];
    out[2] = axis == 0 ? fh[2] : fh[1];
    out[3] = fh[3];
}

/* One stage at one cell (App. B time rule, written in difference form):
 *   out_k = fma(lam, (Fh_{i-1/2} - Fh_{i+1/2}) + (Gh_{j-1/2} - Gh_{j+1/2}), own_k)
 * with lam = dt/(2 dx) for stage 1 and dt/dx for stage 2 (dx = dy).
 * Reading: App. B prints "+" between the face fluxes and no minus sign,
 * which cannot conserve; the conservative difference of the form
 * Q_t + F_x + G_y = 0 is used. */
static void euler_cell(const double *src, const double *own, double *out, int64_t nx, int64_t ny,
                       int64_t i, int64_t j, double lam, double gamma, int limiter)
{
    double fm[4], fp[4], gm[4], gp[4];
    flux_at(src, nx, ny, i - 1, j, 0, gamma, limiter, fm);
    flux_at(src, nx, ny, i, j, 0, gamma, limiter, fp);
    flux_at(src, nx, ny, i, j - 1, 1, gamma, limiter, gm);
    flux_at(src, nx, ny, i, j, 1, gamma, limiter, gp);
    const int64_t plane = nx * ny, c = j * nx + i;
    for (int k = 0; k < 4; ++k) {
        const double d = (fm[k] - fp[k]) + (gm[k] - gp[k]);
        out[k * plane + c] = fma(lam, d, own[k * plane + c]);
    }
}

static void euler_stage(int64_t nx, int64_t ny, double lam, double gamma, int limiter,
                        const double *src, const double *own, double *out)
{
    int64_t j;
#pragma omp parallel for schedule(static)
    for (j = 0; j < ny; ++j)
        for (int64_t i = 0; i < nx; ++i)
            euler_cell(src, own, out, nx, ny, i, j, lam, gamma, limiter);
}

/* RK2 midpoint (App. B):  Q* = Q^n + (dt/2) R(Q^n),  Q^{n+1} = Q^n + dt R(Q*) */
int oracle_euler_run(int64_t nx, int64_t ny, double dt, double dx, double gamma, int limiter,
                     double *q, int64_t nsteps)
{
    if (nx < 5 || ny < 5 || nsteps < 0 || !(dx > 0.0) || limiter < 0 || limiter > 2)
        return ORACLE_EINVAL;
    const size_t n = (size_t)(4 * nx * ny);
    double *a = (double *)malloc(sizeof(double) * n);
    double *b = (double *)malloc(sizeof(double) * n);
    if (!a || !b) {
        free(a);
        free(b);
        return ORACLE_ENOMEM;
    }
    const double lam2 = dt / dx;
    const double lam1 = 0.5 * lam2;
    for (int64_t s = 0; s < nsteps; ++s) {
        euler_stage(nx, ny, lam1, gamma, limiter, q, q, a);
        euler_stage(nx, ny, lam2, gamma, limiter, a, q, b);
        memcpy(q, b, sizeof(double) * n);
    }
    free(a);
    free(b);
    return ORACLE_OK;
}

/* single face flux, exposed for the consistency and limiter pins:
 * states in the face-normal frame, cells -1, 0, 1, 2 */
void oracle_face_flux(const double *qm1, const double *q0, const double *q1, const double *q2,
                      double gamma, int limiter, double *fh)
{
    const double pm1 = cell_pressure(qm1[0], qm1[1], qm1[2], qm1[3], gamma);
    const double p0 = cell_pressure(q0[0], q0[1], q0[2], q0[3], gamma);
    const double p1 = cell_pressure(q1[0], q1[1], q1[2], q1[3], gamma);
    const double p2 = cell_pressure(q2[0], q2[1], q2[2], q2[3], gamma);
    face_flux(qm1, q0, q1, q2, pm1, p0, p1, p2, gamma, limiter, fh);
}

/* cell pressure of one conserved state (rho, m_x, m_y, E), exposed for its pin */
double oracle_cell_pressure(const double *q, double gamma)
{
    return cell_pressure(q[0], q[1], q[2], q[3], gamma);
}

/* limiter factors of one cell, exposed for the minmod pin */
void oracle_limiter(double dm, double dp, int limiter, double *phi_plus, double *phi_minus)
{
    limiter_pair(limiter, dm, dp, phi_plus, phi_minus);
}

/* physical flux of one state (face-normal frame), exposed for the pins */
void oracle_state_flux(const double *q, double gamma, double *f, double *lam)
{
    state_flux(q, gamma, f, lam);
}

/* ======================================================================
 * Swept-schedule replay -- Sec. 3.3, Eq. 1.
 *
 * Levels are RK stages: level 2m is Q^m, level 2m+1 is the stage value of
 * step m ("points are removed after each intermediate step", Sec. 3.3).
 * n is the radius of one stage (1 heat, 2 Euler); b the block edge; d the
 * number of levels one phase advances (1 <= d <= k = b/(2n) - 1, Eq. 1,
 * even so that every phase ends on a whole step).
 *
 * Shapes on a block grid with offset o (0 or b/2 in both x and y), for the
 * levels base+s of one cycle (s = 1..d):
 *   Up-Pyramid on block (I,J): [X+sn, X+b-sn) x [Y+sn, Y+b-sn)
 *       (the footprint loses n points per side per level, i.e. 2n of width)
 *   X-Bridge on the seam x = X+b:  [X+b-sn, X+b+sn) x [Y+sn, Y+b-sn)
 *   Y-Bridge on the seam y = Y+b:  [X+sn, X+b-sn) x [Y+b-sn, Y+b+sn)
 *   Octahedron, lower half, at the corner (X+b, Y+b): [X+b-sn, X+b+sn)^2
 *   Octahedron, upper half: an Up-Pyramid on the block of the grid shifted
 *       by b/2 that is centred on that corner, levels base+d+s.
 * with X = o + I b, Y = o + J b (periodic).  At every level the four kinds
 * partition the plane.  Phase order: Up-Pyramid; then repeated
 * [Bridges, Octahedron] with the grid offset alternating 0 and b/2; then
 * [Bridges, Down-Pyramid (the Octahedron's lower half alone)].  The levels
 * left over after the last whole cycle are taken one step at a time, the way
 * a Standard run takes them (Sec. 3.3 stops only at phase ends; an exact step
 * count is the reading taken here).
 *
 * Every (cell, level) is computed one at a time with the same per-cell
 * functions as the step-by-step runs above, reading from a store that keeps
 * every level.  A read is legal only if the value was produced in an earlier
 * phase, or earlier by the same shape (one shape is one block of work with
 * no communication inside it).
 * ====================================================================== */

typedef struct {
    int64_t nx, ny;
    int ncomp, n, eqn, limiter;
    double c1, c2, gamma; /* heat: r/2, r;   Euler: dt/(2dx), dt/dx */
    int64_t nlev;         /* levels stored: 0..nlev-1 */
    double *val;          /* [nlev][ncomp][ny][nx] */
    int32_t *phase;       /* producer phase of each (level, cell); -1 = not yet */
    int64_t *task;        /* producer shape of each (level, cell) */
    int64_t *reader;      /* last shape that read each (level, cell) from another shape */
    int64_t cur_phase, cur_task;
    int64_t *stats;       /* [0] cells computed, [1] cross-shape reads, [2] error code */
} replay_t;

#define RS_CELLS 0
#define RS_XREADS 1
#define RS_ERR 2
#define RS_BADLEV 3
#define RS_BADX 4
#define RS_BADY 5

static double *lev_ptr(replay_t *R, int64_t l) { return R->val + l * R->ncomp * R->nx * R->ny; }

/* 0: not available; 1: produced by this shape; 2: produced by another shape
 * in an earlier phase and read by this shape for the first time; 3: as 2 but
 * already counted for this shape */
static int avail(replay_t *R, int64_t l, int64_t i, int64_t j)
{
    const int64_t c = l * R->nx * R->ny + wrapi(j, R->ny) * R->nx + wrapi(i, R->nx);
    if (R->phase[c] < 0)
        return 0;
    if (R->task[c] == R->cur_task)
        return 1;
    if (R->phase[c] >= R->cur_phase)
        return 0;
    if (R->reader[c] == R->cur_task)
        return 3;
    R->reader[c] = R->cur_task;
    return 2;
}

static void replay_fail(replay_t *R, int code, int64_t l, int64_t i, int64_t j)
{
    if (R->stats[RS_ERR] == 0) {
        R->stats[RS_ERR] = code;
        R->stats[RS_BADLEV] = l;
        R->stats[RS_BADX] = i;
        R->stats[RS_BADY] = j;
    }
}

/* check the reads of level l at cell (i,j): the stencil cross of radius n at
 * level l-1 and, for a second stage, the cell itself at level l-2 */
static void check_reads(replay_t *R, int64_t l, int64_t i, int64_t j)
{
    const int n = R->n;
    for (int dd = -n; dd <= n; ++dd) {
        int a = avail(R, l - 1, i + dd, j);
        if (!a)
            replay_fail(R, ORACLE_EDEP, l, i, j);
        if (a == 2)
            R->stats[RS_XREADS]++;
        if (dd != 0) {
            a = avail(R, l - 1, i, j + dd);
            if (!a)
                replay_fail(R, ORACLE_EDEP, l, i, j);
            if (a == 2)
                R->stats[RS_XREADS]++;
        }
    }
    if ((l % 2) == 0) {
        const int a = avail(R, l - 2, i, j);
        if (!a)
            replay_fail(R, ORACLE_EDEP, l, i, j);
        if (a == 2)
            R->stats[RS_XREADS]++;
    }
}

static void compute_cell(replay_t *R, int64_t l, int64_t gi, int64_t gj)
{
    const int64_t i = wrapi(gi, R->nx), j = wrapi(gj, R->ny);
    const int64_t plane = R->nx * R->ny;
    const int64_t mark = l * plane + j * R->nx + i;
    if (R->phase[mark] >= 0) {
        replay_fail(R, ORACLE_EDUP, l, i, j);
        return;
    }
    check_reads(R, l, i, j);
    const int stage2 = (l % 2) == 0;
    const double *src = lev_ptr(R, l - 1);
    const double *own = lev_ptr(R, stage2 ? l - 2 : l - 1);
    double *out = lev_ptr(R, l);
    const double c = stage2 ? R->c2 : R->c1;
    if (R->eqn == 0)
        out[j * R->nx + i] = fma(c, heat_t(src, R->nx, R->ny, i, j), own[j * R->nx + i]);
    else
        euler_cell(src, own, out, R->nx, R->ny, i, j, c, R->gamma, R->limiter);
    R->phase[mark] = (int32_t)R->cur_phase;
    R->task[mark] = R->cur_task;
    R->stats[RS_CELLS]++;
}

static void do_rect(replay_t *R, int64_t l, int64_t x0, int64_t x1, int64_t y0, int64_t y1)
{
    for (int64_t y = y0; y < y1; ++y)
        for (int64_t x = x0; x < x1; ++x)
            compute_cell(R, l, x, y);
}

/* shape kinds */
#define SH_UP 0
#define SH_XB 1
#define SH_YB 2
#define SH_LO 3

static void do_shape(replay_t *R, int kind, int64_t X, int64_t Y, int64_t b, int64_t base, int d)
{
    const int64_t n = R->n;
    for (int64_t s = 1; s <= d; ++s) {
        const int64_t l = base + s;
        switch (kind) {
        case SH_UP:
            do_rect(R, l, X + s * n, X + b - s * n, Y + s * n, Y + b - s * n);
            break;
        case SH_XB:
            do_rect(R, l, X + b - s * n, X + b + s * n, Y + s * n, Y + b - s * n);
            break;
        case SH_YB:
            do_rect(R, l, X + s * n, X + b - s * n, Y + b - s * n, Y + b + s * n);
            break;
        default:
            do_rect(R, l, X + b - s * n, X + b + s * n, Y + b - s * n, Y + b + s * n);
            break;
        }
    }
}

/*
 * eqn 0 heat (params: c1 = r/2, c2 = r), eqn 1 Euler (c1 = dt/(2dx),
 * c2 = dt/dx, gamma, limiter).  state is [ncomp][ny][nx]; on success it holds
 * the level 2*nsteps.  stats (>= 8 int64): [0] cells computed, [1] values
 * read by a shape other than the one that produced them (each value counted
 * once per reading shape; the initial state counts as produced elsewhere),
 * [2] error code, [3..5] level/x/y of the
 * first error, [6] swept levels, [7] number of phases.
 * plant: 0 for the schedule above.  Nonzero values plant a known mistake so
 * that a test can show the checker catches it: 1 runs each Octahedron before
 * the Bridges of its cycle, 2 lets every phase advance to the smallest even
 * depth above b/(2n), where the shapes of neighbouring blocks overlap.
 * (Depth b/(2n) itself, one more than Eq. 1 allows, still passes: the
 * pyramid's top level is then empty; Eq. 1 keeps a top 2n wide.)
 */
int oracle_swept_replay(int eqn, int64_t nx, int64_t ny, int64_t b, int d, int64_t nsteps,
                        double c1, double c2, double gamma, int limiter, double *state,
                        int64_t *stats, int plant)
{
    const int n = eqn == 0 ? 1 : 2;
    const int ncomp = eqn == 0 ? 1 : 4;
    if (b <= 2 * n || (b % 2) != 0 || nx % b != 0 || ny % b != 0 || nx / b < 2 || ny / b < 2 ||
        d < 1 || d > b / (2 * n) - 1 || (d % 2) != 0 || nsteps < 0 || plant < 0 || plant > 2)
        return ORACLE_EINVAL;
    if (plant == 2)
        d = (int)(2 * (b / (4 * n)) + 2); /* beyond b/(2n) */
    replay_t R;
    memset(&R, 0, sizeof(R));
    R.nx = nx;
    R.ny = ny;
    R.ncomp = ncomp;
    R.n = n;
    R.eqn = eqn;
    R.limiter = limiter;
    R.c1 = c1;
    R.c2 = c2;
    R.gamma = gamma;
    R.nlev = 2 * nsteps + 1;
    R.stats = stats;
    for (int k = 0; k < 8; ++k)
        stats[k] = 0;
    const int64_t plane = nx * ny;
    R.val = (double *)malloc(sizeof(double) * (size_t)(R.nlev * ncomp * plane));
    R.phase = (int32_t *)malloc(sizeof(int32_t) * (size_t)(R.nlev * plane));
    R.task = (int64_t *)malloc(sizeof(int64_t) * (size_t)(R.nlev * plane));
    R.reader = (int64_t *)malloc(sizeof(int64_t) * (size_t)(R.nlev * plane));
    if (!R.val || !R.phase || !R.task || !R.reader) {
        free(R.val);
        free(R.phase);
        free(R.task);
        free(R.reader);
        return ORACLE_ENOMEM;
    }
    for (int64_t k = 0; k < R.nlev * ncomp * plane; ++k)
        R.val[k] = NAN; /* a read of an unwritten value would show up as NaN */
    for (int64_t k = 0; k < R.nlev * plane; ++k) {
        R.phase[k] = -1;
        R.task[k] = -1;
        R.reader[k] = -1;
    }
    memcpy(R.val, state, sizeof(double) * (size_t)(ncomp * plane));
    for (int64_t k = 0; k < plane; ++k) {
        R.phase[k] = 0; /* level 0: the initial state, phase 0 */
        R.task[k] = -2;
    }
    const int64_t L = 2 * nsteps;
    const int64_t TI = nx / b, TJ = ny / b;
    int64_t swept = 0;
    int64_t ph = 0;
    int64_t taskid = 0;
    if (L >= d) {
        const int64_t m = L / d - 1; /* whole cycles after the Up-Pyramid */
        swept = (m + 1) * d;
        /* Up-Pyramid on the unshifted grid */
        R.cur_phase = ++ph;
        for (int64_t J = 0; J < TJ; ++J)
            for (int64_t I = 0; I < TI; ++I) {
                R.cur_task = taskid++;
                do_shape(&R, SH_UP, I * b, J * b, b, 0, d);
            }
        for (int64_t c = 0; c <= m; ++c) {
            const int64_t o = (c % 2) ? b / 2 : 0;
            const int64_t base = c * d;
            for (int part = 0; part < 2; ++part) {
                const int bridges = (part == 0) != (plant == 1);
                R.cur_phase = ++ph;
                if (bridges) {
                    /* X- and Y-Bridges on the seams of this cycle's grid */
                    for (int64_t J = 0; J < TJ; ++J)
                        for (int64_t I = 0; I < TI; ++I) {
                            R.cur_task = taskid++;
                            do_shape(&R, SH_XB, o + I * b, o + J * b, b, base, d);
                            R.cur_task = taskid++;
                            do_shape(&R, SH_YB, o + I * b, o + J * b, b, base, d);
                        }
                } else {
                    /* Octahedron (c < m) or Down-Pyramid (c == m) at every corner */
                    for (int64_t J = 0; J < TJ; ++J)
                        for (int64_t I = 0; I < TI; ++I) {
                            R.cur_task = taskid++;
                            do_shape(&R, SH_LO, o + I * b, o + J * b, b, base, d);
                            if (c < m)
                                do_shape(&R, SH_UP, o + I * b + b / 2, o + J * b + b / 2, b,
                                         base + d, d);
                        }
                }
            }
        }
    }
    /* remaining levels, one level over the whole grid per phase */
    for (int64_t l = swept + 1; l <= L; ++l) {
        R.cur_phase = ++ph;
        R.cur_task = taskid++;
        do_rect(&R, l, 0, nx, 0, ny);
    }
    stats[6] = swept;
    stats[7] = ph;
    int rc = (int)stats[RS_ERR];
    if (rc == 0) {
        for (int64_t k = plane; k < R.nlev * plane; ++k)
            if (R.phase[k] < 0) {
                const int64_t l = k / plane, c = k % plane;
                replay_fail(&R, ORACLE_EGAP, l, c % nx, c / nx);
                rc = ORACLE_EGAP;
                break;
            }
    }
    if (rc == 0)
        memcpy(state, lev_ptr(&R, L), sizeof(double) * (size_t)(ncomp * plane));
    free(R.val);
    free(R.phase);
    free(R.task);
    free(R.reader);
    return rc;
}

/* ======================================================================
 * Discrete adjoints (reverse mode of the schemes above).
 *
 * The swept rule only reorders the explicit scheme (Sec. 3.3), so its
 * gradient is the gradient of the step-by-step scheme.  For a final-state
 * loss L(Q^N), lam^N = dL/dQ^N and lam^n = (dQ^{n+1}/dQ^n)^T lam^{n+1}.
 * Non-smooth points (the limiter's switches, max of the wave speeds, |u_n|)
 * take the derivative of the branch the forward step took.
 * ====================================================================== */

/* Heat: the step Q' = Q + c2 L(Q + c1 L Q) with symmetric L.  Adjoint step
 * (order pinned): mu* = c2 * t(lam); lam_n = fma(c1, t(mu*), lam + mu*),
 * t(u) = fma(-4, u, (u_W + u_E) + (u_S + u_N)). */
int oracle_heat_adjoint(int64_t nx, int64_t ny, double alpha, double dt, double dx, double *lam,
                        int64_t nsteps)
{
    if (nx < 3 || ny < 3 || nsteps < 0 || !(dx > 0.0) || !(alpha > 0.0) || !(dt > 0.0))
        return ORACLE_EINVAL;
    const double r = oracle_heat_r(alpha, dt, dx);
    const size_t n = (size_t)(nx * ny);
    double *ms = (double *)malloc(sizeof(double) * n);
    double *out = (double *)malloc(sizeof(double) * n);
    if (!ms || !out) {
        free(ms);
        free(out);
        return ORACLE_ENOMEM;
    }
    const double c1 = 0.5 * r;
    for (int64_t s = 0; s < nsteps; ++s) {
        int64_t j;
#pragma omp parallel for schedule(static)
        for (j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i)
                ms[j * nx + i] = r * heat_t(lam, nx, ny, i, j);
#pragma omp parallel for schedule(static)
        for (j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) {
                const int64_t c = j * nx + i;
                out[c] = fma(c1, heat_t(ms, nx, ny, i, j), lam[c] + ms[c]);
            }
        memcpy(lam, out, sizeof(double) * n);
    }
    free(ms);
    free(out);
    return ORACLE_OK;
}

/* --- Euler: reverse mode of one face flux -------------------------------- */

/* adjoint of the cell pressure: P = (gamma-1) fma(-1/2, m_x u + m_y v, E) */
static void cell_pressure_bar(const double q[4], double gamma, double pbar, double qbar[4])
{
    const double inv = 1.0 / q[0];
    const double u = q[1] * inv, v = q[2] * inv;
    const double g1 = gamma - 1.0;
    const double ebar = pbar * g1;
    const double kbar = -0.5 * g1 * pbar;
    double mxbar = kbar * u, mybar = kbar * v;
    const double ubar = kbar * q[1], vbar = kbar * q[2];
    mxbar += ubar * inv;
    mybar += vbar * inv;
    const double invbar = ubar * q[1] + vbar * q[2];
    qbar[0] += -invbar * inv * inv;
    qbar[1] += mxbar;
    qbar[2] += mybar;
    qbar[3] += ebar;
}

/* adjoint of state_flux: given fbar[4] and lambar, accumulate qbar[4] */
static void state_flux_bar(const double q[4], double gamma, const double fbar[4], double lambar,
                           double qbar[4])
{
    const double inv = 1.0 / q[0];
    const double mn = q[1], mt = q[2], E = q[3];
    const double un = mn * inv, ut = mt * inv;
    const double ke2 = fma(mn, un, mt * ut);
    const double g1 = gamma - 1.0;
    const double p = g1 * fma(-0.5, ke2, E);
    const double c = sqrt((gamma * p) * inv);
    double mnbar = fbar[0], mtbar = 0.0, Ebar = 0.0, unbar = 0.0, utbar = 0.0, pbar = 0.0,
           invbar = 0.0;
    /* f1 = mn un + p */
    mnbar += fbar[1] * un;
    unbar += fbar[1] * mn;
    pbar += fbar[1];
    /* f2 = mt un */
    mtbar += fbar[2] * un;
    unbar += fbar[2] * mt;
    /* f3 = (E + p) un */
    Ebar += fbar[3] * un;
    pbar += fbar[3] * un;
    unbar += fbar[3] * (E + p);
    /* lam = |un| + c */
    unbar += un > 0.0 ? lambar : (un < 0.0 ? -lambar : 0.0);
    const double cbar = lambar;
    /* c = sqrt(s), s = gamma p inv */
    const double sbar = c > 0.0 ? cbar / (2.0 * c) : 0.0;
    pbar += sbar * gamma * inv;
    invbar += sbar * gamma * p;
    /* p = g1 (E - ke2/2) */
    Ebar += pbar * g1;
    const double kbar = -0.5 * g1 * pbar;
    /* ke2 = mn un + mt ut */
    mnbar += kbar * un;
    unbar += kbar * mn;
    mtbar += kbar * ut;
    utbar += kbar * mt;
    /* un = mn inv, ut = mt inv */
    mnbar += unbar * inv;
    invbar += unbar * mn;
    mtbar += utbar * inv;
    invbar += utbar * mt;
    qbar[0] += -invbar * inv * inv;
    qbar[1] += mnbar;
    qbar[2] += mtbar;
    qbar[3] += Ebar;
}

/* derivatives of one limiter factor with respect to (dm, dp), for the
 * branch taken: plus = min(dm/dp, 1) or minus = min(dp/dm, 1) where both
 * differences are nonzero with equal signs */
static void limiter_grad(int limiter, int plus, double dm, double dp, double *d_dm, double *d_dp)
{
    *d_dm = 0.0;
    *d_dp = 0.0;
    if (limiter == 2)
        return;
    if (!((dm > 0.0 && dp > 0.0) || (dm < 0.0 && dp < 0.0)))
        return;
    /* which quotient this factor is: textbook plus = dm/dp, minus = dp/dm;
     * the printed orientation swaps them */
    const int over_dp = (limiter == 0) ? plus : !plus; /* factor = dm/dp ? */
    if (over_dp) {
        if (dm / dp < 1.0) {
            *d_dm = 1.0 / dp;
            *d_dp = -dm / (dp * dp);
        }
    } else {
        if (dp / dm < 1.0) {
            *d_dp = 1.0 / dm;
            *d_dm = -dp / (dm * dm);
        }
    }
}

/* Reverse of face_flux at the face between cells 0 and 1 of the line
 * (-1, 0, 1, 2), states in the face-normal frame.  a[4]: adjoint of the
 * numerical flux.  Accumulates into qbar[m][4], m = 0..3 (cells -1..2), the
 * whole gradient of <a, Fh>: through the reconstructed states into cells 0
 * and 1, and through the limiter's pressures into all four cells, each
 * pressure reversed right here for this face (chain rule, face by face). */
static void face_flux_bar(const double *q[4], double gamma, int limiter, const double a[4],
                          double qbar[4][4])
{
    double p[4];
    for (int m = 0; m < 4; ++m)
        p[m] = cell_pressure(q[m][0], q[m][1], q[m][2], q[m][3], gamma);
    double phi0p, phi0m, phi1p, phi1m;
    limiter_pair(limiter, p[1] - p[0], p[2] - p[1], &phi0p, &phi0m);
    limiter_pair(limiter, p[2] - p[1], p[3] - p[2], &phi1p, &phi1m);
    const double hl = 0.5 * phi0p, hr = 0.5 * phi1m;
    double dq[4], ql[4], qr[4], fl[4], fr[4], laml, lamr;
    for (int k = 0; k < 4; ++k) {
        dq[k] = q[2][k] - q[1][k];
        ql[k] = fma(hl, dq[k], q[1][k]);
        qr[k] = fma(-hr, dq[k], q[2][k]);
    }
    state_flux(ql, gamma, fl, &laml);
    state_flux(qr, gamma, fr, &lamr);
    const double r = laml > lamr ? laml : lamr;
    /* Fh_k = 1/2 (r (ql_k - qr_k) + fl_k + fr_k) */
    double qlbar[4], qrbar[4], flbar[4], frbar[4], rbar = 0.0;
    for (int k = 0; k < 4; ++k) {
        flbar[k] = 0.5 * a[k];
        frbar[k] = 0.5 * a[k];
        qlbar[k] = 0.5 * r * a[k];
        qrbar[k] = -0.5 * r * a[k];
        rbar += 0.5 * a[k] * (ql[k] - qr[k]);
    }
    const double lamlbar = laml > lamr ? rbar : 0.0;
    const double lamrbar = laml > lamr ? 0.0 : rbar;
    double sl[4] = {0, 0, 0, 0}, sr[4] = {0, 0, 0, 0};
    state_flux_bar(ql, gamma, flbar, lamlbar, sl);
    state_flux_bar(qr, gamma, frbar, lamrbar, sr);
    for (int k = 0; k < 4; ++k) {
        qlbar[k] += sl[k];
        qrbar[k] += sr[k];
    }
    /* ql = q0 + hl dq, qr = q1 - hr dq, dq = q1 - q0 */
    double hlbar = 0.0, hrbar = 0.0;
    for (int k = 0; k < 4; ++k) {
        const double dqbar = qlbar[k] * hl - qrbar[k] * hr;
        hlbar += qlbar[k] * dq[k];
        hrbar += -qrbar[k] * dq[k];
        qbar[1][k] += qlbar[k] - dqbar;
        qbar[2][k] += qrbar[k] + dqbar;
    }
    /* hl = phi0p / 2 from (p0 - pm1, p1 - p0); hr = phi1m / 2 from (p1 - p0, p2 - p1) */
    double pbar[4] = {0, 0, 0, 0}, g_dm, g_dp;
    limiter_grad(limiter, 1, p[1] - p[0], p[2] - p[1], &g_dm, &g_dp);
    pbar[1] += 0.5 * hlbar * g_dm;
    pbar[0] -= 0.5 * hlbar * g_dm;
    pbar[2] += 0.5 * hlbar * g_dp;
    pbar[1] -= 0.5 * hlbar * g_dp;
    limiter_grad(limiter, 0, p[2] - p[1], p[3] - p[2], &g_dm, &g_dp);
    pbar[2] += 0.5 * hrbar * g_dm;
    pbar[1] -= 0.5 * hrbar * g_dm;
    pbar[3] += 0.5 * hrbar * g_dp;
    pbar[2] -= 0.5 * hrbar * g_dp;
    for (int m = 0; m < 4; ++m)
        cell_pressure_bar(q[m], gamma, pbar[m], qbar[m]);
}

/* out = J^T v for the residual d(Q)_c = (Fh_{i-1/2} - Fh_{i+1/2}) + (Gh_{j-1/2}
 * - Gh_{j+1/2}) of every cell (out is overwritten).  Each face, visited x
 * faces then y faces in raster order, adds its whole contribution for
 * a = v_{right} - v_{left} (face_flux_bar) to the four cells of its line. */
static void euler_residual_vjp(const double *q, const double *v, double *out, int64_t nx,
                               int64_t ny, double gamma, int limiter)
{
    const int64_t plane = nx * ny;
    memset(out, 0, sizeof(double) * (size_t)(4 * plane));
    for (int axis = 0; axis < 2; ++axis)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) {
                /* face between cell (i,j) and its + neighbour along axis */
                double cells[4][4];
                const double *qp[4];
                int64_t idx[4];
                for (int m = 0; m < 4; ++m) {
                    const int64_t ii = axis == 0 ? i - 1 + m : i;
                    const int64_t jj = axis == 1 ? j - 1 + m : j;
                    load_cell(q, nx, ny, ii, jj, axis, cells[m]);
                    qp[m] = cells[m];
                    idx[m] = wrapi(jj, ny) * nx + wrapi(ii, nx);
                }
                /* adjoint of the flux in the face-normal frame */
                double a[4];
                const int64_t cl = idx[1], cr = idx[2];
                for (int k = 0; k < 4; ++k) {
                    const int kk = (axis == 1 && (k == 1 || k == 2)) ? 3 - k : k;
                    a[k] = v[kk * plane + cr] - v[kk * plane + cl];
                }
                double qb[4][4] = {{0}};
                face_flux_bar(qp, gamma, limiter, a, qb);
                for (int m = 0; m < 4; ++m)
                    for (int k = 0; k < 4; ++k) {
                        const int kk = (axis == 1 && (k == 1 || k == 2)) ? 3 - k : k;
                        out[kk * plane + idx[m]] += qb[m][k];
                    }
            }
}

/* One adjoint RK2 step at Q^n (RK2: Q* = Q + lam1 d(Q), Q' = Q + lam2 d(Q*)):
 *   mu*  = lam2 J(Q*)^T lam'
 *   lam  = lam' + mu* + lam1 J(Q)^T mu*                                  */
static void euler_adjoint_step(const double *q, double *lam, int64_t nx, int64_t ny, double lam1,
                               double lam2, double gamma, int limiter, double *qs, double *ms,
                               double *tmp)
{
    const int64_t n4 = 4 * nx * ny;
    euler_stage(nx, ny, lam1, gamma, limiter, q, q, qs); /* Q* */
    euler_residual_vjp(qs, lam, tmp, nx, ny, gamma, limiter);
    for (int64_t k = 0; k < n4; ++k)
        ms[k] = lam2 * tmp[k];
    euler_residual_vjp(q, ms, tmp, nx, ny, gamma, limiter);
    for (int64_t k = 0; k < n4; ++k)
        lam[k] = lam[k] + ms[k] + lam1 * tmp[k];
}

/* Gradient of L(Q^N) with respect to Q^0.  lam holds dL/dQ^N on entry and
 * dL/dQ^0 on return.  Forward states are checkpointed every `ckpt` steps and
 * recomputed step by step inside each segment. */
int oracle_euler_adjoint(int64_t nx, int64_t ny, double dt, double dx, double gamma, int limiter,
                         const double *q0, double *lam, int64_t nsteps, int64_t ckpt)
{
    if (nx < 5 || ny < 5 || nsteps < 0 || ckpt < 1 || !(dx > 0.0) || limiter < 0 || limiter > 2)
        return ORACLE_EINVAL;
    const size_t n4 = (size_t)(4 * nx * ny);
    const int64_t nseg = (nsteps + ckpt - 1) / ckpt;
    double *cps = (double *)malloc(sizeof(double) * n4 * (size_t)(nseg > 0 ? nseg : 1));
    double *seg = (double *)malloc(sizeof(double) * n4 * (size_t)(ckpt + 1));
    double *qs = (double *)malloc(sizeof(double) * n4);
    double *ms = (double *)malloc(sizeof(double) * n4);
    double *tmp = (double *)malloc(sizeof(double) * n4);
    if (!cps || !seg || !qs || !ms || !tmp) {
        free(cps);
        free(seg);
        free(qs);
        free(ms);
        free(tmp);
        return ORACLE_ENOMEM;
    }
    const double lam2 = dt / dx, lam1 = 0.5 * lam2;
    /* forward pass: checkpoints Q^{s*ckpt} */
    memcpy(seg, q0, sizeof(double) * n4);
    for (int64_t s = 0; s < nseg; ++s) {
        memcpy(cps + (size_t)s * n4, seg, sizeof(double) * n4);
        const int64_t len = (s + 1) * ckpt <= nsteps ? ckpt : nsteps - s * ckpt;
        for (int64_t t = 0; t < len; ++t) {
            euler_stage(nx, ny, lam1, gamma, limiter, seg, seg, qs);
            euler_stage(nx, ny, lam2, gamma, limiter, qs, seg, tmp);
            memcpy(seg, tmp, sizeof(double) * n4);
        }
    }
    /* backward pass, segment by segment */
    for (int64_t s = nseg - 1; s >= 0; --s) {
        const int64_t len = (s + 1) * ckpt <= nsteps ? ckpt : nsteps - s * ckpt;
        memcpy(seg, cps + (size_t)s * n4, sizeof(double) * n4);
        for (int64_t t = 0; t < len - 1; ++t) {
            double *cur = seg + (size_t)t * n4, *nxt = seg + (size_t)(t + 1) * n4;
            euler_stage(nx, ny, lam1, gamma, limiter, cur, cur, qs);
            euler_stage(nx, ny, lam2, gamma, limiter, qs, cur, nxt);
        }
        for (int64_t t = len - 1; t >= 0; --t)
            euler_adjoint_step(seg + (size_t)t * n4, lam, nx, ny, lam1, lam2, gamma, limiter, qs,
                               ms, tmp);
    }
    free(cps);
    free(seg);
    free(qs);
    free(ms);
    free(tmp);
    return ORACLE_OK;
}

/* single-face reverse mode, exposed for the adjoint pins: qbar[16] += the
 * gradient of <a, Fh(q-1, q0, q1, q2)> with respect to the four states */
void oracle_face_flux_vjp(const double *qm1, const double *q0, const double *q1, const double *q2,
                          double gamma, int limiter, const double *a, double *qbar)
{
    const double *q[4] = {qm1, q0, q1, q2};
    double qb[4][4] = {{0}};
    face_flux_bar(q, gamma, limiter, a, qb);
    for (int m = 0; m < 4; ++m)
        for (int k = 0; k < 4; ++k)
            qbar[4 * m + k] += qb[m][k];
}
