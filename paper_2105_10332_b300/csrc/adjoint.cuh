// adjoint.cuh -- discrete adjoints (reverse mode) of the two schemes.
//
// The swept rule only reorders the explicit scheme (Sec. 3.3), so the
// gradient of a final-state loss L(Q^N) is the gradient of the step-by-step
// scheme: lam^N = dL/dQ^N, lam^n = (dQ^{n+1}/dQ^n)^T lam^{n+1}.  Non-smooth
// points (the limiter's switches, max of the wave speeds, |u_n|) take the
// derivative of the branch the forward step took.
//
// Heat (App. A): the RK2 step Q' = Q + c2 L(Q + c1 L Q) has a symmetric L,
// so its adjoint step is again a two-stage stencil update of radius 1,
//   mu* = c2 t(lam),   lam_n = fma(c1, t(mu*), lam + mu*),
// and runs through the swept kernels unchanged (equation type HeatAdj).
//
// Euler (App. B): per reverse step, with Q* = Q + lam1 d(Q) rebuilt from Q,
//   mu*   = lam2 J(Q*)^T lam'
//   lam_n = (lam' + mu*) + lam1 J(Q)^T mu*
// where d(Q)_c = (Fh_{i-1/2} - Fh_{i+1/2}) + (Gh_{j-1/2} - Gh_{j+1/2}).  J^T v
// is assembled face by face: each face's flux depends on the four cells of
// its line, and its adjoint input is v_right - v_left; k_face_vjp writes the
// four cells' contributions of every face and k_gather sums, per cell, the
// contributions of its faces (x faces, then y faces, each in the order of
// the face's index along its line, wrapped periodically).  A face's flux
// reaches its two cells through the reconstructed states and all four cells
// of its line through the limiter's pressures; the pressure's own reverse is
// linear in the pressure adjoint and the same for every face of a cell, so
// the faces hand over pressure adjoints and k_gather applies that reverse
// once per cell to their sum.  What several faces share is computed once
// beforehand, with the same operations in the same order: per cell the
// pressure, 1/rho and the velocities (k_vjp_cells), per cell and axis the
// half limiter factors and their derivatives (k_vjp_limiters).
#pragma once

#include "kernels.cuh"

namespace sweep {

// ------------------------------------------------------------------ heat

struct HeatAdj {
    static constexpr int NC = 1;
    static constexpr int N = 1;
    static constexpr int SWEPT_THREADS = 256, STD_THREADS = 256;
};

template <int C>
struct Stage<HeatAdj, C> {
    __device__ __forceinline__ static void run(const Params &p, Block<HeatAdj, C> &B, int64_t level,
                                               Rect R)
    {
        const bool second = (level & 1) == 0;
        const double *src = B.lev(level - 1);
        const double *own = B.lev(level);
        const int wp = B.wp;
        const Fx F = p.ek.f;
        for_rect(band(R, B.rank, C), [&](int x, int y) {
            const int i = y * wp + x;
            const double s = fadd(fadd(src[i - 1], src[i + 1], F), fadd(src[i - wp], src[i + wp], F), F);
            const double t = __fma_rn(-4.0, src[i], s);
            // first stage: mu* = r t(lam); second: fma(r/2, t(mu*), lam + mu*)
            const double v = second ? __fma_rn(p.c1, t, fadd(own[i], src[i], F))
                                    : fmul(p.c2, t, F);
            B.put(level, 0, i, v);
        });
    }
};

// ------------------------------------------------------------------ Euler

// Half limiter factors of one cell (as limiter_halves) and, for the branch
// taken, their derivatives with respect to dm and dp.  A factor that is a
// quotient below 1 has derivative (1/den, -num/den^2) in (num, den); a
// factor clipped to 1, or zero, has derivative 0.
__device__ __forceinline__ void limiter_halves_grad(double dm, double dp, int mode, const Fx &F,
                                                    double &hp, double &hm, double &dhp_dm,
                                                    double &dhp_dp, double &dhm_dm, double &dhm_dp)
{
    limiter_halves(dm, dp, mode, F, hp, hm);
    dhp_dm = dhp_dp = dhm_dm = dhm_dp = 0.0;
    if (mode == 2)
        return;
    const bool same = (dm > 0.0 && dp > 0.0) || (dm < 0.0 && dp < 0.0);
    if (!same)
        return;
    // dm/dp and dp/dm, each used only where it is the factor and below 1
    const double q_mp = __ddiv_rn(dm, dp);
    const double q_pm = __ddiv_rn(dp, dm);
    // textbook: plus = dm/dp, minus = dp/dm; printed orientation swaps them
    const bool plus_is_mp = mode == 0;
    double g_mp_dm = 0.0, g_mp_dp = 0.0, g_pm_dm = 0.0, g_pm_dp = 0.0;
    if (q_mp < 1.0) {
        g_mp_dm = __ddiv_rn(1.0, dp);
        g_mp_dp = __ddiv_rn(-dm, fmul(dp, dp, F));
    }
    if (q_pm < 1.0) {
        g_pm_dp = __ddiv_rn(1.0, dm);
        g_pm_dm = __ddiv_rn(-dp, fmul(dm, dm, F));
    }
    // the halves carry a factor 1/2
    dhp_dm = fmul(0.5, plus_is_mp ? g_mp_dm : g_pm_dm, F);
    dhp_dp = fmul(0.5, plus_is_mp ? g_mp_dp : g_pm_dp, F);
    dhm_dm = fmul(0.5, plus_is_mp ? g_pm_dm : g_mp_dm, F);
    dhm_dp = fmul(0.5, plus_is_mp ? g_pm_dp : g_mp_dp, F);
}

// reverse of cell_pressure: add to qb the gradient of pb * P(q), given the
// cell's momenta (mn, mt) in the face-normal frame and its 1/rho and
// velocities (un, ut) in the same frame
__device__ __forceinline__ void cell_pressure_vjp(double mn, double mt, double inv, double un,
                                                  double ut, const EulerConst &k, double pb,
                                                  double qb[4])
{
    const Fx &F = k.f;
    const double eb = fmul(pb, k.gm1, F);
    const double kb = fmul(fmul(-0.5, k.gm1, F), pb, F);
    const double ub = fmul(kb, mn, F), vb = fmul(kb, mt, F);
    const double mxb = fadd(fmul(kb, un, F), fmul(ub, inv, F), F);
    const double myb = fadd(fmul(kb, ut, F), fmul(vb, inv, F), F);
    const double invb = fadd(fmul(ub, mn, F), fmul(vb, mt, F), F);
    qb[0] = fadd(qb[0], fmul(fmul(-invb, inv, F), inv, F), F);
    qb[1] = fadd(qb[1], mxb, F);
    qb[2] = fadd(qb[2], myb, F);
    qb[3] = fadd(qb[3], eb, F);
}

// reverse of state_flux (face-normal frame): add to qb the gradient of
// <fb, F(q)> + lb * lam(q); s holds the forward pass's intermediates and sb
// the adjoint of c^2 = (gamma p) inv, lb / (2c) (0 where lb or c is 0),
// which the caller forms once for the one state that carries lb
__device__ __forceinline__ void state_flux_vjp(const double q[4], const FluxParts &s,
                                               const EulerConst &k, const double fb[4], double lb,
                                               double sb, double qb[4])
{
    const Fx &F = k.f;
    const double inv = s.inv, un = s.un, ut = s.ut, p = s.p;
    const double mn = q[1], mt = q[2], E = q[3];
    double mnb = fb[0], mtb, Eb, unb, utb, pb, invb;
    // f1 = mn un + p
    mnb = fadd(mnb, fmul(fb[1], un, F), F);
    unb = fmul(fb[1], mn, F);
    pb = fb[1];
    // f2 = mt un
    mtb = fmul(fb[2], un, F);
    unb = fadd(unb, fmul(fb[2], mt, F), F);
    // f3 = (E + p) un
    Eb = fmul(fb[3], un, F);
    pb = fadd(pb, fmul(fb[3], un, F), F);
    unb = fadd(unb, fmul(fb[3], fadd(E, p, F), F), F);
    // lam = |un| + c
    unb = fadd(unb, un > 0.0 ? lb : (un < 0.0 ? -lb : 0.0), F);
    // c = sqrt(s), s = (gamma p) inv
    pb = fadd(pb, fmul(fmul(sb, k.gamma, F), inv, F), F);
    invb = fmul(fmul(sb, k.gamma, F), p, F);
    // p = g1 (E - ke2/2)
    Eb = fadd(Eb, fmul(pb, k.gm1, F), F);
    const double kb = fmul(fmul(-0.5, k.gm1, F), pb, F);
    // ke2 = mn un + mt ut
    mnb = fadd(mnb, fmul(kb, un, F), F);
    unb = fadd(unb, fmul(kb, mn, F), F);
    mtb = fadd(mtb, fmul(kb, ut, F), F);
    utb = fmul(kb, mt, F);
    // un = mn inv, ut = mt inv
    mnb = fadd(mnb, fmul(unb, inv, F), F);
    invb = fadd(invb, fmul(unb, mn, F), F);
    mtb = fadd(mtb, fmul(utb, inv, F), F);
    invb = fadd(invb, fmul(utb, mt, F), F);
    qb[0] = fadd(qb[0], fmul(fmul(-invb, inv, F), inv, F), F);
    qb[1] = fadd(qb[1], mnb, F);
    qb[2] = fadd(qb[2], mtb, F);
    qb[3] = fadd(qb[3], Eb, F);
}

// Reverse of the numerical flux at the face between cells 1 and 2 of the
// line of cells 0..3 (face-normal frame).  q1, q2: the states of cells 1
// and 2; lim1 = (h+, dh+/ddm, dh+/ddp) of cell 1 and lim2 = (h-, dh-/ddm,
// dh-/ddp) of cell 2 along the face's axis; a: adjoint of the flux.
// qb[0], qb[1] receive the gradient for cells 1 and 2 through the
// reconstructed states, pb[m] the adjoint of cell m's pressure.
__device__ __forceinline__ void face_flux_vjp(const double q1[4], const double q2[4],
                                              const double lim1[3], const double lim2[3],
                                              const double a[4], const EulerConst &k,
                                              double qb[2][4], double pb[4])
{
    const Fx &F = k.f;
    const double hl = lim1[0], dl_dm = lim1[1], dl_dp = lim1[2];
    const double hr = lim2[0], dr_dm = lim2[1], dr_dp = lim2[2];
    double dq[4], ql[4], qr[4], fl[4], fr[4], laml, lamr;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        dq[c] = fadd(q2[c], -q1[c], F);
        ql[c] = __fma_rn(hl, dq[c], q1[c]);
        qr[c] = __fma_rn(-hr, dq[c], q2[c]);
    }
    FluxParts pl, pr;
    state_flux(ql[0], ql[1], ql[2], ql[3], k, fl, laml, pl);
    state_flux(qr[0], qr[1], qr[2], qr[3], k, fr, lamr, pr);
    const bool left = __double_as_longlong(laml) > __double_as_longlong(lamr);
    const double r = left ? laml : lamr;
    // Fh_c = 1/2 (r (ql_c - qr_c) + fl_c + fr_c)
    // (-r/2) a rounds to exactly -((r/2) a), signed zeros included (round
    // to nearest is symmetric), so qrb starts as the negation of qlb
    double qlb[4], qrb[4], flb[4], frb[4], rb = 0.0;
    const double half_r = fmul(0.5, r, F);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        flb[c] = fmul(0.5, a[c], F);
        frb[c] = flb[c];
        qlb[c] = fmul(half_r, a[c], F);
        qrb[c] = -qlb[c];
        rb = fadd(rb, fmul(flb[c], fadd(ql[c], -qr[c], F), F), F);
    }
    // r = lam of one state: only that state's sound speed carries rb
    const double cm = left ? pl.c : pr.c;
    const double sbm = cm > 0.0 ? __ddiv_rn(rb, fmul(2.0, cm, F)) : 0.0;
    double sl[4] = {0.0, 0.0, 0.0, 0.0}, sr[4] = {0.0, 0.0, 0.0, 0.0};
    state_flux_vjp(ql, pl, k, flb, left ? rb : 0.0, left ? sbm : 0.0, sl);
    state_flux_vjp(qr, pr, k, frb, left ? 0.0 : rb, left ? 0.0 : sbm, sr);
    double hlb = 0.0, hrb = 0.0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        qlb[c] = fadd(qlb[c], sl[c], F);
        qrb[c] = fadd(qrb[c], sr[c], F);
        // ql = q1 + hl dq, qr = q2 - hr dq, dq = q2 - q1
        const double dqb = fadd(fmul(qlb[c], hl, F), -fmul(qrb[c], hr, F), F);
        hlb = fadd(hlb, fmul(qlb[c], dq[c], F), F);
        hrb = fadd(hrb, fmul(-qrb[c], dq[c], F), F);
        qb[0][c] = fadd(qlb[c], -dqb, F);
        qb[1][c] = fadd(qrb[c], dqb, F);
    }
    // pressures: hl from (p1 - p0, p2 - p1), hr from (p2 - p1, p3 - p2)
#pragma unroll
    for (int m = 0; m < 4; ++m)
        pb[m] = 0.0;
    const double a1 = fmul(hlb, dl_dm, F), a2 = fmul(hlb, dl_dp, F);
    pb[1] = fadd(pb[1], a1, F);
    pb[0] = fadd(pb[0], -a1, F);
    pb[2] = fadd(pb[2], a2, F);
    pb[1] = fadd(pb[1], -a2, F);
    const double b1 = fmul(hrb, dr_dm, F), b2 = fmul(hrb, dr_dp, F);
    pb[2] = fadd(pb[2], b1, F);
    pb[1] = fadd(pb[1], -b1, F);
    pb[3] = fadd(pb[3], b2, F);
    pb[2] = fadd(pb[2], -b2, F);
}

// Per cell: cp[0..3][cell] = pressure, 1/rho, u, v (the arithmetic of
// cell_pressure, whose sum of momentum terms is symmetric in x and y).
__global__ void __launch_bounds__(kThreads) k_vjp_cells(const __grid_constant__ Params p, const double *q, double *cp)
{
    const int64_t plane = p.nx * p.ny;
    const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= plane)
        return;
    const Fx &F = p.ek.f;
    const double rho = q[cell], mx = q[plane + cell], my = q[2 * plane + cell];
    const double E = q[3 * plane + cell];
    const double inv = __drcp_rn(rho);
    const double u = fmul(mx, inv, F), v = fmul(my, inv, F);
    const double ke2 = fadd(fmul(mx, u, F), fmul(my, v, F), F);
    cp[cell] = fmul(p.ek.gm1, __fma_rn(-0.5, ke2, E), F);
    cp[plane + cell] = inv;
    cp[2 * plane + cell] = u;
    cp[3 * plane + cell] = v;
}

// Per cell and axis: lp[(axis*6 + t)*plane + cell] = h+, dh+/ddm, dh+/ddp,
// h-, dh-/ddm, dh-/ddp of the cell's half limiter factors, from
// dm = P_i - P_{i-1} and dp = P_{i+1} - P_i along the axis.
__global__ void __launch_bounds__(kThreads) k_vjp_limiters(const __grid_constant__ Params p, const double *cp, double *lp)
{
    const int64_t plane = p.nx * p.ny;
    const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= plane)
        return;
    const Fx &F = p.ek.f;
    const int64_t i = cell % p.nx, j = cell / p.nx;
    const int64_t im = i == 0 ? p.nx - 1 : i - 1, ip = i == p.nx - 1 ? 0 : i + 1;
    const int64_t jm = j == 0 ? p.ny - 1 : j - 1, jp = j == p.ny - 1 ? 0 : j + 1;
    const double pc = cp[cell];
    const double nb[2][2] = {{cp[j * p.nx + im], cp[j * p.nx + ip]},
                             {cp[jm * p.nx + i], cp[jp * p.nx + i]}};
#pragma unroll
    for (int axis = 0; axis < 2; ++axis) {
        double hp, hm, dp_dm, dp_dp, dm_dm, dm_dp;
        limiter_halves_grad(fadd(pc, -nb[axis][0], F), fadd(nb[axis][1], -pc, F), p.literal, F,
                            hp, hm, dp_dm, dp_dp, dm_dm, dm_dp);
        double *o = lp + (int64_t)axis * 6 * plane + cell;
        o[0] = hp;
        o[plane] = dp_dm;
        o[2 * plane] = dp_dp;
        o[3 * plane] = hm;
        o[4 * plane] = dm_dm;
        o[5 * plane] = dm_dp;
    }
}

// Per face (axis 0: between (i,j) and (i+1,j); axis 1: between (i,j) and
// (i,j+1)): the contributions of <v_right - v_left, Fh(Q)>.  Layout
// fo[(axis*12 + t) * plane + j*nx + i]: t = 0..3 the gradient for the
// face's left cell (cell 1 of its line), t = 4..7 for its right cell (cell
// 2), components in the (rho, m_x, m_y, E) order; t = 8..11 the pressure
// adjoints of cells 0..3 of its line (offsets -1..2 along the axis).
// lp: k_vjp_limiters of q.  128-thread CTAs held to 128 registers: four
// CTAs (16 warps) per SM to hide the long divide and square-root chains.
#ifndef SWEEP_VJP_THREADS
#define SWEEP_VJP_THREADS 128
#endif
constexpr int kVjpThreads = SWEEP_VJP_THREADS;
constexpr int kFacePlanes = 12;  // per axis
__global__ void __launch_bounds__(kVjpThreads, 512 / kVjpThreads)
    k_face_vjp(const __grid_constant__ Params p, const double *q, const double *lp, const double *v, double *fo)
{
    const int64_t plane = p.nx * p.ny;
    const Fx F = p.ek.f;
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= 2 * plane)
        return;
    const int axis = (int)(f / plane);
    const int64_t cell = f - axis * plane;
    const int64_t i = cell % p.nx, j = cell / p.nx;
    // normal-frame component order: (rho, m_n, m_t, E)
    const int c1 = axis == 0 ? 1 : 2, c2 = axis == 0 ? 2 : 1;
    // cells 1 and 2 of the line: this cell and its + neighbour
    int64_t right;
    if (axis == 0)
        right = j * p.nx + (i + 1 == p.nx ? 0 : i + 1);
    else
        right = (j + 1 == p.ny ? 0 : j + 1) * p.nx + i;
    const double q1[4] = {q[cell], q[c1 * plane + cell], q[c2 * plane + cell], q[3 * plane + cell]};
    const double q2[4] = {q[right], q[c1 * plane + right], q[c2 * plane + right],
                          q[3 * plane + right]};
    const double *L = lp + (int64_t)axis * 6 * plane;
    const double lim1[3] = {L[cell], L[plane + cell], L[2 * plane + cell]};
    const double lim2[3] = {L[3 * plane + right], L[4 * plane + right], L[5 * plane + right]};
    const double a[4] = {fadd(v[right], -v[cell], F),
                         fadd(v[c1 * plane + right], -v[c1 * plane + cell], F),
                         fadd(v[c2 * plane + right], -v[c2 * plane + cell], F),
                         fadd(v[3 * plane + right], -v[3 * plane + cell], F)};
    double qb[2][4], pb[4];
    face_flux_vjp(q1, q2, lim1, lim2, a, p.ek, qb, pb);
    double *o = fo + (int64_t)axis * kFacePlanes * plane + cell;
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        o[(m * 4 + 0) * plane] = qb[m][0];
        o[(m * 4 + c1) * plane] = qb[m][1];
        o[(m * 4 + c2) * plane] = qb[m][2];
        o[(m * 4 + 3) * plane] = qb[m][3];
    }
#pragma unroll
    for (int m = 0; m < 4; ++m)
        o[(8 + m) * plane] = pb[m];
}

// Per cell: S = J^T v at the cell.  The face at index e along an axis
// reaches this cell as cell m of its line, e = pos + 1 - m (wrapped); the
// faces are summed in increasing e, x faces then y faces: the gradients
// through the reconstructed states (m = 1, 2) into S, the pressure adjoints
// (m = 0..3) into pb; then S takes the reverse of the cell's pressure for
// pb (q, cp: the state and its k_vjp_cells terms), and
//   mode 0:  mu = lam2 S                 (mu: out)
//   mode 1:  lam = (lam + mu) + lam1 S   (lam: in place)
__global__ void __launch_bounds__(kThreads) k_gather(const __grid_constant__ Params p, const double *fo, const double *q,
                                                     const double *cp, double *lam, double *mu,
                                                     int mode)
{
    const int64_t plane = p.nx * p.ny;
    const Fx F = p.ek.f;
    const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= plane)
        return;
    const int64_t i = cell % p.nx, j = cell / p.nx;
    int64_t ex[4], ey[4];
    int mx[4], my[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        int64_t e = i + 1 - m;
        ex[m] = e < 0 ? e + p.nx : (e >= p.nx ? e - p.nx : e);
        e = j + 1 - m;
        ey[m] = e < 0 ? e + p.ny : (e >= p.ny ? e - p.ny : e);
        mx[m] = m;
        my[m] = m;
    }
    // sort the four (e, m) pairs by e (insertion sort of four)
#pragma unroll
    for (int s = 1; s < 4; ++s)
        for (int t = s; t > 0 && ex[t - 1] > ex[t]; --t) {
            const int64_t te = ex[t];
            ex[t] = ex[t - 1];
            ex[t - 1] = te;
            const int tm = mx[t];
            mx[t] = mx[t - 1];
            mx[t - 1] = tm;
        }
#pragma unroll
    for (int s = 1; s < 4; ++s)
        for (int t = s; t > 0 && ey[t - 1] > ey[t]; --t) {
            const int64_t te = ey[t];
            ey[t] = ey[t - 1];
            ey[t - 1] = te;
            const int tm = my[t];
            my[t] = my[t - 1];
            my[t - 1] = tm;
        }
    const double *fx = fo, *fy = fo + (int64_t)kFacePlanes * plane;
    double S[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        double s = 0.0;
#pragma unroll
        for (int t = 0; t < 4; ++t)
            if (mx[t] == 1 || mx[t] == 2)
                s = fadd(s, fx[(int64_t)((mx[t] - 1) * 4 + c) * plane + j * p.nx + ex[t]], F);
#pragma unroll
        for (int t = 0; t < 4; ++t)
            if (my[t] == 1 || my[t] == 2)
                s = fadd(s, fy[(int64_t)((my[t] - 1) * 4 + c) * plane + ey[t] * p.nx + i], F);
        S[c] = s;
    }
    double pb = 0.0;
#pragma unroll
    for (int t = 0; t < 4; ++t)
        pb = fadd(pb, fx[(int64_t)(8 + mx[t]) * plane + j * p.nx + ex[t]], F);
#pragma unroll
    for (int t = 0; t < 4; ++t)
        pb = fadd(pb, fy[(int64_t)(8 + my[t]) * plane + ey[t] * p.nx + i], F);
    cell_pressure_vjp(q[plane + cell], q[2 * plane + cell], cp[plane + cell], cp[2 * plane + cell],
                      cp[3 * plane + cell], p.ek, pb, S);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int64_t o = c * plane + cell;
        if (mode == 0)
            mu[o] = fmul(p.c2, S[c], F);
        else
            lam[o] = fadd(fadd(lam[o], mu[o], F), fmul(p.c1, S[c], F), F);
    }
}

}  // namespace sweep
