// numerics.cuh -- pointwise stage updates of the two problems, FP64.
//
// Every operation is an explicit round-to-nearest intrinsic (__fma_rn,
// __ddiv_rn, __drcp_rn, __dsqrt_rn) so that the compiler cannot fuse or
// reorder anything; the library is also built with -fmad=false.  Sums and
// products are issued as fused multiply-adds with an exact unit operand:
//   a + b = fma(1, a, b)     a b = fma(a, b, -0)
// hold bit for bit for all inputs (the one rounding of the fma is the
// rounding of the sum or product; -0 is the additive identity that keeps the
// sign of a zero product).  On B300 an FP64 add or multiply issues at 0.84
// of the fma rate (471 vs 559 G lane-ops/s measured), so the fused form is
// faster.  1 and -0 come in as kernel arguments (Fx), which keeps the
// compiler from folding the fma back into an add or a multiply.
// The rounding order is the one the method's arithmetic specification pins
// (the paper gives none), so that the Swept and Standard kernels -- which
// both call these functions -- agree bit for bit, and agree with any other
// implementation of the same specification.
#pragma once

#include <cstdint>

namespace sweep {

struct Fx {
    double one;    // 1.0
    double nzero;  // -0.0
};
__device__ __forceinline__ double fadd(double a, double b, const Fx &f) { return __fma_rn(f.one, a, b); }
__device__ __forceinline__ double fmul(double a, double b, const Fx &f) { return __fma_rn(a, b, f.nzero); }

// ---------------------------------------------------------------- heat, App. A
// t = fma(-4, T, (T_W + T_E) + (T_S + T_N));  T' = fma(c, t, T_own)
// with c = r/2 for the first RK2 stage and r for the second (App. A update
// with r_x = r_y = r, taken as a midpoint rule).
__device__ __forceinline__ double heat_update(double uc, double uw, double ue, double us,
                                              double un, double own, double c, const Fx &f)
{
    const double s = fadd(fadd(uw, ue, f), fadd(us, un, f), f);
    const double t = __fma_rn(-4.0, uc, s);
    return __fma_rn(c, t, own);
}

// ---------------------------------------------------------------- Euler, App. B
struct EulerConst {
    double gamma;  // ratio of specific heats
    double gm1;    // gamma - 1 (rounded once, on the host)
    Fx f;          // the unit operands of fadd / fmul
};

// Cell pressure for the limiter, symmetric in x and y:
// inv = 1/rho, u = m_x inv, v = m_y inv, p = (gamma-1) fma(-1/2, m_x u + m_y v, E)
__device__ __forceinline__ double cell_pressure(double rho, double mx, double my, double E,
                                                const EulerConst &k)
{
    const Fx &f = k.f;
    const double inv = __drcp_rn(rho);  // correctly rounded, equal to 1.0 / rho
    const double u = fmul(mx, inv, f);
    const double v = fmul(my, inv, f);
    const double ke2 = fadd(fmul(mx, u, f), fmul(my, v, f), f);
    return fmul(k.gm1, __fma_rn(-0.5, ke2, E), f);
}

// Half limiter factors of one cell along one axis from dm = P_i - P_{i-1} and
// dp = P_{i+1} - P_i: hp = phi_plus/2 (towards the + face), hm = phi_minus/2.
// phi_plus = min(dm/dp, 1), phi_minus = min(dp/dm, 1) where both differences
// are nonzero with equal signs, else 0 (pressure-ratio minmod, App. B).
// One division suffices: when |dm| < |dp| the exact dm/dp is below 1, so its
// rounding is <= 1 and min() keeps it, while dp/dm > 1 rounds to >= 1 and
// min() gives 1; symmetrically otherwise.  The sign and magnitude tests are
// integer operations on the bit patterns, which keeps them off the FP64 pipe.
// mode 1 swaps the two factors (the orientation printed in App. B); mode 2
// applies no limiting (both factors 1: the face value is the two cells'
// average), which is not a scheme of the paper and serves to check the
// adjoint against finite differences where the scheme is smooth.
__device__ __forceinline__ void limiter_halves(double dm, double dp, int literal, const Fx &f,
                                               double &hp, double &hm)
{
    if (literal == 2) {
        hp = 0.5;
        hm = 0.5;
        return;
    }
    const unsigned long long bm = (unsigned long long)__double_as_longlong(dm);
    const unsigned long long bp = (unsigned long long)__double_as_longlong(dp);
    const unsigned long long am = bm & 0x7fffffffffffffffull;
    const unsigned long long ap = bp & 0x7fffffffffffffffull;
    const bool same = ((bm ^ bp) >> 63) == 0 && am != 0 && ap != 0;
    const bool mlt = am < ap;  // |dm| < |dp|
    // Where the factors are 0 the quotient is unused; dividing 1 by 1 there
    // keeps the division on its fast path (a zero divisor would send the
    // lane, and with it the warp, through the special-case path).
    const double q = __ddiv_rn(same ? (mlt ? dm : dp) : 1.0, same ? (mlt ? dp : dm) : 1.0);
    const double hq = fmul(0.5, q, f);
    double plus = mlt ? hq : 0.5;
    double minus = mlt ? 0.5 : hq;
    if (!same) {
        plus = 0.0;
        minus = 0.0;
    }
    if (literal) {
        hp = minus;
        hm = plus;
    } else {
        hp = plus;
        hm = minus;
    }
}

// Flux of one reconstructed state in the face-normal frame (rho, m_n, m_t, E):
// inv = 1/rho, u_n = m_n inv, u_t = m_t inv,
// p = (gamma-1) fma(-1/2, fma(m_n, u_n, m_t u_t), E), c = sqrt((gamma p) inv),
// f = (m_n, fma(m_n, u_n, p), m_t u_n, (E + p) u_n), lam = |u_n| + c.
// The intermediate values of one state flux (a reverse pass reuses them).
struct FluxParts {
    double inv, un, ut, p, c;
};

__device__ __forceinline__ void state_flux(double rho, double mn, double mt, double E,
                                           const EulerConst &k, double f[4], double &lam,
                                           FluxParts &s)
{
    const Fx &x = k.f;
    s.inv = __drcp_rn(rho);  // correctly rounded, equal to 1.0 / rho
    s.un = fmul(mn, s.inv, x);
    s.ut = fmul(mt, s.inv, x);
    const double ke2 = __fma_rn(mn, s.un, fmul(mt, s.ut, x));
    s.p = fmul(k.gm1, __fma_rn(-0.5, ke2, E), x);
    s.c = __dsqrt_rn(fmul(fmul(k.gamma, s.p, x), s.inv, x));
    f[0] = mn;
    f[1] = __fma_rn(mn, s.un, s.p);
    f[2] = fmul(mt, s.un, x);
    f[3] = fmul(fadd(E, s.p, x), s.un, x);
    lam = fadd(fabs(s.un), s.c, x);
}

__device__ __forceinline__ void state_flux(double rho, double mn, double mt, double E,
                                           const EulerConst &k, double f[4], double &lam)
{
    FluxParts s;
    state_flux(rho, mn, mt, E, k, f, lam, s);
}

// larger of two non-negative, non-NaN doubles by their bit patterns (integer
// compare, same result as the floating-point max for such values)
__device__ __forceinline__ double max_nonneg(double a, double b)
{
    return __double_as_longlong(a) > __double_as_longlong(b) ? a : b;
}

// Rusanov-form numerical flux (App. B) at the face between cells "0" and "1",
// states in the face-normal frame, hl = phi_plus(0)/2, hr = phi_minus(1)/2:
//   Q_L = fma(hl, Q1 - Q0, Q0),  Q_R = fma(-hr, Q1 - Q0, Q1)
//   Fh = 1/2 fma(r, Q_L - Q_R, F(Q_L) + F(Q_R)),  r = max(lam_L, lam_R)
__device__ __forceinline__ void face_flux(const double q0[4], const double q1[4], double hl,
                                          double hr, const EulerConst &k, double fh[4])
{
    const Fx &x = k.f;
    double ql[4], qr[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const double dq = fadd(q1[c], -q0[c], x);
        ql[c] = __fma_rn(hl, dq, q0[c]);
        qr[c] = __fma_rn(-hr, dq, q1[c]);
    }
    double fl[4], fr[4], laml, lamr;
    state_flux(ql[0], ql[1], ql[2], ql[3], k, fl, laml);
    state_flux(qr[0], qr[1], qr[2], qr[3], k, fr, lamr);
    const double r = max_nonneg(laml, lamr);
#pragma unroll
    for (int c = 0; c < 4; ++c)
        fh[c] = fmul(0.5, __fma_rn(r, fadd(ql[c], -qr[c], x), fadd(fl[c], fr[c], x)), x);
}

// face_flux taken by the two lanes of a pair (lanes 2k and 2k+1 of a warp,
// side = lane & 1): side 0 reconstructs Q_L and returns components 0 and 1
// of Fh in fa, fb; side 1 reconstructs Q_R and returns components 2 and 3.
// Each lane computes one state flux and hands its partner, by shuffle, the
// state and flux components the partner returns; every component takes
// face_flux's operations in face_flux's order, so the bits are the same.
// mask: the lanes taking part (both lanes of every pair).
__device__ __forceinline__ void face_flux_half(const double q0[4], const double q1[4], double hl,
                                               double hr, int side, unsigned mask,
                                               const EulerConst &k, double &fa, double &fb)
{
    const Fx &x = k.f;
    const double h = side ? -hr : hl;
    double st[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const double dq = fadd(q1[c], -q0[c], x);
        st[c] = __fma_rn(h, dq, side ? q1[c] : q0[c]);
    }
    double f[4], lam;
    state_flux(st[0], st[1], st[2], st[3], k, f, lam);
    // the partner's state and flux for the two components this lane returns
    const double pq0 = __shfl_xor_sync(mask, side ? st[0] : st[2], 1);
    const double pq1 = __shfl_xor_sync(mask, side ? st[1] : st[3], 1);
    const double pf0 = __shfl_xor_sync(mask, side ? f[0] : f[2], 1);
    const double pf1 = __shfl_xor_sync(mask, side ? f[1] : f[3], 1);
    const double plam = __shfl_xor_sync(mask, lam, 1);
    const double r = side ? max_nonneg(plam, lam) : max_nonneg(lam, plam);
    const double m0 = side ? st[2] : st[0], m1 = side ? st[3] : st[1];
    const double g0 = side ? f[2] : f[0], g1 = side ? f[3] : f[1];
    const double ql0 = side ? pq0 : m0, qr0 = side ? m0 : pq0;
    const double ql1 = side ? pq1 : m1, qr1 = side ? m1 : pq1;
    const double fl0 = side ? pf0 : g0, fr0 = side ? g0 : pf0;
    const double fl1 = side ? pf1 : g1, fr1 = side ? g1 : pf1;
    fa = fmul(0.5, __fma_rn(r, fadd(ql0, -qr0, x), fadd(fl0, fr0, x)), x);
    fb = fmul(0.5, __fma_rn(r, fadd(ql1, -qr1, x), fadd(fl1, fr1, x)), x);
}

// out = fma(lam, (Fh_{i-1/2} - Fh_{i+1/2}) + (Gh_{j-1/2} - Gh_{j+1/2}), own)
__device__ __forceinline__ double euler_combine(double fm, double fp, double gm, double gp,
                                                double own, double lam, const Fx &f)
{
    const double d = fadd(fadd(fm, -fp, f), fadd(gm, -gp, f), f);
    return __fma_rn(lam, d, own);
}

}  // namespace sweep
