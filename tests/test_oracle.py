"""Pins for the CPU oracle (no GPU).

Each test ties the oracle to something other than itself: a closed form,
an invariant, a special case whose value is known by hand, a convergence
rate, or a brute-force replay.  The choice is made so that a plausible slip
(a dropped term, a wrong sign, index or coefficient, a transposed operand)
fails at least one of them.
"""
import math

import numpy as np
import pytest

from paper_2105_10332_b300 import workloads as W

EPS = np.finfo(np.float64).eps


# ---------------------------------------------------------------- heat (App. A)

def heat_growth(kx, ky, nx, ny, r, scheme):
    """Amplification of one periodic mode: lambda = -4(sin^2(pi kx/nx) + sin^2(pi ky/ny)),
    z = r lambda; RK2 midpoint G = 1 + z + z^2/2, forward Euler G = 1 + z."""
    lam = -4.0 * (math.sin(math.pi * kx / nx) ** 2 + math.sin(math.pi * ky / ny) ** 2)
    z = r * lam
    return 1.0 + z + 0.5 * z * z if scheme == 0 else 1.0 + z


def heat_run_r(oracle_lib, u0, r, nsteps, scheme=0):
    """Heat run at mesh ratio r: dx = 1/nx and dt = r dx^2 (alpha = 1) handed to
    the oracle, which forms r = alpha dt / dx^2 itself."""
    dt, dx = W.heat_dt(u0.shape[-1], r)
    return oracle_lib.heat_run(u0, nsteps, dt, dx, scheme=scheme)


def test_heat_r_is_alpha_dt_over_dx_squared(oracle_lib):
    """App. A: r = alpha dt / dx^2.  The oracle's value against exact rational
    arithmetic (a dropped alpha, dx in place of dx^2 or an inverted ratio fails)."""
    from fractions import Fraction
    rng = np.random.default_rng(17)
    for _ in range(500):
        alpha = float(rng.uniform(0.1, 3.0))
        dx = 1.0 / int(rng.integers(8, 20000))
        dt = float(rng.uniform(0.01, 0.3)) * dx * dx / alpha
        exact = Fraction(alpha) * Fraction(dt) / (Fraction(dx) * Fraction(dx))
        got = oracle_lib.heat_r(dt, dx, alpha)
        assert abs(Fraction(got) - exact) <= 2 * EPS * exact
    # powers of two make every step exact: r = 0.1 at 64^2 comes back as the double 0.1
    dt, dx = W.heat_dt(64, 0.1)
    assert oracle_lib.heat_r(dt, dx) == 0.1 and dt == 0.1 / 4096
    assert oracle_lib.heat_r(dt, dx, 2.0) == 0.2


def test_heat_closed_form_sine_64(oracle_lib):
    """Heat 64^2, r = 0.1, 500 RK2 steps of T0 = sin 2pi x sin 2pi y (App. A)."""
    u0 = W.heat_sine(64, 64)
    u = heat_run_r(oracle_lib, u0, 0.1, 500)
    G = heat_growth(1, 1, 64, 64, 0.1, 0)
    assert abs(G ** 500 - 0.38172528846400894) < 1e-15
    err = np.max(np.abs(u - G ** 500 * u0)) / np.max(np.abs(u0))
    assert err <= 1e-13, err


@pytest.mark.parametrize("scheme", [0, 1])
def test_heat_closed_form_modes(oracle_lib, scheme):
    """Seeded sum of 8 modes on a non-square grid: each mode decays by its own G^N."""
    nx, ny, r, N = 48, 40, 0.1, 200
    x, y = W.heat_grid(nx, ny)
    u0 = np.zeros((ny, nx))
    expect = np.zeros((ny, nx))
    for a, kx, ky, phx, phy in W.heat_modes_spec(seed=7, nmodes=8, kmax=16):
        mode = np.outer(np.sin(2 * math.pi * ky * y + phy), np.sin(2 * math.pi * kx * x + phx))
        u0 += a * mode
        expect += a * heat_growth(kx, ky, nx, ny, r, scheme) ** N * mode
    u = heat_run_r(oracle_lib, u0, r, N, scheme=scheme)
    err = np.max(np.abs(u - expect)) / np.max(np.abs(u0))
    assert err <= 1e-13, err


def test_heat_vs_analytic(oracle_lib):
    """App. A analytic solution T0 exp(-8 pi^2 alpha t); the gap, relative to the
    decayed amplitude, is the O(dx^2) truncation error of the 5-point Laplacian,
    predicted (pi/64)^2/3 * 8 pi^2 t = 7.75e-4."""
    nx, r, N = 64, 0.1, 500
    dt, dx = W.heat_dt(nx, r)
    t = N * dt
    assert t == 0.01220703125
    u0 = W.heat_sine(nx, nx)
    u = oracle_lib.heat_run(u0, N, dt, dx)
    decay = math.exp(-8 * math.pi ** 2 * t)
    gap = np.max(np.abs(u - decay * u0)) / (decay * np.max(np.abs(u0)))
    predicted = (math.pi / nx) ** 2 / 3 * 8 * math.pi ** 2 * t
    assert 1e-4 < gap <= 1e-3
    assert abs(gap - predicted) / predicted < 0.01


def test_heat_conservation(oracle_lib):
    u0 = W.heat_modes(40, 36, seed=3) + 0.25
    N = 300
    u = heat_run_r(oracle_lib, u0, 0.1, N)
    drift = abs(math.fsum(u.ravel()) - math.fsum(u0.ravel()))
    assert drift <= 64 * EPS * N * math.fsum(np.abs(u0).ravel())


def test_heat_transpose_and_constant(oracle_lib):
    rng = np.random.default_rng(11)
    u0 = rng.standard_normal((24, 36))
    dt, dx = W.heat_dt(36, 0.1)
    a = oracle_lib.heat_run(u0, 17, dt, dx)
    b = oracle_lib.heat_run(np.ascontiguousarray(u0.T), 17, dt, dx)
    assert np.array_equal(a.T, b)
    c = np.full((20, 20), 0.7135)
    assert np.array_equal(heat_run_r(oracle_lib, c, 0.1, 25), c)


def test_heat_brute_force_single_point(oracle_lib):
    """A delta on a tiny grid spreads by the 5-point stencil: after one forward
    Euler step the centre holds 1 - 4r and each neighbour r (exact in binary for r = 1/8)."""
    u0 = np.zeros((8, 8))
    u0[3, 4] = 1.0
    u = heat_run_r(oracle_lib, u0, 0.125, 1, scheme=1)
    expect = np.zeros((8, 8))
    expect[3, 4] = 0.5
    for j, i in ((2, 4), (4, 4), (3, 3), (3, 5)):
        expect[j, i] = 0.125
    assert np.array_equal(u, expect)
    # RK2 midpoint: one step is u + r L u + (r^2/2) L^2 u; L^2 of a delta has
    # centre 20, ring-1 -8, diagonals 2, ring-2 1.
    u = heat_run_r(oracle_lib, u0, 0.125, 1, scheme=0)
    r = 0.125
    L2 = np.zeros((8, 8))
    L2[3, 4] = 20
    for j, i in ((2, 4), (4, 4), (3, 3), (3, 5)):
        L2[j, i] = -8
    for j, i in ((2, 3), (2, 5), (4, 3), (4, 5)):
        L2[j, i] = 2
    for j, i in ((1, 4), (5, 4), (3, 2), (3, 6)):
        L2[j, i] = 1
    expect2 = expect + 0.5 * r * r * L2
    assert np.max(np.abs(u - expect2)) <= 4 * EPS


# ---------------------------------------------------------------- Euler (App. B)

GAMMA = 1.4


def conserved(rho, u, v, p, gamma=GAMMA):
    return np.array([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


def test_state_flux_hand_values(oracle_lib):
    """Physical flux F = (rho u, rho u^2 + p, rho u v, (E + p) u) and |u| + c."""
    q = conserved(2.0, 2.0, 1.0, 3.0)
    f, lam = oracle_lib.state_flux(q)
    expect = np.array([4.0, 11.0, 4.0, (q[3] + 3.0) * 2.0])
    assert np.max(np.abs(f - expect) / np.abs(expect)) <= 8 * EPS
    assert abs(lam - (2.0 + math.sqrt(1.4 * 3.0 / 2.0))) <= 8 * EPS * lam
    # at rest: only the pressure term survives
    f, lam = oracle_lib.state_flux(np.array([1.0, 0.0, 0.0, 2.5]))
    assert f[0] == 0.0 and f[2] == 0.0 and f[3] == 0.0
    assert abs(f[1] - 1.0) <= 4 * EPS and abs(lam - math.sqrt(1.4)) <= 4 * EPS


def test_flux_consistency(oracle_lib):
    """Fh(Q, Q) = F(Q) bitwise (no jump, no dissipation, the limiter sees dP = 0)."""
    rng = np.random.default_rng(5)
    for _ in range(50):
        q = conserved(rng.uniform(0.2, 3), rng.normal(), rng.normal(), rng.uniform(0.2, 3))
        f, _ = oracle_lib.state_flux(q)
        for lim in (0, 1, 2):
            assert np.array_equal(oracle_lib.face_flux(q, q, q, q, limiter=lim), f)


def test_rusanov_sod_states(oracle_lib):
    """Two constant states (Sod's): the limiter gives phi = 0 on both sides, so
    Fh = 1/2 (F(QA) + F(QB) + r (QA - QB)), r = max(|u| + c) = sqrt(1.4)."""
    qa = np.array([1.0, 0.0, 0.0, 2.5])      # p = 1
    qb = np.array([0.125, 0.0, 0.0, 0.25])   # p = 0.1
    fh = oracle_lib.face_flux(qa, qa, qb, qb)
    s = math.sqrt(1.4)
    expect = np.array([0.5 * s * 0.875, 0.5 * 1.1, 0.0, 0.5 * s * 2.25])
    assert fh[2] == 0.0
    assert np.max(np.abs(fh - expect)) <= 16 * EPS


def test_cell_pressure_from_primitives(oracle_lib):
    """The limiter's pressure is the App. B EOS p = (gamma-1)(E - rho(u^2+v^2)/2)
    of the conserved state: states built from primitives give their p back.
    A wrong kinetic term (E - rho|u|^2, or E alone) or a wrong factor fails."""
    q = np.array([2.0, 3.0, -1.0, 10.0])  # rho 2, u 1.5, v -0.5: E - KE = 7.5 exactly
    assert abs(oracle_lib.cell_pressure(q) - 0.4 * 7.5) <= 4 * EPS * 3.0
    rng = np.random.default_rng(23)
    for _ in range(200):
        rho, p = rng.uniform(0.3, 3.0, 2)
        u, v = rng.uniform(-1.5, 1.5, 2)
        q = conserved(rho, u, v, p)
        assert abs(oracle_lib.cell_pressure(q) - p) <= 64 * EPS * (p + 0.5 * rho * (u * u + v * v))
    # symmetric in x and y
    q = conserved(1.3, 0.9, -0.2, 1.7)
    assert oracle_lib.cell_pressure(q) == oracle_lib.cell_pressure(q[[0, 2, 1, 3]])


def rusanov_by_hand(qa, qb, gamma=GAMMA):
    """1/2 (F(QL) + F(QR) + max(|u_n|+c) (QL - QR)) from primitives, in numpy."""
    out = []
    for q in (qa, qb):
        rho, mn, mt, E = q
        un, ut = mn / rho, mt / rho
        p = (gamma - 1.0) * (E - 0.5 * rho * (un * un + ut * ut))
        c = math.sqrt(gamma * p / rho)
        out.append((np.array([mn, mn * un + p, mt * un, (E + p) * un]), abs(un) + c))
    (fa, la), (fb, lb) = out
    return 0.5 * (fa + fb + max(la, lb) * (qa - qb))


def test_face_flux_limiter_sees_cell_pressures(oracle_lib):
    """Four cells of a line with pressures 1, 2, 4, 5 and different velocities:
    theta = dm/dp = 1/2 on cell 0 towards its + face and dp/dm = 1/2 on cell 1
    towards its - face, so Q_L = Q_0 + (Q_1 - Q_0)/4 and Q_R = Q_1 - (Q_1 - Q_0)/4
    (App. B reconstruction with phi/2 = 1/4), and the face flux is the Rusanov
    flux of those two states.  The limiter takes its pressures from the
    conserved states, so a wrong kinetic-energy term moves theta and fails here."""
    prims = [(1.0, 0.5, 0.25, 1.0), (1.25, 0.75, -0.5, 2.0), (0.8, 1.0, 0.5, 4.0),
             (1.1, 0.25, 0.0, 5.0)]
    qs = [conserved(*pr) for pr in prims]
    for lim in (0, 1):
        # the printed orientation (1) takes dp/dm on cell 0 and dm/dp on cell 1: both 2 -> 1
        h = 0.25 if lim == 0 else 0.5
        ql = qs[1] + h * (qs[2] - qs[1])
        qr = qs[2] - h * (qs[2] - qs[1])
        got = oracle_lib.face_flux(*qs, limiter=lim)
        exp = rusanov_by_hand(ql, qr)
        assert np.max(np.abs(got - exp)) <= 1e-13 * np.max(np.abs(exp)), (lim, got, exp)
    # the same line with the kinetic term doubled in the limiter's pressure would
    # give theta = 0.429 on cell 0; the resulting flux differs at the 1e-3 level
    k = [0.5 * r * (u * u + v * v) for r, u, v, _ in prims]
    pw = [p - 0.4 * kk for (_, _, _, p), kk in zip(prims, k)]
    th = (pw[1] - pw[0]) / (pw[2] - pw[1])
    wrong = rusanov_by_hand(qs[1] + 0.5 * th * (qs[2] - qs[1]),
                            qs[2] - 0.5 * min((pw[3] - pw[2]) / (pw[2] - pw[1]), 1.0) * (qs[2] - qs[1]))
    assert np.max(np.abs(wrong - oracle_lib.face_flux(*qs))) > 1e-4


def minmod(a, b):
    if a * b <= 0:
        return 0.0
    return a if abs(a) < abs(b) else b


def test_limiter_is_textbook_minmod(oracle_lib):
    """phi_plus * dP+ = minmod(dP-, dP+) and phi_minus * dP- = minmod(dP-, dP+)."""
    rng = np.random.default_rng(9)
    for _ in range(2000):
        dm, dp = rng.normal(size=2) * 10.0 ** rng.integers(-6, 6, size=2)
        pp, pm = oracle_lib.limiter(dm, dp, 0)
        mm = minmod(dm, dp)
        assert abs(pp * dp - mm) <= 2 * EPS * abs(mm)
        assert abs(pm * dm - mm) <= 2 * EPS * abs(mm)
        assert 0.0 <= pp <= 1.0 and 0.0 <= pm <= 1.0
        lp, lm = oracle_lib.limiter(dm, dp, 1)
        assert (lp, lm) == (pm, pp)  # the printed orientation swaps the two
        assert oracle_lib.limiter(dm, dp, 2) == (1.0, 1.0)
    for dm, dp in ((0.0, 1.0), (1.0, 0.0), (0.0, 0.0), (1.0, -2.0), (-3.0, 0.5)):
        assert oracle_lib.limiter(dm, dp, 0) == (0.0, 0.0)
    assert oracle_lib.limiter(2.5, 2.5, 0) == (1.0, 1.0)
    assert oracle_lib.limiter(-1e-300, -1e300, 0)[1] == 1.0


def test_euler_constant_state(oracle_lib):
    q0 = np.ascontiguousarray(np.broadcast_to(conserved(1.3, 0.7, -0.4, 2.1)[:, None, None],
                                              (4, 12, 16)))
    q = oracle_lib.euler_run(q0, 0.01, 0.1, 10)
    assert np.array_equal(q, q0)


def test_euler_conservation(oracle_lib):
    q0, dx = W.vortex(32)
    dt, _ = W.vortex_dt(q0, dx, 1.0)
    N = 60
    q = oracle_lib.euler_run(q0, dt, dx, N)
    for k in range(4):
        drift = abs(math.fsum(q[k].ravel()) - math.fsum(q0[k].ravel()))
        assert drift <= 64 * EPS * N * math.fsum(np.abs(q0[k]).ravel()), (k, drift)


def swap_xy(q):
    return np.ascontiguousarray(np.stack([q[0].T, q[2].T, q[1].T, q[3].T]))


def test_euler_transpose_symmetry(oracle_lib):
    """Swapping x with y (and rho u with rho v) commutes with the scheme, bitwise."""
    q0, dx = W.vortex(32, 24, xc=0.7, yc=-1.1)
    q0[1] *= 1.3  # break the u = v symmetry of the free stream
    dt, _ = W.vortex_dt(q0, dx, 1.0)
    a = oracle_lib.euler_run(q0, dt, dx, 12)
    b = oracle_lib.euler_run(swap_xy(q0), dt, dx, 12)
    assert np.array_equal(swap_xy(a), b)


def test_euler_1d_reduction(oracle_lib):
    """A field varying in x only stays uniform in y and keeps rho v = 0 exactly."""
    nx, ny = 40, 8
    x = (np.arange(nx) + 0.5) / nx
    rho = 1.0 + 0.2 * np.sin(2 * math.pi * x)
    p = 1.0 + 0.1 * np.cos(2 * math.pi * x)
    u = 0.5 + 0.1 * np.sin(4 * math.pi * x)
    q1 = conserved(rho, u, 0.0 * u, p)
    q0 = np.ascontiguousarray(np.repeat(q1[:, None, :], ny, axis=1))
    q = oracle_lib.euler_run(q0, 0.002, 1.0 / nx, 30)
    assert np.all(q[2] == 0.0)
    assert np.all(q == q[:, :1, :])
    assert not np.array_equal(q, q0)


def vortex_l1_errors(oracle_lib, limiter, sizes=(32, 64, 128), T=1.0):
    errs = []
    for nx in sizes:
        q0, dx = W.vortex(nx)
        dt, N = W.vortex_dt(q0, dx, T)
        q = oracle_lib.euler_run(q0, dt, dx, N, limiter=limiter)
        ex, _ = W.vortex(nx, xc=T, yc=T)  # exact: translation by (u, v) t = (1, 1) t
        errs.append(float(np.mean(np.abs(q[0] - ex[0]))))
    return errs


def test_vortex_second_order_without_limiter(oracle_lib):
    """With the limiter off (phi = 1) the flux, the conservative update and the
    RK2 rule are second order: the L1 density error drops 4x per refinement."""
    e = vortex_l1_errors(oracle_lib, 2)
    for a, b in zip(e, e[1:]):
        assert 3.7 < a / b < 4.3, e


def test_vortex_converges_with_pressure_minmod(oracle_lib):
    """With the pressure-ratio minmod of App. B the vortex still converges to the
    translated solution; the limiter clips at the core's pressure minimum, so
    the observed order at these sizes is about 1.1-1.3, not 2."""
    e = vortex_l1_errors(oracle_lib, 0)
    for a, b in zip(e, e[1:]):
        assert a / b > 1.9, e
    assert e[-1] < 1.5e-3, e


# ---------------------------------------------------------------- swept replay (Sec. 3.3)

def heat_cases():
    for nx, ny in ((32, 32), (48, 32)):
        for b in (8, 16):
            if nx % b or ny % b or nx // b < 2 or ny // b < 2:
                continue
            for d in range(2, b // 2, 2):  # d <= k = b/2 - 1, even
                yield nx, ny, b, d


@pytest.mark.parametrize("nx,ny,b,d", list(heat_cases()))
@pytest.mark.parametrize("nsteps", [0, 1, 2, 3, 7, 13])
def test_replay_heat_equals_step_by_step(oracle_lib, nx, ny, b, d, nsteps):
    u0 = W.heat_modes(nx, ny, seed=nx + b + d)
    dt, dx = W.heat_dt(nx, 0.1)
    r = oracle_lib.heat_r(dt, dx)
    ref = oracle_lib.heat_run(u0, nsteps, dt, dx)
    out, st = oracle_lib.swept_replay(0, u0, b, d, nsteps, 0.5 * r, r)
    assert np.array_equal(out, ref)
    assert st["cells"] == 2 * nsteps * nx * ny
    assert st["swept_levels"] == ((2 * nsteps) // d) * d if 2 * nsteps >= d else st["swept_levels"] == 0


@pytest.mark.parametrize("nx,b,d,nsteps", [(32, 16, 2, 5), (64, 16, 2, 3), (64, 32, 2, 3),
                                           (64, 32, 4, 5), (64, 32, 6, 7), (64, 32, 6, 2)])
def test_replay_euler_equals_step_by_step(oracle_lib, nx, b, d, nsteps):
    q0, dx = W.vortex(nx, xc=0.3, yc=-0.2)
    dt, _ = W.vortex_dt(q0, dx, 1.0)
    ref = oracle_lib.euler_run(q0, dt, dx, nsteps)
    lam2 = dt / dx
    out, st = oracle_lib.swept_replay(1, q0, b, d, nsteps, 0.5 * lam2, lam2)
    assert np.array_equal(out, ref)
    assert st["cells"] == 2 * nsteps * nx * nx


@pytest.mark.parametrize("plant", [1, 2])
def test_replay_catches_planted_schedule_mistakes(oracle_lib, plant):
    u0 = W.heat_modes(32, 32, seed=1)
    with pytest.raises(RuntimeError, match="unavailable|twice|never"):
        oracle_lib.swept_replay(0, u0, 8, 2, 9, 0.05, 0.1, plant=plant)


@pytest.mark.parametrize("b,d", [(8, 3), (8, 4), (12, 2), (4, 2), (16, 0)])
def test_replay_rejects_invalid_geometry(oracle_lib, b, d):
    """Eq. 1 bounds the depth (d <= b/(2n) - 1, even here); tiles divide the grid."""
    u0 = W.heat_modes(32, 32, seed=1)
    with pytest.raises(RuntimeError, match="invalid"):
        oracle_lib.swept_replay(0, u0, b, d, 4, 0.05, 0.1)
