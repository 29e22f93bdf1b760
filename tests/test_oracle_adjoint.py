"""Pins for the oracle's discrete adjoints (reverse mode of App. A / App. B).

The gradient of a final-state loss must equal central finite differences
where the scheme is smooth.  The pressure-ratio minmod of App. B is only
piecewise smooth: min(ratio, 1) switches wherever the ratio crosses 1, which
a smooth field does in many cells, so a central difference with h = 1e-6
straddles switches and measures nothing useful.  The h = 1e-6 pins therefore
run with the reconstruction unlimited (limiter mode 2, phi = 1), and the
minmod derivative is pinned face by face and over one step with h = 1e-8.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_2105_10332_b300 import workloads as W


def smooth_field(n, seed=4, amp=2e-3):
    """Vortex plus small smooth modes in every component (no flat regions)."""
    q, dx = W.vortex(n, xc=0.3, yc=-0.4)
    rng = np.random.default_rng(seed)
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x)
    for k in range(4):
        a = rng.uniform(0.5, 1.5, 3)
        q[k] = q[k] + amp * (a[0] * np.sin(2 * math.pi * (X + a[1])) +
                             a[2] * np.cos(2 * math.pi * (2 * Y + a[1])))
    return np.ascontiguousarray(q), dx


def density_loss(oracle_lib, q0, dt, dx, N, limiter, target):
    qN = oracle_lib.euler_run(q0, dt, dx, N, limiter=limiter)
    L = float(np.sum((qN[0] - target[0]) ** 2))
    lamT = np.zeros_like(q0)
    lamT[0] = 2.0 * (qN[0] - target[0])
    return L, lamT


def fd_errors(oracle_lib, q0, dt, dx, N, limiter, h, ndir, ckpt=4, seed=20210521):
    target, _ = W.vortex(q0.shape[-1], beta=4.5, xc=0.5, yc=0.5)
    _, lamT = density_loss(oracle_lib, q0, dt, dx, N, limiter, target)
    g = oracle_lib.euler_adjoint(q0, lamT, dt, dx, N, ckpt=ckpt, limiter=limiter)
    rng = np.random.default_rng(seed)
    errs = []
    for _ in range(ndir):
        d = rng.standard_normal(q0.shape)
        lp, _ = density_loss(oracle_lib, q0 + h * d, dt, dx, N, limiter, target)
        lm, _ = density_loss(oracle_lib, q0 - h * d, dt, dx, N, limiter, target)
        fd = (lp - lm) / (2 * h)
        ad = float(np.sum(g * d))
        errs.append(abs(fd - ad) / abs(ad))
    return errs


def test_euler_adjoint_matches_fd_unlimited(oracle_lib):
    """16 seeded N(0,1) directions, h = 1e-6, relative error <= 1e-6."""
    q0, dx = smooth_field(16)
    dt, _ = W.vortex_dt(q0, dx, 1.0)
    errs = fd_errors(oracle_lib, q0, dt, dx, 6, 2, 1e-6, 16)
    assert max(errs) <= 1e-6, errs


def test_euler_adjoint_matches_fd_minmod_one_step(oracle_lib):
    q0, dx = smooth_field(16)
    dt, _ = W.vortex_dt(q0, dx, 1.0)
    errs = fd_errors(oracle_lib, q0, dt, dx, 1, 0, 1e-8, 8)
    assert max(errs) <= 1e-5, errs


def test_face_vjp_matches_fd_every_limiter(oracle_lib):
    L = oracle_lib.lib()
    dp = ctypes.POINTER(ctypes.c_double)
    L.oracle_face_flux_vjp.argtypes = [dp, dp, dp, dp, ctypes.c_double, ctypes.c_int, dp, dp]
    rng = np.random.default_rng(1)

    def cons(rho, u, v, p):
        return np.array([rho, rho * u, rho * v, p / 0.4 + 0.5 * rho * (u * u + v * v)])

    for lim in (0, 1, 2):
        worst = 0.0
        for _ in range(200):
            qs = [cons(rng.uniform(0.8, 1.2), rng.normal(0, 0.3), rng.normal(0, 0.3),
                       rng.uniform(0.8, 1.2)) for _ in range(4)]
            a = rng.standard_normal(4)
            g = np.zeros(16)
            L.oracle_face_flux_vjp(*[oracle_lib._dptr(np.ascontiguousarray(x)) for x in qs], 1.4,
                                   lim, oracle_lib._dptr(np.ascontiguousarray(a)),
                                   oracle_lib._dptr(g))
            d = [rng.standard_normal(4) for _ in range(4)]
            h = 1e-7
            fp = oracle_lib.face_flux(*[q + h * e for q, e in zip(qs, d)], limiter=lim)
            fm = oracle_lib.face_flux(*[q - h * e for q, e in zip(qs, d)], limiter=lim)
            fd = float(np.dot(a, (fp - fm) / (2 * h)))
            ad = float(np.dot(g, np.concatenate(d)))
            worst = max(worst, abs(fd - ad) / max(abs(ad), 1e-12))
        assert worst <= 1e-5, (lim, worst)


def test_euler_adjoint_checkpoint_invariant(oracle_lib):
    """Checkpoint spacing changes where states are recomputed, not the result."""
    q0, dx = smooth_field(16)
    dt, _ = W.vortex_dt(q0, dx, 1.0)
    lamT = np.random.default_rng(2).standard_normal(q0.shape)
    g1 = oracle_lib.euler_adjoint(q0, lamT, dt, dx, 7, ckpt=1)
    g3 = oracle_lib.euler_adjoint(q0, lamT, dt, dx, 7, ckpt=3)
    g64 = oracle_lib.euler_adjoint(q0, lamT, dt, dx, 7, ckpt=64)
    assert np.array_equal(g1, g3) and np.array_equal(g1, g64)


def test_euler_adjoint_zero_steps_identity(oracle_lib):
    q0, dx = smooth_field(8)
    lamT = np.random.default_rng(3).standard_normal(q0.shape)
    assert np.array_equal(oracle_lib.euler_adjoint(q0, lamT, 1e-3, dx, 0), lamT)


def test_heat_adjoint_dot_product(oracle_lib):
    """<A^N u, v> = <u, (A^T)^N v> for the RK2 heat step (linear, symmetric L)."""
    rng = np.random.default_rng(7)
    u = rng.standard_normal((20, 28))
    v = rng.standard_normal((20, 28))
    N = 37
    dt, dx = W.heat_dt(28, 0.1)
    Au = oracle_lib.heat_run(u, N, dt, dx)
    Atv = oracle_lib.heat_adjoint(v, N, dt, dx)
    lhs = math.fsum((Au * v).ravel())
    rhs = math.fsum((u * Atv).ravel())
    assert abs(lhs - rhs) <= 1e-12 * math.fsum(np.abs(Au * v).ravel())


def test_heat_adjoint_closed_form(oracle_lib):
    """A mode is an eigenvector of the adjoint step with the same G (L symmetric)."""
    n, N, r = 32, 50, 0.1
    x, y = W.heat_grid(n, n)
    mode = np.outer(np.sin(2 * math.pi * 3 * y + 0.4), np.sin(2 * math.pi * 2 * x + 1.1))
    lam = -4 * (math.sin(math.pi * 2 / n) ** 2 + math.sin(math.pi * 3 / n) ** 2)
    z = r * lam
    G = 1 + z + 0.5 * z * z
    dt, dx = W.heat_dt(n, r)
    got = oracle_lib.heat_adjoint(mode, N, dt, dx)
    assert np.max(np.abs(got - G ** N * mode)) <= 1e-13


def test_minmod_adjoint_blows_up_unlimited_stays_bounded(oracle_lib):
    """The branch-taken derivative of min(dm/dp, 1) is 1/dp, unbounded where the
    pressure is flat to rounding while the momentum is not (the vortex's far
    field): the minmod scheme's exact discrete adjoint grows by orders of
    magnitude per step there, while the unlimited reconstruction's stays O(1).
    Long-horizon gradients therefore use the unlimited reconstruction."""
    n = 64
    q0, dx = W.vortex(n)
    dt, _ = W.vortex_dt(q0, dx, 10.0)
    tgt, _ = W.vortex(n, beta=4.5, xc=0.5, yc=0.5)
    out = {}
    for lim in (0, 2):
        qN = oracle_lib.euler_run(q0, dt, dx, 60, limiter=lim)
        lamT = np.zeros_like(q0)
        lamT[0] = 2 * (qN[0] - tgt[0])
        out[lim] = float(np.max(np.abs(oracle_lib.euler_adjoint(q0, lamT, dt, dx, 60, limiter=lim))))
    assert out[0] > 1e20 and out[2] < 10.0, out
