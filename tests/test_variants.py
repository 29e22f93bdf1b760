"""Paper-literal variants: the forward-Euler heat rule of App. A, the printed
limiter orientation (covered in the parity tests), and the Table A1 vortex."""
import math
import os

import numpy as np
import pytest

from paper_2105_10332_b300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


def table_a1():
    vals = {}
    for line in open(os.path.join(HERE, "golden", "table_a1.txt")):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()
            vals[k] = float(v)
    return vals


def test_table_a1_generator_follows_the_table():
    t = table_a1()
    g = t["gamma"]
    q, dx = W.vortex_table_a1(128, gamma=g, half_width=t["L"])
    rho, mx, my, E = q
    u, v = mx / rho, my / rho
    p = (g - 1.0) * (E - 0.5 * rho * (u * u + v * v))
    M = math.sqrt(2.0 / g)
    # free stream (a corner cell, r ~ 7): rho -> 1, p -> 1/gamma, speed M at alpha = 45 deg
    a = math.radians(t["alpha_deg"])
    assert abs(rho[0, 0] - t["rho_inf"]) < 1e-9
    assert abs(p[0, 0] - t["p_inf"] / g) < 1e-9
    assert abs(u[0, 0] - M * math.cos(a)) < 1e-9 and abs(v[0, 0] - M * math.sin(a)) < 1e-9
    # isentropic: p = rho^gamma / gamma everywhere
    assert np.max(np.abs(p - rho ** g / g)) < 1e-13
    # the vortex is centred at the origin and its core is the density minimum
    j, i = np.unravel_index(np.argmin(rho), rho.shape)
    assert abs(-5 + (i + 0.5) * dx) < dx and abs(-5 + (j + 0.5) * dx) < dx


def test_heat_forward_euler_is_symmetric(oracle_lib):
    """<A u, v> = <u, A v> for the App. A forward-Euler step (its own adjoint)."""
    rng = np.random.default_rng(5)
    u, v = rng.standard_normal((2, 18, 26))
    dt, dx = W.heat_dt(26, 0.1)
    Au = oracle_lib.heat_run(u, 9, dt, dx, scheme=1)
    Av = oracle_lib.heat_run(v, 9, dt, dx, scheme=1)
    lhs, rhs = math.fsum((Au * v).ravel()), math.fsum((u * Av).ravel())
    assert abs(lhs - rhs) <= 1e-12 * math.fsum(np.abs(Au * v).ravel())


@pytest.mark.gpu
@pytest.mark.parametrize("nx,tile,depth", [(64, 16, 6), (64, 16, 2), (96, 32, 14), (48, 12, 4)])
@pytest.mark.parametrize("nsteps", [1, 2, 5, 17, 31])
def test_heat_forward_euler_gpu(oracle_lib, nx, tile, depth, nsteps):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_10332_b300 import sweep as S
    dt, dx = W.heat_dt(nx, 0.2)
    s = S.Solver("heat", nx, nx, dt, dx, tile, depth, scheme=1)
    u0 = W.heat_modes(nx, nx, seed=tile + nsteps)
    ref = oracle_lib.heat_run(u0, nsteps, dt, dx, scheme=1)
    for method in ("run_swept", "run_standard"):
        u = torch.from_numpy(u0).cuda()
        getattr(s, method)(u, nsteps)
        assert np.array_equal(u.cpu().numpy(), ref), method
    lam = s.adjoint(None, torch.from_numpy(u0).cuda(), nsteps).cpu().numpy()
    assert np.array_equal(lam, ref)  # the step is symmetric: adjoint = forward


@pytest.mark.gpu
def test_table_a1_vortex_gpu(oracle_lib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_10332_b300 import sweep as S
    q0, dx = W.vortex_table_a1(64)
    dt, _ = W.vortex_dt(q0, dx, 1.0)
    s = S.Solver("euler", 64, 64, dt, dx, 32, 6)
    q = torch.from_numpy(q0).cuda()
    s.run_swept(q, 13)
    assert np.array_equal(q.cpu().numpy(), oracle_lib.euler_run(q0, dt, dx, 13))
