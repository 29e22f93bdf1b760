"""GPU parity: the CUDA path against the CPU oracle, and Swept against Standard.

Bars (written per test):
  - GPU Standard and GPU Swept against the oracle: at most 1e-12 relative
    max-norm (both follow the same pinned arithmetic, so the gap is expected
    to be zero; any nonzero gap is reported in the assertion message);
  - GPU Swept against GPU Standard: bit-identical (torch.equal).
"""
import math

import numpy as np
import pytest

from paper_2105_10332_b300 import workloads as W

pytestmark = pytest.mark.gpu

REL = 1e-12
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_10332_b300 import build
    build.build()
    return torch


def relerr(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def gpu_run(torch, solver, state_np, nsteps, method, poison=True):
    st = torch.from_numpy(np.ascontiguousarray(state_np)).cuda()
    ws = solver.workspace(st.device)
    if poison:
        ws.view(torch.float64)[: ws.numel() // 8].fill_(float("nan"))
    getattr(solver, method)(st, nsteps)
    torch.cuda.synchronize()
    return st.cpu().numpy()


def heat_solver(S, nx, ny, tile, depth, r=0.1, **kw):
    """A heat solver at mesh ratio r (App. A: r = alpha dt / dx^2, alpha = 1,
    dx = 1/nx).  Returns (solver, dt, dx): the oracle gets the same physical
    inputs and forms r itself, so nothing the library computes feeds it."""
    dt, dx = W.heat_dt(nx, r)
    s = S.Solver("heat", nx, ny, dt, dx, tile, depth, **kw)
    assert abs(s.get("r") - r) <= 4 * EPS * r
    return s, dt, dx


def euler_solver(S, nx, ny, tile, depth, T=1.0, **kw):
    q0, dx = W.vortex(nx, ny, xc=0.4, yc=-0.3)
    dt, N = W.vortex_dt(q0, dx, T)
    return S.Solver("euler", nx, ny, dt, dx, tile, depth, **kw), q0, dt, dx


# ------------------------------------------------------------------- heat

def test_heat_standard_matches_oracle_sine64(torch_cuda, oracle_lib):
    from paper_2105_10332_b300 import sweep as S
    s, dt, dx = heat_solver(S, 64, 64, 16, 6)
    u0 = W.heat_sine(64, 64)
    ref = oracle_lib.heat_run(u0, 500, dt, dx)
    got = gpu_run(torch_cuda, s, u0, 500, "run_standard")
    e = relerr(got, ref)
    assert e <= REL, e
    assert np.array_equal(got, ref), "standard vs oracle not bitwise (rel %.3g)" % e


@pytest.mark.parametrize("nx,ny,tile", [(64, 64, 8), (64, 64, 16), (96, 64, 16), (64, 64, 32),
                                        (48, 72, 12), (80, 40, 20), (56, 84, 14), (40, 60, 10)])
# block edges 14 and 10 (2 mod 4) put the shifted windows on odd columns:
# their level-store traffic takes the one-cell path instead of 16-byte pairs
@pytest.mark.parametrize("nsteps", [1, 3, 4, 7, 26])
def test_heat_swept_bit_identical(torch_cuda, oracle_lib, nx, ny, tile, nsteps):
    from paper_2105_10332_b300 import sweep as S
    u0 = W.heat_modes(nx, ny, seed=nx * 7 + tile)
    k = tile // 2 - 1
    ref = None
    for d in range(2, k + 1, 2):
        s, dt, dx = heat_solver(S, nx, ny, tile, d)
        if ref is None:
            ref = oracle_lib.heat_run(u0, nsteps, dt, dx)
            std = gpu_run(torch_cuda, s, u0, nsteps, "run_standard")
            assert np.array_equal(std, ref), relerr(std, ref)
        sw = gpu_run(torch_cuda, s, u0, nsteps, "run_swept")
        assert np.array_equal(sw, std), ("d=%d" % d, relerr(sw, std))


@pytest.mark.parametrize("nx,ny", [(128, 128), (256, 256), (1024, 1024), (2048, 512)])
@pytest.mark.parametrize("depth", [14, 30])
def test_heat_block64_large_levels(torch_cuda, oracle_lib, nx, ny, depth):
    """Block 64.  From 2^16 cells heat runs the wide swept kernels (levels
    of at least 16 cells per thread take two neighbouring cells per thread,
    smaller ones one), from 2^20 cells the paired Standard step; below, the
    one-cell kernels.  Swept and Standard match the oracle bit for bit."""
    from paper_2105_10332_b300 import sweep as S
    s, dt, dx = heat_solver(S, nx, ny, 64, depth)
    u0 = W.heat_modes(nx, ny, seed=depth)
    for nsteps in (17, 31):
        ref = oracle_lib.heat_run(u0, nsteps, dt, dx)
        for method in ("run_swept", "run_standard"):
            got = gpu_run(torch_cuda, s, u0, nsteps, method)
            assert np.array_equal(got, ref), (method, nsteps, relerr(got, ref))


@pytest.mark.parametrize("cluster,passes", [(2, 1), (4, 1), (1, 2), (2, 2)])
def test_heat_wide_kernels_in_bands(torch_cuda, oracle_lib, cluster, passes):
    """The wide heat kernels with a window shared by a cluster of CTAs, or
    walked in sub-bands: each band of a level takes the pair or the one-cell
    branch on its own size.  1024^2, block 64, against the oracle."""
    from paper_2105_10332_b300 import sweep as S
    s, dt, dx = heat_solver(S, 1024, 1024, 64, 30)
    s.set("cluster", cluster)
    s.set("passes", passes)
    u0 = W.heat_modes(1024, 1024, seed=cluster * 10 + passes)
    ref = oracle_lib.heat_run(u0, 31, dt, dx)
    got = gpu_run(torch_cuda, s, u0, 31, "run_swept")
    assert np.array_equal(got, ref), relerr(got, ref)


@pytest.mark.parametrize("n,tile,depth", [(1036, 14, 6), (1026, 18, 8)])
def test_heat_wide_kernels_odd_half_edges(torch_cuda, oracle_lib, n, tile, depth):
    """Above 2^20 cells with block edges whose half is odd: the shifted
    windows start on odd columns, so a level's pairs start on either parity
    of column; the Standard edge is the smallest even divisor (14, 18).
    Swept and Standard against the oracle, bit for bit."""
    from paper_2105_10332_b300 import sweep as S
    s, dt, dx = heat_solver(S, n, n, tile, depth)
    u0 = W.heat_modes(n, n, seed=tile)
    ref = oracle_lib.heat_run(u0, 13, dt, dx)
    for method in ("run_swept", "run_standard"):
        got = gpu_run(torch_cuda, s, u0, 13, method)
        assert np.array_equal(got, ref), (method, relerr(got, ref))


def test_heat_wide_kernels_pair_levels(torch_cuda, oracle_lib):
    """Block 96 on 1056^2: the Up-Pyramid's and the Octahedron's largest
    levels hold at least 16 cells per thread, so the wide kernels take their
    two-cells-per-thread branch there (with block 64 no level is that
    large).  50 steps (two swept cycles of depth 46) against the oracle."""
    from paper_2105_10332_b300 import sweep as S
    s, dt, dx = heat_solver(S, 1056, 1056, 96, 46)
    u0 = W.heat_modes(1056, 1056, seed=96)
    ref = oracle_lib.heat_run(u0, 50, dt, dx)
    got = gpu_run(torch_cuda, s, u0, 50, "run_swept")
    assert np.array_equal(got, ref), relerr(got, ref)


@pytest.mark.parametrize("n,edge", [(1024, 32), (2048, 64)])
def test_heat_standard_paired_step(torch_cuda, oracle_lib, n, edge):
    """From 2^20 cells the Standard heat step takes two cells per thread,
    on 64-wide blocks with 512 threads: the default edges at 1024^2 and
    2048^2 against the oracle, bit for bit."""
    from paper_2105_10332_b300 import sweep as S
    s, dt, dx = heat_solver(S, n, n, 32, 14)
    assert s.get("standard_tile") == edge
    u0 = W.heat_modes(n, n, seed=11)
    ref = oracle_lib.heat_run(u0, 9, dt, dx)
    got = gpu_run(torch_cuda, s, u0, 9, "run_standard")
    assert np.array_equal(got, ref), relerr(got, ref)


def test_heat_swept_sine64_and_closed_form(torch_cuda, oracle_lib):
    """Heat sine 64^2, r = 0.1, 500 steps, tile 16: Swept = Standard = oracle,
    and the discrete closed form G^500 within 1e-13."""
    from paper_2105_10332_b300 import sweep as S
    s, dt, dx = heat_solver(S, 64, 64, 16, 6)
    u0 = W.heat_sine(64, 64)
    sw = gpu_run(torch_cuda, s, u0, 500, "run_swept")
    ref = oracle_lib.heat_run(u0, 500, dt, dx)
    assert np.array_equal(sw, ref), relerr(sw, ref)
    z = 0.1 * (-8.0 * math.sin(math.pi / 64) ** 2)  # the workload's r = 0.1
    G = 1 + z + 0.5 * z * z
    assert relerr(sw, G ** 500 * u0) <= 1e-13


# ------------------------------------------------------------------- Euler

def test_euler_standard_matches_oracle(torch_cuda, oracle_lib):
    from paper_2105_10332_b300 import sweep as S
    s, q0, dt, dx = euler_solver(S, 64, 64, 32, 6)
    ref = oracle_lib.euler_run(q0, dt, dx, 40)
    got = gpu_run(torch_cuda, s, q0, 40, "run_standard")
    e = relerr(got, ref)
    assert e <= REL, e
    assert np.array_equal(got, ref), "standard vs oracle not bitwise (rel %.3g)" % e


@pytest.mark.parametrize("nx,ny,tile", [(48, 72, 12), (64, 64, 16), (64, 64, 32), (96, 48, 24),
                                        (72, 108, 36), (40, 60, 20), (72, 36, 18)])
@pytest.mark.parametrize("nsteps", [1, 3, 5, 11])
def test_euler_swept_bit_identical(torch_cuda, oracle_lib, nx, ny, tile, nsteps):
    from paper_2105_10332_b300 import sweep as S
    k = tile // 4 - 1
    std = None
    for d in range(2, k + 1, 2):
        s, q0, dt, dx = euler_solver(S, nx, ny, tile, d)
        if std is None:
            ref = oracle_lib.euler_run(q0, dt, dx, nsteps)
            std = gpu_run(torch_cuda, s, q0, nsteps, "run_standard")
            assert np.array_equal(std, ref), relerr(std, ref)
        sw = gpu_run(torch_cuda, s, q0, nsteps, "run_swept")
        assert np.array_equal(sw, std), ("d=%d" % d, relerr(sw, std))


def test_euler_literal_limiter(torch_cuda, oracle_lib):
    from paper_2105_10332_b300 import sweep as S
    s, q0, dt, dx = euler_solver(S, 64, 64, 16, 2, limiter=1)
    ref = oracle_lib.euler_run(q0, dt, dx, 9, limiter=1)
    sw = gpu_run(torch_cuda, s, q0, 9, "run_swept")
    assert np.array_equal(sw, ref), relerr(sw, ref)


def test_constant_states_preserved(torch_cuda):
    from paper_2105_10332_b300 import sweep as S
    s, _, dt, dx = euler_solver(S, 64, 64, 16, 2)
    rho, u, v, p = 1.3, 0.7, -0.4, 2.1
    q = np.stack([np.full((64, 64), x) for x in (rho, rho * u, rho * v,
                                                p / 0.4 + 0.5 * rho * (u * u + v * v))])
    assert np.array_equal(gpu_run(torch_cuda, s, q, 13, "run_swept"), q)
    h, _, _ = heat_solver(S, 64, 64, 16, 6)
    c = np.full((64, 64), -3.25)
    assert np.array_equal(gpu_run(torch_cuda, h, c, 13, "run_swept"), c)


def test_zero_steps_is_identity(torch_cuda):
    from paper_2105_10332_b300 import sweep as S
    h, _, _ = heat_solver(S, 64, 64, 16, 6)
    u0 = W.heat_modes(64, 64, seed=2)
    assert np.array_equal(gpu_run(torch_cuda, h, u0, 0, "run_swept"), u0)


def test_resume_is_bit_identical(torch_cuda):
    """run(N1) then run(N2) equals run(N1 + N2), phase-aligned or not."""
    from paper_2105_10332_b300 import sweep as S
    s, q0, dt, dx = euler_solver(S, 64, 64, 32, 6)
    full = gpu_run(torch_cuda, s, q0, 17, "run_swept")
    for n1 in (3, 6, 8):
        a = gpu_run(torch_cuda, s, q0, n1, "run_swept")
        b = gpu_run(torch_cuda, s, a, 17 - n1, "run_swept")
        assert np.array_equal(b, full), n1


# ------------------------------------------------------------------- full sizes

def test_euler_vortex256_full_run(torch_cuda, oracle_lib):
    """Vortex 256^2, CFL 0.25, t = 10 (2999 steps), tile 32, d = 6 --
    the launch configuration the benchmark times.  Swept = Standard bitwise,
    and both equal the oracle's full run."""
    from paper_2105_10332_b300 import sweep as S
    q0, dx = W.vortex(256)
    dt, N = W.vortex_dt(q0, dx, 10.0)
    assert N == 2999
    s = S.Solver("euler", 256, 256, dt, dx, 32, 6)
    sw = gpu_run(torch_cuda, s, q0, N, "run_swept", poison=False)
    std = gpu_run(torch_cuda, s, q0, N, "run_standard", poison=False)
    assert np.array_equal(sw, std), relerr(sw, std)
    ref = oracle_lib.euler_run(q0, dt, dx, N)
    e = relerr(sw, ref)
    assert e <= REL, e
    assert np.array_equal(sw, ref), "swept vs oracle not bitwise (rel %.3g)" % e
    for k in range(4):  # conservation over the whole run
        drift = abs(math.fsum(sw[k].ravel()) - math.fsum(q0[k].ravel()))
        assert drift <= 64 * np.finfo(float).eps * N * math.fsum(np.abs(q0[k]).ravel())


def test_heat_large_sampled_closed_form(torch_cuda):
    """The seeded 8-mode heat field (r = 0.1) at 4096^2 for 200 steps:
    Swept = Standard bitwise and sampled cells match the discrete closed form."""
    from paper_2105_10332_b300 import sweep as S
    torch = torch_cuda
    n, N = 4096, 200
    dt, dx = W.heat_dt(n, 0.1)
    s = S.Solver("heat", n, n, dt, dx, 32, 14)
    r = 0.1  # the workload's mesh ratio, not the library's
    u0 = W.heat_modes(n, n)
    a = torch.from_numpy(u0).cuda()
    b = a.clone()
    s.run_swept(a, N)
    s.run_standard(b, N)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    rng = np.random.default_rng(3)
    js, is_ = rng.integers(0, n, 64), rng.integers(0, n, 64)
    got = a[js, is_].cpu().numpy()
    x, y = W.heat_grid(n, n)
    exp = np.zeros(64)
    for amp, kx, ky, phx, phy in W.heat_modes_spec():
        lam = -4 * (math.sin(math.pi * kx / n) ** 2 + math.sin(math.pi * ky / n) ** 2)
        z = r * lam
        G = 1 + z + 0.5 * z * z
        exp += amp * G ** N * np.sin(2 * math.pi * ky * y[js] + phy) * np.sin(2 * math.pi * kx * x[is_] + phx)
    assert np.max(np.abs(got - exp)) <= 1e-12 * np.max(np.abs(u0))


# ------------------------------------------------------------------- clusters

@pytest.mark.parametrize("cluster,passes", [(1, 1), (2, 1), (4, 1), (1, 2), (2, 2), (1, 4)])
@pytest.mark.parametrize("eqn,nx,ny,tile", [("euler", 64, 64, 32), ("euler", 96, 48, 24),
                                             ("euler", 72, 108, 36), ("heat", 64, 64, 16),
                                             ("heat", 80, 40, 20), ("heat", 56, 56, 14)])
def test_cluster_sizes_bit_identical(torch_cuda, oracle_lib, cluster, passes, eqn, nx, ny, tile):
    """A window shared by 1, 2 or 4 CTAs (distributed shared memory), each
    taking its rows in 1, 2 or 4 passes, gives the same bits as the oracle for
    every legal depth and several step counts."""
    from paper_2105_10332_b300 import sweep as S
    n = 1 if eqn == "heat" else 2
    k = tile // (2 * n) - 1
    for d in range(2, k + 1, 2):
        if eqn == "euler":
            s, q0, dt, dx = euler_solver(S, nx, ny, tile, d)
        else:
            s, hdt, hdx = heat_solver(S, nx, ny, tile, d)
            q0 = W.heat_modes(nx, ny, seed=tile + d)
        try:
            s.set("cluster", cluster)
            s.set("passes", passes)
        except S.SweepError:
            continue  # window does not fit this cluster size's shared memory
        for N in (3, 8):
            if eqn == "euler":
                ref = oracle_lib.euler_run(q0, dt, dx, N)
            else:
                ref = oracle_lib.heat_run(q0, N, hdt, hdx)
            got = gpu_run(torch_cuda, s, q0, N, "run_swept")
            assert np.array_equal(got, ref), (cluster, d, N, relerr(got, ref))


def test_heat_modes16384_full_size(torch_cuda):
    """Heat 16384^2 at its full size and in the launch configuration
    bench.py times (2000 steps, block 64, depth 30): Swept = Standard
    bitwise, and 256 sampled cells match the discrete closed form
    (measured gap 5.5e-14 of max|u0|)."""
    from paper_2105_10332_b300 import sweep as S
    torch = torch_cuda
    n, N = 16384, 2000
    dt, dx = W.heat_dt(n, 0.1)
    s = S.Solver("heat", n, n, dt, dx, 64, 30)
    r = 0.1  # the workload's mesh ratio, not the library's
    u0 = W.heat_modes(n, n)
    a = torch.from_numpy(u0).cuda()
    b = a.clone()
    s.run_swept(a, N)
    s.run_standard(b, N)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    del b
    rng = np.random.default_rng(3)
    js, is_ = rng.integers(0, n, 256), rng.integers(0, n, 256)
    got = a[torch.from_numpy(js).cuda(), torch.from_numpy(is_).cuda()].cpu().numpy()
    x, y = W.heat_grid(n, n)
    exp = np.zeros(256)
    for amp, kx, ky, phx, phy in W.heat_modes_spec():
        lam = -4 * (math.sin(math.pi * kx / n) ** 2 + math.sin(math.pi * ky / n) ** 2)
        z = r * lam
        G = 1 + z + 0.5 * z * z
        exp += amp * G ** N * np.sin(2 * math.pi * ky * y[js] + phy) * np.sin(2 * math.pi * kx * x[is_] + phx)
    assert np.max(np.abs(got - exp)) <= 1e-12 * np.max(np.abs(u0))
