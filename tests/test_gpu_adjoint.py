"""GPU discrete adjoint (sweep_adjoint) against the oracle's adjoint and
against central finite differences of the GPU forward solver.

Bars: the heat adjoint bit-identical to the oracle's (both are the same
two-stage stencil update in the same pinned order); the Euler adjoint within
1e-12 relative max-norm of the oracle's at 64x64 (the oracle applies the
chain rule face by face, as the reverse mode reads plainly, while the kernels
sum each cell's pressure adjoints before reversing its pressure once, so the
two round differently); finite differences (h = 1e-6, 16 seeded N(0,1)
directions) within 1e-6 relative, with the unlimited reconstruction (the
minmod limiter's switches make the scheme only piecewise smooth, so
differences straddling them measure nothing).
"""
import math

import numpy as np
import pytest

from paper_2105_10332_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_10332_b300 import build
    build.build()
    return torch


def relerr(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def smooth_vortex(n, seed=4, amp=2e-3):
    q, dx = W.vortex(n, xc=0.3, yc=-0.4)
    rng = np.random.default_rng(seed)
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x)
    for k in range(4):
        a = rng.uniform(0.5, 1.5, 3)
        q[k] = q[k] + amp * (a[0] * np.sin(2 * math.pi * (X + a[1])) +
                             a[2] * np.cos(2 * math.pi * (2 * Y + a[1])))
    return np.ascontiguousarray(q), dx


@pytest.mark.parametrize("nsteps", [1, 7, 40])
def test_heat_adjoint_matches_oracle(torch_cuda, oracle_lib, nsteps):
    torch = torch_cuda
    from paper_2105_10332_b300 import sweep as S
    dt, dx = W.heat_dt(64, 0.1)
    s = S.Solver("heat", 64, 64, dt, dx, 16, 6)
    lamT = np.random.default_rng(nsteps).standard_normal((64, 64))
    got = s.adjoint(None, torch.from_numpy(lamT).cuda(), nsteps).cpu().numpy()
    ref = oracle_lib.heat_adjoint(lamT, nsteps, dt, dx)
    assert np.array_equal(got, ref), relerr(got, ref)


@pytest.mark.parametrize("limiter", [0, 1, 2])
def test_euler_adjoint_matches_oracle_64(torch_cuda, oracle_lib, limiter):
    """64x64 vortex, 20 steps, checkpoints every 8 (three segments), every
    limiter mode: within 1e-12 relative max-norm of the oracle's adjoint."""
    torch = torch_cuda
    from paper_2105_10332_b300 import sweep as S
    q0, dx = W.vortex(64, xc=0.3, yc=-0.4)
    dt, _ = W.vortex_dt(q0, dx, 1.0)
    s = S.Solver("euler", 64, 64, dt, dx, 32, 6, limiter=limiter)
    target, _ = W.vortex(64, beta=4.5, xc=0.5, yc=0.5)
    qN = oracle_lib.euler_run(q0, dt, dx, 20, limiter=limiter)
    lamT = np.zeros_like(q0)
    lamT[0] = 2.0 * (qN[0] - target[0])
    ref = oracle_lib.euler_adjoint(q0, lamT, dt, dx, 20, ckpt=8, limiter=limiter)
    got = s.adjoint(torch.from_numpy(q0).cuda(), torch.from_numpy(lamT).cuda(), 20, 8)
    got = got.cpu().numpy()
    e = relerr(got, ref)
    assert e <= 1e-12, e


def test_euler_adjoint_fd_1024(torch_cuda):
    """1024^2 vortex with smooth modes, 60 steps, checkpoints every 16: the
    adjoint against central differences of the GPU forward solver along 16
    seeded directions (h = 1e-6), unlimited reconstruction."""
    torch = torch_cuda
    from paper_2105_10332_b300 import sweep as S
    n, N = 1024, 60
    q0, dx = smooth_vortex(n)
    dt, _ = W.vortex_dt(q0, dx, 10.0)
    s = S.Solver("euler", n, n, dt, dx, 32, 6, limiter=2)
    target = torch.from_numpy(W.vortex(n, beta=4.5, xc=0.5, yc=0.5)[0][0]).cuda()
    q0d = torch.from_numpy(q0).cuda()

    def loss(q):
        qq = q.clone()
        s.run_swept(qq, N)
        return float(torch.sum((qq[0] - target) ** 2))

    qN = q0d.clone()
    s.run_swept(qN, N)
    lamT = torch.zeros_like(q0d)
    lamT[0] = 2.0 * (qN[0] - target)
    g = s.adjoint(q0d, lamT, N, 16)
    gen = torch.Generator(device="cuda").manual_seed(20210521)
    h = 1e-6
    errs = []
    for _ in range(16):
        d = torch.randn(q0d.shape, generator=gen, device="cuda", dtype=torch.float64)
        fd = (loss(q0d + h * d) - loss(q0d - h * d)) / (2 * h)
        ad = float(torch.sum(g * d))
        errs.append(abs(fd - ad) / abs(ad))
    assert max(errs) <= 1e-6, errs


def test_autograd_function(torch_cuda, oracle_lib):
    """swept_run as a torch.autograd.Function: loss.backward() gives the adjoint."""
    torch = torch_cuda
    from paper_2105_10332_b300 import sweep as S
    q0, dx = W.vortex(64)
    dt, _ = W.vortex_dt(q0, dx, 1.0)
    s = S.Solver("euler", 64, 64, dt, dx, 32, 6)
    target = torch.from_numpy(W.vortex(64, beta=4.5, xc=0.5, yc=0.5)[0][0]).cuda()
    q = torch.from_numpy(q0).cuda().requires_grad_(True)
    qN = S.swept_run(q, s, 12, 5)
    loss = torch.sum((qN[0] - target) ** 2)
    loss.backward()
    ref_qN = oracle_lib.euler_run(q0, dt, dx, 12)
    assert np.array_equal(qN.detach().cpu().numpy(), ref_qN)
    lamT = np.zeros_like(q0)
    lamT[0] = 2.0 * (ref_qN[0] - target.cpu().numpy())
    ref = oracle_lib.euler_adjoint(q0, lamT, dt, dx, 12, ckpt=5)
    assert relerr(q.grad.cpu().numpy(), ref) <= 1e-12


def test_euler_adjoint_1024_full_size(torch_cuda):
    """The 1024^2 vortex adjoint at its full size, as bench.py runs it (2000
    steps, checkpoints every 64, unlimited reconstruction, loss
    sum((rho_T - rho_target)^2)): the gradient against central differences of
    the GPU forward solver along 16 seeded N(0,1) directions, h = 1e-6."""
    torch = torch_cuda
    import bench
    from paper_2105_10332_b300 import sweep as S
    wl = bench.workload("adjoint1024")
    s = S.Solver("euler", wl["nx"], wl["ny"], wl["dt"], wl["dx"], wl["tile"], wl["depth"],
                 limiter=wl["limiter"])
    N, K = wl["nsteps"], wl["ckpt"]
    q0 = torch.from_numpy(wl["state"]).cuda()
    target = torch.from_numpy(wl["target"]).cuda()

    def loss(q):
        qq = q.clone()
        s.run_swept(qq, N)
        return float(torch.sum((qq[0] - target) ** 2))

    qN = q0.clone()
    s.run_swept(qN, N)
    lamT = torch.zeros_like(q0)
    lamT[0] = 2.0 * (qN[0] - target)
    g = s.adjoint(q0, lamT, N, K)
    gen = torch.Generator(device="cuda").manual_seed(20210521)
    h = 1e-6
    errs = []
    for _ in range(16):
        d = torch.randn(q0.shape, generator=gen, device="cuda", dtype=torch.float64)
        fd = (loss(q0 + h * d) - loss(q0 - h * d)) / (2 * h)
        ad = float(torch.sum(g * d))
        errs.append(abs(fd - ad) / abs(ad))
    assert max(errs) <= 1e-6, errs
