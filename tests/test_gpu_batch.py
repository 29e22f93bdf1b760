"""Batched swept runs (sweep_batch_run) and the autotuner.

Bars: every instance of a batch matches the CPU oracle within 1e-12 relative
max-norm (bit identity expected and reported), and is bit-identical to the
same instance run alone, eagerly and through a captured CUDA graph; the full
256-instance batch of heat and Euler grids is bit-identical to its solo runs.
"""
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


def make_instances(torch, S):
    specs = [("heat", 64, 16, 6, 23), ("euler", 96, 32, 6, 9), ("heat", 160, 32, 14, 30),
             ("euler", 64, 16, 2, 5), ("heat", 96, 32, 6, 1), ("euler", 128, 32, 4, 7),
             ("heat", 256, 64, 30, 40), ("euler", 192, 32, 6, 13)]
    solvers, states, steps, init = [], [], [], []
    for eqn, n, b, d, N in specs:
        if eqn == "heat":
            dt, dx = W.heat_dt(n, 0.1)
            u0 = W.heat_modes(n, n, seed=n + b)
        else:
            u0, dx = W.vortex(n, xc=0.2, yc=0.1)
            dt, _ = W.vortex_dt(u0, dx, 1.0)
        solvers.append(S.Solver(eqn, n, n, dt, dx, b, d))
        t = torch.from_numpy(u0).cuda()
        states.append(t.clone())
        init.append(t)
        steps.append(N)
    return solvers, states, steps, init


def solo(torch, solvers, init, steps):
    out = []
    for s, t, N in zip(solvers, init, steps):
        u = t.clone()
        s.run_swept(u, N)
        out.append(u)
    torch.cuda.synchronize()
    return out


def test_batch_equals_solo(torch_cuda):
    torch = torch_cuda
    from paper_2105_10332_b300 import sweep as S
    solvers, states, steps, init = make_instances(torch, S)
    ref = solo(torch, solvers, init, steps)
    b = S.Batch(solvers, states, steps)
    for st in states:
        st.view(-1)[:] = float("nan")  # overwritten below
    for st, t in zip(states, init):
        st.copy_(t)
    b.run()
    torch.cuda.synchronize()
    for k, (a, r) in enumerate(zip(states, ref)):
        assert torch.equal(a, r), k


def test_batch_graph_replay_equals_solo(torch_cuda):
    torch = torch_cuda
    from paper_2105_10332_b300 import sweep as S
    solvers, states, steps, init = make_instances(torch, S)
    ref = solo(torch, solvers, init, steps)
    b = S.Batch(solvers, states, steps)
    b.capture()
    for rep in range(2):
        for st, t in zip(states, init):
            st.copy_(t)
        b.replay()
        torch.cuda.synchronize()
        for k, (a, r) in enumerate(zip(states, ref)):
            assert torch.equal(a, r), (rep, k)


def test_autotuner_picks_a_legal_config(torch_cuda):
    torch = torch_cuda
    from paper_2105_10332_b300 import autotune
    tuner = autotune.Autotuner()
    u0, dx = W.vortex(128)
    dt, _ = W.vortex_dt(u0, dx, 1.0)
    cfg = tuner.best("euler", 128, dt, dx, torch.from_numpy(u0).cuda())
    assert cfg in autotune.candidates("euler", 128)
    assert len(tuner.log) == len(autotune.candidates("euler", 128))
    hd, hdx = W.heat_dt(256, 0.1)
    cfg = tuner.best("heat", 256, hd, hdx, torch.from_numpy(W.heat_modes(256, 256)).cuda())
    assert cfg["tile"] in autotune.HEAT_TILES


def relerr(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def test_mixed_batch_matches_oracle(torch_cuda, oracle_lib):
    """Heat and Euler instances of uneven sides (powers of two and not),
    tiles, depths and step counts in one batch, replayed from a CUDA graph:
    each against the oracle's step-by-step run."""
    torch = torch_cuda
    from paper_2105_10332_b300 import sweep as S
    specs = [("heat", 96, 32, 14, 31), ("euler", 96, 32, 6, 17), ("heat", 352, 32, 6, 23),
             ("euler", 224, 32, 4, 9), ("heat", 160, 16, 6, 40), ("euler", 352, 16, 2, 7),
             ("heat", 480, 32, 14, 15), ("euler", 160, 32, 6, 12), ("heat", 72, 12, 4, 29),
             ("euler", 120, 24, 4, 11)]
    solvers, states, steps, refs, init = [], [], [], [], []
    for k, (eqn, n, b, d, N) in enumerate(specs):
        if eqn == "heat":
            dt, dx = W.heat_dt(n, 0.1)
            u0 = W.heat_modes(n, n, seed=100 + k)
            refs.append(oracle_lib.heat_run(u0, N, dt, dx))
        else:
            u0, dx = W.vortex(n, xc=0.1 * k, yc=-0.05 * k)
            dt, _ = W.vortex_dt(u0, dx, 1.0)
            refs.append(oracle_lib.euler_run(u0, dt, dx, N))
        solvers.append(S.Solver(eqn, n, n, dt, dx, b, d))
        t = torch.from_numpy(u0).cuda()
        init.append(t)
        states.append(t.clone())
        steps.append(N)
    batch = S.Batch(solvers, states, steps)
    batch.capture()
    for st, t in zip(states, init):
        st.copy_(t)
    batch.replay()
    torch.cuda.synchronize()
    for k, (st, ref) in enumerate(zip(states, refs)):
        got = st.cpu().numpy()
        e = relerr(got, ref)
        assert e <= 1e-12, (specs[k], e)
        assert np.array_equal(got, ref), (specs[k], "within 1e-12 but not bitwise", e)


def test_full_256_instance_batch(torch_cuda, oracle_lib):
    """The batched workload at full size: 256 instances (even index heat, odd
    Euler vortex), sides log-uniform in [64, 2048] (multiples of 32, seeded),
    500 steps each, configurations from the autotuner's class ranking (here
    ranked by tile and depth instead of timed, to keep the test short), all
    in one CUDA-graph replay.  Every instance is bit-identical to its solo
    run, and the instances of side 64 and 96 to the oracle's full run."""
    torch = torch_cuda
    from paper_2105_10332_b300 import autotune, sweep as S
    sides = W.batch_sides(256)
    tuner = autotune.Autotuner()
    rank = lambda cfg: -cfg["tile"] - 0.01 * cfg["depth"] + 0.1 * cfg.get("cluster_oct", 1)
    N = 500
    solvers, init, specs = [], [], []
    for k, n in enumerate(sides):
        if k % 2 == 0:
            dt, dx = W.heat_dt(n, 0.1)
            u0 = W.heat_modes(n, n, seed=20210521 + k)
            eqn = "heat"
        else:
            u0, dx = W.vortex(n)
            dt, _ = W.vortex_dt(u0, dx, 10.0)
            eqn = "euler"
        cfg = dict(tuner.select(eqn, n, rank))
        tile, depth = cfg.pop("tile"), cfg.pop("depth")
        solvers.append(S.Solver(eqn, n, n, dt, dx, tile, depth, **cfg))
        init.append(torch.from_numpy(u0).cuda())
        specs.append((eqn, n, dt, dx, u0))
    solo = []
    for s_, t in zip(solvers, init):
        u = t.clone()
        s_.run_swept(u, N)
        solo.append(u)
        s_._ws = None  # release the solo workspace; the batch has its own
    torch.cuda.synchronize()
    states = [t.clone() for t in init]
    batch = S.Batch(solvers, states, N)
    batch.capture()
    for st, t in zip(states, init):
        st.copy_(t)
    batch.replay()
    torch.cuda.synchronize()
    for k, (a, b) in enumerate(zip(states, solo)):
        assert torch.equal(a, b), (k, specs[k][:2])
    checked = 0
    for k, (eqn, n, dt, dx, u0) in enumerate(specs):
        if n > 96:
            continue
        ref = (oracle_lib.heat_run(u0, N, dt, dx) if eqn == "heat"
               else oracle_lib.euler_run(u0, dt, dx, N))
        got = states[k].cpu().numpy()
        assert relerr(got, ref) <= 1e-12 and np.array_equal(got, ref), (k, eqn, n)
        checked += 1
    assert checked >= 8
