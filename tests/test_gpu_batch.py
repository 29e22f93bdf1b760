"""Batched swept runs (sweep_batch_run) and the autotuner.

Bar: every instance of a batch is bit-identical to the same instance run
alone, eagerly and through a captured CUDA graph.
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
