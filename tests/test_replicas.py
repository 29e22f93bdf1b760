"""bench.py's multi-process path on CPU: two ranks over gloo.

The solver exchanges nothing between ranks (every rank is an independent
replica), so what N > 1 adds is host logic: the barriers around the timed
region, the max of the per-rank times, the whole-job rate over all ranks, and
the single-GPU arms running on rank 0 alone.  No GPU is touched here."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch
    import bench
    rep = bench.Replicas("gloo", torch.device("cpu"))
    rep.barrier()
    slowest = rep.max(times[rank])
    rate = bench.job_rate(rep.world, 4096, 500, 3, slowest)
    rep.barrier()
    rep.close()
    out.put((rank, rep.world, slowest, rate))


def test_two_replicas_share_the_slowest_time_and_sum_the_work():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    times = [0.25, 0.75]  # seconds of the timed region on each rank
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, world, slowest, rate in res:
        assert world == 2
        assert slowest == 0.75  # every rank reports the max over ranks
        # whole-job rate: both ranks' cell-steps over the slowest rank's time
        assert rate == pytest.approx(2 * 4096 * 500 * 3 / 0.75 / 1e9, rel=1e-15)


def test_single_rank_needs_no_process_group(monkeypatch):
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    rep = bench.Replicas("gloo", None)
    rep.barrier()
    assert rep.max(1.5) == 1.5
    rep.close()
    assert bench.job_rate(1, 65536, 2999, 5, 2.0) == pytest.approx(65536 * 2999 * 5 / 2.0 / 1e9)


@pytest.mark.parametrize("arm", ["reference", "adjoint", "batch"])
def test_single_gpu_arms_run_on_rank_zero_only(monkeypatch, capsys, arm):
    """Under torchrun the reference arm (the CPU oracle) and the single-GPU
    adjoint and batch measurements run on rank 0; rank 1 returns at once,
    prints nothing and touches neither the oracle nor a GPU."""
    import argparse
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    args = argparse.Namespace(steps=1, warmup=0, gpus=2, impl=arm, workload="heat64")
    fn = {"reference": bench.run_reference, "adjoint": bench.run_adjoint,
          "batch": bench.run_batch}[arm]
    assert fn(args, {"name": "unused"}) is None
    assert capsys.readouterr().out == ""
