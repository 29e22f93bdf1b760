#!/usr/bin/env python3
"""Benchmark: Gcell-steps/s of the swept-rule solver against the Standard
solver on one B300 (FP64), with the roofline of its dominant kernel.

One bench step = one whole run of the workload.  The default workload is the
large heat problem: a 16384 x 16384 periodic grid, a seeded sum of 8 Fourier
modes, r = 0.1, 2000 RK2 steps, swept block 64, depth 30 (30 stage-levels per
phase).  Inputs are seeded and synthetic and stay resident in device memory;
the state (2 GiB) and the level store (62 GiB) are far larger than L2, which
is also flushed (a 256 MiB write) between timed iterations.  The same line
carries the Euler vortex at 256 x 256 advanced to t = 10 (2999 steps, block
32, depth 6), Swept against Standard, as extra keys.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload heat16384|euler256|euler1024|heat64|heat4096|adjoint1024|batch256]
  python bench.py --peaks                      # the FP64 probe alone
  python bench.py --workload heat16384|heat64|euler256 --sweep
        # the block-size sweep (tile edge x depth x cluster), one line each
  python bench.py ... --l2-fetch 0|32|64|128   # the L2 fetch limit (default 32)
  python bench.py --workload W --ncu-run swept|standard
        # W warm-up runs then one run, nothing timed: the command that the
        # ncu captures summarised under profiles/ run

--impl reference times the CPU oracle (the plain fp64 C reference) on the
host cores on a bounded sample of the same workload.  Under torchrun
(N > 1) every rank runs its own replica; the solver has no data-path
exchange on one GPU.
"""
import argparse
import csv
import ctypes
import glob
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gcell-steps/s Swept vs Standard (FP64, 1 B300); % of HBM roofline"
UNIT = "Gcell-steps/s"
DEFAULT_WORKLOAD = "heat16384"

# Algorithmic FP64 work per cell and stage of the arithmetic specification
# (fma = 2 flops; add, mul, div, sqrt = 1): heat 3 adds + 2 fma = 7; Euler 187
# (cell pressure 9, limiter 6, two faces of 76, update 20).
FLOPS_PER_CELL_STAGE = {"heat": 7, "euler": 187}
SM_COUNT = 148
SM_MAX_MHZ_FALLBACK = 2032.0  # B300 maximum SM clock, used when no clock was sampled
HBM_FALLBACK_GBS = 6400.0  # used only where no measured copy bandwidth is on file
L2_FLUSH_BYTES = 256 << 20
CSRC = os.path.join(ROOT, "paper_2105_10332_b300", "csrc")
TRAFFIC_CSV = os.path.join(ROOT, "profiles", "dram_per_launch.csv")


def hbm_peak_gbs():
    """Measured HBM copy bandwidth of the B300s (GB/s) and its source."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK_GBS, "fallback"


def kernel_source_digest():
    """Digest of the library's CUDA sources and header: a traffic figure taken
    with ncu holds only for the build it was taken on."""
    h = hashlib.sha256()
    files = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh")))
    for f in files + [os.path.join(ROOT, "include", "sweep.h")]:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_per_launch(workload_name, kernel, path=TRAFFIC_CSV):
    """ncu DRAM bytes (read + write) of one launch of `kernel` in `workload_name`,
    from the committed capture list, or None when there is none for the
    current sources (the kernels changed since the counters were taken)."""
    try:
        with open(path, newline="") as f:
            rows = list(csv.DictReader(f))
    except OSError:
        return None
    digest = kernel_source_digest()
    for r in rows:
        if r["workload"] == workload_name and r["kernel"] == kernel and r["sources"] == digest:
            return int(r["dram_read_bytes"]) + int(r["dram_write_bytes"])
    return None


def workload(name):
    from paper_2105_10332_b300 import workloads as W
    if name == "euler256":
        q0, dx = W.vortex(256)
        dt, N = W.vortex_dt(q0, dx, 10.0, cfl=0.25)
        return dict(name="euler_vortex_256x256_t10", eqn="euler", nx=256, ny=256, dt=dt, dx=dx,
                    nsteps=N, tile=32, depth=6, state=q0)
    if name == "euler1024":
        # a larger vortex grid for the DRAM-bytes comparison (state 32 MiB)
        q0, dx = W.vortex(1024)
        dt, _ = W.vortex_dt(q0, dx, 10.0, cfl=0.25)
        return dict(name="euler_vortex_1024x1024_120steps", eqn="euler", nx=1024, ny=1024, dt=dt,
                    dx=dx, nsteps=120, tile=32, depth=6, state=q0)
    if name == "heat64":
        dt, dx = W.heat_dt(64, 0.1)
        return dict(name="heat_sine_64x64_500steps", eqn="heat", nx=64, ny=64, dt=dt, dx=dx,
                    nsteps=500, tile=16, depth=6, state=W.heat_sine(64, 64))
    if name == "heat4096":
        # a profiling-size heat case: state 128 MiB (larger than L2), level store 4 GiB
        dt, dx = W.heat_dt(4096, 0.1)
        return dict(name="heat_modes_4096x4096_200steps", eqn="heat", nx=4096, ny=4096, dt=dt,
                    dx=dx, nsteps=200, tile=64, depth=30, state=W.heat_modes(4096, 4096))
    if name == "heat16384":
        dt, dx = W.heat_dt(16384, 0.1)
        return dict(name="heat_modes_16384x16384_2000steps", eqn="heat", nx=16384, ny=16384,
                    dt=dt, dx=dx, nsteps=2000, tile=64, depth=30,
                    state=W.heat_modes(16384, 16384))
    if name == "batch256":
        return dict(name="batch_256_heat_euler_sides_64_2048_500steps", batch=True, count=256,
                    nsteps=500)
    if name == "adjoint1024":
        q0, dx = W.vortex(1024)
        dt, _ = W.vortex_dt(q0, dx, 10.0, cfl=0.25)
        target, _ = W.vortex(1024, beta=4.5, xc=0.5, yc=0.5)
        # unlimited reconstruction: the minmod limiter's branch derivative is
        # unbounded where the pressure is flat, and its exact discrete adjoint
        # overflows long before 2000 steps
        return dict(name="euler_vortex_1024x1024_2000steps_adjoint_ckpt64_unlimited", eqn="euler",
                    nx=1024, ny=1024, dt=dt, dx=dx, nsteps=2000, tile=32, depth=6, state=q0,
                    target=target[0], ckpt=64, adjoint=True, limiter=2)
    raise SystemExit("unknown workload %s" % name)


def shape_cells(eqn, b, d, kind, tiles):
    """Algorithmic cell-stages one launch of a swept kernel computes."""
    n = 1 if eqn == "heat" else 2
    up = sum((b - 2 * s * n) ** 2 for s in range(1, d + 1))
    lower = sum((2 * s * n) ** 2 for s in range(1, d + 1))
    bridge = 2 * sum((2 * s * n) * (b - 2 * s * n) for s in range(1, d + 1))
    return tiles * {"up_pyramid": up, "bridges": bridge, "octahedron": lower + up,
                    "down_pyramid": lower}[kind]


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for name, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Replicas:
    """N independent replicas, one per rank (torchrun).  The solver exchanges
    nothing between ranks, so the only collectives are the barriers around the
    timed region and the max of the per-rank times.  backend: "nccl" on GPUs
    ("gloo" on CPU); device: where the reduced value lives."""

    def __init__(self, backend, device):
        self.world, self.rank, self.local = dist_setup()
        self.device = device
        if self.world > 1:
            import torch
            import torch.distributed as dist
            kw = {"device_id": device} if backend == "nccl" else {}
            dist.init_process_group(backend, **kw)
            self._torch, self._dist = torch, dist

    def barrier(self):
        if self.world > 1:
            self._dist.barrier()

    def max(self, x):
        if self.world == 1:
            return x
        t = self._torch.tensor([float(x)], dtype=self._torch.float64, device=self.device)
        self._dist.all_reduce(t, op=self._dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.world > 1:
            self._dist.destroy_process_group()


def job_rate(world, cells, nsteps, runs, seconds):
    """Whole-job Gcell-steps/s: each of `world` replicas advanced `cells` cells
    by `nsteps` steps `runs` times within `seconds` (the slowest rank's time)."""
    return world * cells * nsteps * runs / seconds / 1e9


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample(wl, budget_s):
    """Time the CPU oracle on chunks of the workload, from its initial state,
    until budget_s passes; a workload shorter than the budget is run again
    from the start.  Returns (Gcell-steps/s, steps run, seconds)."""
    import oracle
    cells = wl["nx"] * wl["ny"]
    state = wl["state"]
    steps, t_total, in_run = 0, 0.0, 0
    chunk = max(1, int(2e7 // (cells * (40 if wl["eqn"] == "euler" else 1))))
    while t_total < budget_s:
        c = min(chunk, wl["nsteps"] - in_run)
        t0 = time.perf_counter()
        if wl["eqn"] == "euler":
            state = oracle.euler_run(state, wl["dt"], wl["dx"], c)
        else:
            state = oracle.heat_run(state, c, wl["dt"], wl["dx"])
        t_total += time.perf_counter() - t0
        steps += c
        in_run += c
        if in_run == wl["nsteps"]:
            state, in_run = wl["state"], 0
    return cells * steps / t_total / 1e9, steps, t_total


def run_reference(args, wl):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    os.environ.setdefault("OMP_NUM_THREADS", str(cpu_cores()))
    cores = int(os.environ["OMP_NUM_THREADS"])
    for _ in range(args.warmup):
        oracle_sample(wl, 0.5)
    vals, secs, nsteps = [], 0.0, 0
    for _ in range(args.steps):
        v, n, s = oracle_sample(wl, 5.0)
        vals.append(v)
        secs += s
        nsteps += n
    value = wl["nx"] * wl["ny"] * nsteps / secs / 1e9
    sample = ("%d RK2 steps per bench step of the %s workload (%d-step runs from its initial "
              "state), oracle compiled -O2 -ffp-contract=off, OpenMP"
              % (nsteps // args.steps, wl["name"], wl["nsteps"]))
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1000 * secs / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["name"], "nx": wl["nx"], "ny": wl["ny"],
                       "steps_per_run": wl["nsteps"], "solver": "cpu oracle, step by step"},
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batch(args, wl):
    """256 instances (even index heat, odd Euler vortex), square sides drawn
    log-uniform in [64, 2048] (multiples of 32, seeded), 500 steps each, knobs
    from the autotuner per (equation, size class).  One bench step = one
    replay of the captured batch graph; the baseline runs each instance alone,
    one after another."""
    if dist_setup()[1] != 0:
        return  # a single-GPU measurement: under torchrun rank 0 alone runs it
    import torch
    from paper_2105_10332_b300 import autotune, sweep as S, workloads as W
    dev = torch.device("cuda", torch.cuda.current_device())
    sides = W.batch_sides(wl["count"])
    tuner = autotune.Autotuner()
    solvers, init, cells = [], [], 0
    for k, n in enumerate(sides):
        if k % 2 == 0:
            dt, dx = W.heat_dt(n, 0.1)
            u0 = W.heat_modes(n, n, seed=20210521 + k)
            eqn = "heat"
        else:
            u0, dx = W.vortex(n)
            dt, _ = W.vortex_dt(u0, dx, 10.0)
            eqn = "euler"
        t = torch.from_numpy(u0).to(dev)
        cfg = dict(tuner.best(eqn, n, dt, dx, t))
        tile, depth = cfg.pop("tile"), cfg.pop("depth")
        solvers.append(S.Solver(eqn, n, n, dt, dx, tile, depth, **cfg))
        init.append(t)
        cells += n * n
    N = wl["nsteps"]
    states = [t.clone() for t in init]
    # each instance alone, one after another
    ev = lambda: torch.cuda.Event(enable_timing=True)
    solo_ms = 0.0
    for s_, st, t in zip(solvers, states, init):
        st.copy_(t)
        s_.run_swept(st, N)  # warm-up of this instance's kernels
        st.copy_(t)
        torch.cuda.synchronize(dev)
        a, b = ev(), ev()
        a.record()
        s_.run_swept(st, N)
        b.record()
        torch.cuda.synchronize(dev)
        solo_ms += a.elapsed_time(b)
    solo_out = [st.clone() for st in states]
    batch = S.Batch(solvers, states, N)
    batch.capture()
    for _ in range(max(args.warmup, 1)):
        for st, t in zip(states, init):
            st.copy_(t)
        batch.replay()
    torch.cuda.synchronize(dev)
    ms = 0.0
    for _ in range(args.steps):
        for st, t in zip(states, init):
            st.copy_(t)
        torch.cuda.synchronize(dev)
        a, b = ev(), ev()
        a.record()
        batch.replay()
        b.record()
        torch.cuda.synchronize(dev)
        ms += a.elapsed_time(b)
    ms /= args.steps
    identical = all(torch.equal(x, y) for x, y in zip(states, solo_out))
    classes = sorted(set((k[0], k[1]) for k in tuner.cache))
    line = {"metric": "aggregate Gcell-steps/s, batched (one graph launch) vs each instance alone",
            "value": round(cells * N / (ms / 1e3) / 1e9, 6), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded heat modes / isentropic vortices)",
            "config": {"workload": wl["name"], "instances": len(sides), "steps_per_instance": N,
                       "cells_total": cells},
            "solo": {"value": round(cells * N / (solo_ms / 1e3) / 1e9, 6), "ms": round(solo_ms, 3)},
            "batched_over_solo": round(solo_ms / ms, 4), "bit_identical_to_solo": identical,
            "autotuned": {"%s/%d" % c: tuner.cache[c] for c in classes}}
    print(json.dumps(line), flush=True)


def run_adjoint(args, wl):
    """Gradient of sum((rho_T - rho_target)^2) w.r.t. the initial state: one bench
    step = one sweep_adjoint call (checkpointed swept forward pass + reverse
    pass).  Reports Gcell-steps/s of the gradient and its time over the plain
    swept forward run."""
    if dist_setup()[1] != 0:
        return  # a single-GPU measurement: under torchrun rank 0 alone runs it
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    N, cells = wl["nsteps"], wl["nx"] * wl["ny"]
    ms_adj, ms_fwd, gnorm = measure_adjoint(wl, dev, args.warmup, args.steps)
    line = {"metric": "Gcell-steps/s of the discrete adjoint (FP64, 1 B300)",
            "value": round(cells * N / (ms_adj / 1e3) / 1e9, 6), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_adj, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded isentropic vortex)",
            "config": {"workload": wl["name"], "nx": wl["nx"], "ny": wl["ny"], "steps_per_run": N,
                       "ckpt_every": wl["ckpt"], "tile": wl["tile"], "depth": wl["depth"]},
            "forward_ms": round(ms_fwd, 3), "adjoint_over_forward": round(ms_adj / ms_fwd, 3),
            "grad_norm": gnorm}
    print(json.dumps(line), flush=True)


def measure_adjoint(wl, dev, warmup, steps):
    """Milliseconds of one gradient (mean of `steps` sweep_adjoint calls after
    `warmup`), of one plain swept forward run, and the gradient's norm."""
    import torch
    from paper_2105_10332_b300 import sweep as S
    solver = S.Solver(wl["eqn"], wl["nx"], wl["ny"], wl["dt"], wl["dx"], wl["tile"], wl["depth"],
                      limiter=wl.get("limiter", 0))
    N = wl["nsteps"]
    q0 = torch.from_numpy(wl["state"]).to(dev)
    target = torch.from_numpy(wl["target"]).to(dev)
    qN = q0.clone()
    solver.run_swept(qN, N)
    lamT = torch.zeros_like(q0)
    lamT[0] = 2.0 * (qN[0] - target)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    for _ in range(warmup):
        solver.adjoint(q0, lamT, N, wl["ckpt"])
    torch.cuda.synchronize(dev)
    a0, a1 = ev(), ev()
    a0.record()
    for _ in range(steps):
        g = solver.adjoint(q0, lamT, N, wl["ckpt"])
    a1.record()
    torch.cuda.synchronize(dev)
    ms_adj = a0.elapsed_time(a1) / steps
    f0, f1 = ev(), ev()
    q = q0.clone()
    f0.record()
    solver.run_swept(q, N)
    f1.record()
    torch.cuda.synchronize(dev)
    return ms_adj, f0.elapsed_time(f1), float(torch.linalg.vector_norm(g))


def measure_fp64(dev, target_s=0.25, launches=5):
    """The FP64 rate of this GPU from the library's fma probe (sweep_fp64_probe):
    4 CTAs of 256 threads per SM, 8 independent chains per thread, timed
    with CUDA events on the launching stream while nvidia-smi samples the SM
    clock.  The roofline peak is the measured rate scaled from the sampled
    clock to the maximum SM clock: 148 SMs x (measured fma lanes per clock and
    SM) x 2 flops x the maximum clock."""
    import torch
    from paper_2105_10332_b300 import sweep as S
    blocks, threads = 4 * SM_COUNT, 256
    out = torch.empty(blocks * threads, dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream(dev)

    def launch(iters):
        rc = S.sweep_fp64_probe(ctypes.c_void_p(out.data_ptr()), iters, blocks, threads,
                                ctypes.c_void_p(st.cuda_stream))
        if rc != S.SWEEP_OK:
            raise RuntimeError("sweep_fp64_probe: status %d" % rc)

    def timed(iters):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        launch(iters)
        b.record(st)
        return a, b

    launch(1000)  # warm-up (module load)
    a, b = timed(2000)
    torch.cuda.synchronize(dev)
    iters = max(2000, int(2000 * target_s * 1e3 / max(a.elapsed_time(b), 1e-3)))
    flops = 16.0 * iters * blocks * threads
    sampler = ClockSampler(dev.index if dev.index is not None else 0)
    with sampler:
        time.sleep(0.3)
        evs = [timed(iters) for _ in range(launches)]
        torch.cuda.synchronize(dev)
    rates = sorted(flops / (x.elapsed_time(y) / 1e3) / 1e12 for x, y in evs)
    tflops = statistics.median(rates)
    clk = sampler.summary()
    sm_max = clk["sm_max_mhz"] or SM_MAX_MHZ_FALLBACK
    sm = clk["sm_mhz"] or sm_max
    lanes = tflops * 1e12 / 2 / (SM_COUNT * sm * 1e6)
    peak = SM_COUNT * lanes * 2 * sm_max * 1e6 / 1e12
    return {"tflops_measured": round(tflops, 4), "sm_mhz": sm, "sm_max_mhz": sm_max,
            "fma_lanes_per_clk_per_sm": round(lanes, 3), "peak_tflops": round(peak, 4),
            "clock_samples": clk["samples"], "reasons": clk["reasons"],
            "basis": "sweep_fp64_probe: %d CTAs x %d threads x 8 fma chains, median of %d "
                     "launches; peak = 148 SMs x measured fma lanes/clk/SM x 2 flops x max SM clock"
                     % (blocks, threads, launches)}


# Library parameters every bench solver takes: the 32-byte L2 fetch
# granularity for the process (the level store's column pieces use one
# sector of each line; with the default the swept kernels read about 2.5x
# the bytes they use, run time being the same either way).
BENCH_PARAMS = {"l2_fetch_bytes": 32}


class Runner:
    """One workload's solver, device state and workspace, with each method's
    whole run (all its launches) captured once into a CUDA graph and
    replayed, so that host launch overhead enters neither method's timing."""

    def __init__(self, wl, dev):
        import torch
        from paper_2105_10332_b300 import sweep as S
        self.torch, self.wl, self.dev = torch, wl, dev
        self.solver = S.Solver(wl["eqn"], wl["nx"], wl["ny"], wl["dt"], wl["dx"], wl["tile"],
                               wl["depth"], **BENCH_PARAMS)
        self.N, self.cells = wl["nsteps"], wl["nx"] * wl["ny"]
        self.init = torch.from_numpy(wl["state"]).to(dev)
        self.state = self.init.clone()
        self.ws = self.solver.workspace(dev)
        self.flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
        self.stream = torch.cuda.current_stream(dev)
        self.graphs = {}

    def graph(self, method):
        torch = self.torch
        if method not in self.graphs:
            getattr(self.solver, method)(self.state, self.N, self.ws)  # attributes set before capture
            torch.cuda.synchronize(self.dev)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                getattr(self.solver, method)(self.state, self.N, self.ws)
            self.graphs[method] = g
        return self.graphs[method]

    def warm(self, method, W):
        for _ in range(W):
            self.state.copy_(self.init)
            self.graph(method).replay()
        self.torch.cuda.synchronize(self.dev)

    def timed(self, method, K):
        """Total device milliseconds of K whole runs, L2 flushed before each."""
        torch = self.torch
        g = self.graph(method)
        evs = []
        for _ in range(K):
            self.state.copy_(self.init)
            self.flush.fill_(1)  # evict the state and level store from L2
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            g.replay()
            e1.record(self.stream)
            evs.append((e0, e1))
        torch.cuda.synchronize(self.dev)
        return sum(a.elapsed_time(b) for a, b in evs)

    def profile(self):
        """One more swept run with an event pair around each launch."""
        self.solver.set("profile", 1)
        self.state.copy_(self.init)
        self.flush.fill_(1)
        self.solver.run_swept(self.state, self.N, self.ws)
        prof = self.solver.profile()
        self.solver.set("profile", 0)
        return prof


def roofline(wl, prof, fp64):
    """FP64-ALU roofline of the dominant kernel: its algorithmic flops per
    launch over its live mean launch time, against the measured FP64 peak;
    and the HBM side of the same kernel from its ncu DRAM bytes per launch."""
    tiles = (wl["nx"] // wl["tile"]) * (wl["ny"] // wl["tile"])
    dom = max((k for k in prof if prof[k][1] > 0), key=lambda k: prof[k][0])
    dom_ms = prof[dom][0] / prof[dom][1]
    cells = wl["nx"] * wl["ny"]
    dom_cells = 2 * cells if dom == "standard" else shape_cells(wl["eqn"], wl["tile"], wl["depth"],
                                                                 dom, tiles)
    flops = dom_cells * FLOPS_PER_CELL_STAGE[wl["eqn"]]
    achieved = flops / (dom_ms / 1e3) / 1e12
    traffic = traffic_per_launch(wl["name"], dom)
    peak = fp64["peak_tflops"]
    out = {"bound": "alu", "achieved": round(achieved, 4), "peak": peak, "unit": "TFLOP/s",
           "frac": round(achieved / peak, 4), "traffic": traffic, "kernel": dom,
           "launch_ms": round(dom_ms, 5), "flops_per_launch": flops,
           "peak_basis": "FP64, of measured (probe rate at the sampled clock scaled to the "
                         "maximum clock)",
           "fp64_probe": fp64,
           "kernels": {k: {"ms_total": round(v[0], 4), "launches": v[1]} for k, v in prof.items()}}
    if traffic is not None:
        peak_gbs, basis = hbm_peak_gbs()
        gbs = traffic / (dom_ms / 1e3) / 1e9
        out["hbm"] = {"achieved": round(gbs, 2), "peak": peak_gbs, "unit": "GB/s",
                      "frac": round(gbs / peak_gbs, 4), "peak_basis": basis}
    return out


def run_peaks(args):
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    print(json.dumps({"fp64_probe": measure_fp64(dev)}), flush=True)


def run_ncu(args, wl):
    """W eager warm-up runs and one more run of one method, nothing timed: the
    command an ncu capture wraps (its -s skips the launches before the one
    to capture).  Prints the launches of the last run."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    r = Runner(wl, dev)
    method = "run_swept" if args.ncu_run == "swept" else "run_standard"
    for _ in range(args.warmup):
        r.state.copy_(r.init)
        getattr(r.solver, method)(r.state, r.N, r.ws)
    r.solver.set("profile", 1)
    r.state.copy_(r.init)
    getattr(r.solver, method)(r.state, r.N, r.ws)
    prof = r.solver.profile()
    print(json.dumps({"ncu_run": wl["name"], "method": args.ncu_run, "runs": args.warmup + 1,
                      "launches_per_run": {k: v[1] for k, v in prof.items()}}), flush=True)


SWEEP_PLANS = {
    # the block-size sweep of the large heat workload: tile edges 8-64, for each
    # the largest even depth and about half of it (edges 12 and 24 do not
    # divide 16384 and run on 16368 = 12 x 1364 = 24 x 682)
    "heat16384": dict(tiles=(8, 12, 16, 24, 32, 48, 64), clusters=(1,), depths="max_half",
                      standard_tiles=(16, 32, 64)),
    # the small heat grid: every depth and cluster size of edges 8, 16, 32
    "heat64": dict(tiles=(8, 16, 32), clusters=(1, 2, 4), depths="all", standard_tiles=(8, 16, 32)),
    "euler256": dict(tiles=(16, 32), clusters=(1, 2, 4), depths="all", standard_tiles=(8, 16)),
}


def sweep_configs(wl, plan):
    """(nx, tile, depth, cluster) of a block-size sweep of workload wl."""
    n = 1 if wl["eqn"] == "heat" else 2
    out = []
    for b in plan["tiles"]:
        nx = (wl["nx"] // b) * b  # the largest multiple of the edge that fits
        if nx // b < 2 or nx % 2:
            continue
        k = b // (2 * n) - 1
        ds = [d for d in range(2, k + 1, 2)]
        if not ds:
            continue
        if plan["depths"] == "max_half":
            ds = sorted({ds[-1], ds[max(0, len(ds) // 2 - 1)]})
        for d in ds:
            for c in plan["clusters"]:
                out.append((nx, b, d, c))
    return out


# steps per run of the heat grids of a Standard-edge sweep over grid sides
HEAT_SIDE_STEPS = {256: 2000, 512: 2000, 1024: 1000, 2048: 500, 4096: 200, 8192: 100}


def side_workload(wl, n):
    """The heat workload wl on an n x n grid (same mesh ratio and field)."""
    from paper_2105_10332_b300 import workloads as W
    w = dict(wl, name="heat_modes_%dx%d_%dsteps" % (n, n, HEAT_SIDE_STEPS[n]), nx=n, ny=n,
             nsteps=HEAT_SIDE_STEPS[n], state=W.heat_modes(n, n))
    w["dt"], w["dx"] = W.heat_dt(n, 0.1)
    return w


def run_sweep_standard(args, wl, dev):
    """Standard Gcell-steps/s of the workload at each block edge of its plan;
    with --sides (heat), of the same workload on those grid sides instead,
    each with Swept at the workload's tile and depth beside it.  One JSON
    line per grid."""
    import torch
    from paper_2105_10332_b300 import sweep as S
    cases = [side_workload(wl, n) for n in args.sides] if args.sides else [wl]
    for w in cases:
        r = Runner(w, dev)
        line = {"sweep": w["name"], "default_standard_tile": int(r.solver.get("standard_tile"))}
        for t in SWEEP_PLANS[args.workload]["standard_tiles"]:
            try:
                r.solver.set("standard_tile", t)
            except S.SweepError:
                continue  # the edge does not divide this grid
            r.graphs.pop("run_standard", None)
            r.warm("run_standard", 2)
            ms = r.timed("run_standard", args.steps) / args.steps
            line["standard_%d" % t] = round(job_rate(1, r.cells, r.N, 1, ms / 1e3), 4)
        if args.sides:
            r.warm("run_swept", 2)
            ms = r.timed("run_swept", args.steps) / args.steps
            line["swept"] = round(job_rate(1, r.cells, r.N, 1, ms / 1e3), 4)
        print(json.dumps(line), flush=True)
        del r
        torch.cuda.empty_cache()


def run_sweep(args, wl):
    """Swept Gcell-steps/s of the workload for each (tile, depth, cluster) of
    its plan, and Standard once per grid size; one JSON line per
    configuration (graph replay, L2 flushed, K = --steps runs each).  With
    --sweep-standard, the Standard solver at each block edge of the plan
    instead."""
    import torch
    from paper_2105_10332_b300 import sweep as S, workloads as W
    dev = torch.device("cuda", torch.cuda.current_device())
    if args.sweep_standard:
        run_sweep_standard(args, wl, dev)
        return
    plan = dict(SWEEP_PLANS[args.workload])
    if args.tiles:
        plan["tiles"] = tuple(t for t in plan["tiles"] if t in args.tiles)
    done_std, states = set(), {}
    for nx, b, d, c in sweep_configs(wl, plan):
        cfg = dict(wl)
        if nx != wl["nx"]:  # heat only: the edge does not divide the grid
            if nx not in states:
                states[nx] = W.heat_modes(nx, nx)
            cfg.update(nx=nx, ny=nx, name=wl["name"].replace(str(wl["nx"]), str(nx)),
                       state=states[nx])
            cfg["dt"], cfg["dx"] = W.heat_dt(nx, 0.1)
        cfg.update(tile=b, depth=d)
        try:
            r = Runner(cfg, dev)
            if c != r.solver.get("cluster_oct") or c != r.solver.get("cluster_bridges"):
                r.solver.set("cluster", c)
        except S.SweepError as e:
            print(json.dumps({"sweep": cfg["name"], "tile": b, "depth": d, "cluster": c,
                              "skipped": str(e)}), flush=True)
            continue
        r.warm("run_swept", 1)
        ms = r.timed("run_swept", args.steps) / args.steps
        line = {"sweep": cfg["name"], "tile": b, "depth": d, "cluster": c,
                "swept": round(job_rate(1, r.cells, r.N, 1, ms / 1e3), 4), "ms_per_run": round(ms, 4)}
        if nx not in done_std:
            r.warm("run_standard", 1)
            mt = r.timed("run_standard", args.steps) / args.steps
            line.update(standard=round(job_rate(1, r.cells, r.N, 1, mt / 1e3), 4),
                        standard_tile=int(r.solver.get("standard_tile")))
            done_std.add(nx)
        print(json.dumps(line), flush=True)
        del r
        torch.cuda.empty_cache()


def paired_extra(name, dev, fp64, K):
    """Swept against Standard on another workload: K whole runs of each."""
    w = workload(name)
    r = Runner(w, dev)
    r.warm("run_swept", 3)
    r.warm("run_standard", 3)
    vs = job_rate(1, r.cells, r.N, K, r.timed("run_swept", K) / 1e3)
    vt = job_rate(1, r.cells, r.N, K, r.timed("run_standard", K) / 1e3)
    roof = roofline(w, r.profile(), fp64)
    roof.pop("fp64_probe")
    return {"workload": w["name"], "runs": K, "swept": round(vs, 6), "standard": round(vt, 6),
            "swept_over_standard": round(vs / vt, 4), "roofline": roof}


def run_ours(args, wl):
    import torch
    world, rank, local = dist_setup()
    dev = torch.device("cuda", local if world > 1 else torch.cuda.current_device())
    torch.cuda.set_device(dev)
    rep = Replicas("nccl", dev)
    barrier, max_over_ranks = rep.barrier, rep.max

    main = Runner(wl, dev)
    N, cells = main.N, main.cells
    K = args.steps
    # the Standard solver is the comparison, not the headline: it is timed on
    # at most 3 whole runs (each run of the large heat workload is ~11 s)
    K_std = min(K, 3)

    # warm-up (untimed), including the graph captures
    main.warm("run_swept", args.warmup)
    main.warm("run_standard", 1)

    # timed region: K swept runs, clocks sampled throughout
    sampler = ClockSampler(dev.index if dev.index is not None else 0)
    barrier()
    torch.cuda.synchronize(dev)
    with sampler:
        ms_swept = main.timed("run_swept", K)
        torch.cuda.synchronize(dev)
    barrier()
    ms_swept = max_over_ranks(ms_swept)
    clocks = sampler.summary()

    barrier()
    torch.cuda.synchronize(dev)
    ms_std = max_over_ranks(main.timed("run_standard", K_std))
    barrier()

    prof = main.profile()
    launches_per_run = sum(n for _, n in prof.values())

    # end to end through the public API with host buffers (pinned): H2D copy,
    # run, D2H copy inside the timed region
    host0 = torch.from_numpy(wl["state"]).pin_memory()
    host = host0.clone().pin_memory()
    K_e2e = max(1, min(K, 2))
    e2e_s = 0.0
    for _ in range(K_e2e):
        host.copy_(host0)
        main.flush.fill_(1)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        main.solver.run_swept(host, N)
        torch.cuda.synchronize(dev)
        e2e_s += time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s)
    state_bytes = main.init.numel() * 8
    del host, host0

    value = job_rate(world, cells, N, K, ms_swept / 1e3)
    v_std = job_rate(world, cells, N, K_std, ms_std / 1e3)
    v_e2e = job_rate(world, cells, N, K_e2e, e2e_s)
    fp64 = measure_fp64(dev)
    roof = roofline(wl, prof, fp64)

    line = None
    if rank == 0:
        extras = {}
        if wl["name"] == workload(DEFAULT_WORKLOAD)["name"] and not args.no_extras:
            # the other single-instance workloads under the same clock: the
            # Euler vortex at 256^2 and heat at 64^2, Swept against Standard
            # on the same protocol (graph replay, L2 flushed), and one
            # gradient of the Euler adjoint at 1024^2
            for key in ("euler256", "heat64"):
                extras[key] = paired_extra(key, dev, fp64, max(1, min(K, 5)))
            aw = workload("adjoint1024")
            ms_adj, ms_fwd, _ = measure_adjoint(aw, dev, 1, 1)
            extras["adjoint1024"] = {
                "workload": aw["name"], "gradients": 1,
                "value": round(aw["nx"] * aw["ny"] * aw["nsteps"] / (ms_adj / 1e3) / 1e9, 6),
                "gradient_ms": round(ms_adj, 3), "forward_ms": round(ms_fwd, 3),
                "adjoint_over_forward": round(ms_adj / ms_fwd, 3)}
        os.environ.setdefault("OMP_NUM_THREADS", str(cpu_cores()))
        cb_value, cb_steps, cb_secs = oracle_sample(wl, 12.0)
        cpu_baseline = {"value": round(cb_value, 6), "unit": UNIT,
                        "cores": int(os.environ["OMP_NUM_THREADS"]), "kind": "oracle",
                        "sample": "%d RK2 steps of the same workload (%d-step runs from its "
                                  "initial state), %.1f s" % (cb_steps, N, cb_secs)}
        line = {"metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world,
                "steps": K, "warmup": args.warmup,
                "ms_per_step": round(ms_swept / K, 3), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (seeded heat modes / isentropic vortex)",
                "config": {"workload": wl["name"], "nx": wl["nx"], "ny": wl["ny"],
                           "steps_per_run": N, "tile": wl["tile"], "depth": wl["depth"],
                           "standard_tile": int(main.solver.get("standard_tile")),
                           "l2": "inputs larger than L2, and flushed (256 MiB write) between "
                                 "timed iterations",
                           "launch": "each run captured once into a CUDA graph and replayed",
                           "standard_runs_timed": K_std, "e2e_runs": K_e2e,
                           "library_params": BENCH_PARAMS,
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "standard": {"value": round(v_std, 6), "ms_per_step": round(ms_std / K_std, 3)},
                "swept_over_standard": round(value / v_std, 4),
                "e2e": {"value": round(v_e2e, 6), "unit": UNIT, "h2d_bytes_per_step": state_bytes,
                        "d2h_bytes_per_step": state_bytes},
                "gpu_launches": int(launches_per_run * K),
                "roofline": roof, "cpu_baseline": cpu_baseline, "clocks": clocks}
        line.update(extras)
        print(json.dumps(line), flush=True)
    rep.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--peaks", action="store_true")
    ap.add_argument("--ncu-run", choices=["swept", "standard"], default=None)
    ap.add_argument("--sweep", action="store_true")
    ap.add_argument("--tiles", type=lambda v: [int(t) for t in v.split(",")], default=None,
                    help="with --sweep: only these tile edges of the plan (comma list)")
    ap.add_argument("--sweep-standard", action="store_true",
                    help="with --sweep: the Standard solver at each block edge of the plan")
    ap.add_argument("--sides", type=lambda v: [int(t) for t in v.split(",")], default=None,
                    help="with --sweep-standard (heat): these grid sides instead of the "
                         "workload's (" + ",".join(str(n) for n in HEAT_SIDE_STEPS) + ")")
    ap.add_argument("--no-extras", action="store_true",
                    help="the default workload's line without its extra workloads")
    ap.add_argument("--l2-fetch", type=int, choices=[0, 32, 64, 128], default=32,
                    help="L2 fetch-granularity limit the solvers set for the process "
                         "(0: leave the context's default)")
    args = ap.parse_args()
    BENCH_PARAMS["l2_fetch_bytes"] = args.l2_fetch
    if args.peaks:
        run_peaks(args)
        return
    if args.warmup < 3 and args.impl == "ours" and args.ncu_run is None:
        args.warmup = 3
    wl = workload(args.workload)
    if args.impl == "reference":
        run_reference(args, wl)
    elif args.ncu_run:
        run_ncu(args, wl)
    elif args.sweep:
        run_sweep(args, wl)
    elif wl.get("adjoint"):
        run_adjoint(args, wl)
    elif wl.get("batch"):
        run_batch(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
