"""bench.py's host-side arithmetic, on CPU: the algorithmic cell-stage counts
behind the roofline, the CPU oracle sample and the HBM peak lookup."""
import json

import pytest


@pytest.mark.parametrize("eqn,b,d", [("heat", 16, 6), ("heat", 64, 30), ("heat", 32, 2),
                                     ("euler", 32, 6), ("euler", 24, 4), ("euler", 12, 2)])
def test_shape_cells_partition_every_cycle(eqn, b, d):
    """Every (cell, level) is computed once (Sec. 3.3): per cycle the Bridges
    and the Octahedron together compute each of a block's b^2 cells at d
    levels, and so do the Up-Pyramid, the first Bridges and the
    Down-Pyramid of a one-cycle run."""
    import bench
    tiles = 7
    full = tiles * b * b * d
    cycle = bench.shape_cells(eqn, b, d, "bridges", tiles) + bench.shape_cells(eqn, b, d, "octahedron", tiles)
    assert cycle == full
    first = (bench.shape_cells(eqn, b, d, "up_pyramid", tiles) +
             bench.shape_cells(eqn, b, d, "bridges", tiles) +
             bench.shape_cells(eqn, b, d, "down_pyramid", tiles))
    assert first == full


def test_oracle_sample_repeats_a_short_workload(oracle_lib):
    """A workload shorter than the time budget runs again from its initial
    state, so the sample is bounded by time, not by the workload's length."""
    import bench
    from paper_2105_10332_b300 import workloads as W
    dt, dx = W.heat_dt(16, 0.1)
    wl = dict(eqn="heat", nx=16, ny=16, dt=dt, dx=dx, nsteps=3, state=W.heat_sine(16, 16))
    bench.oracle_sample(wl, 1e-9)  # one chunk: starts the OpenMP threads
    rate, steps, secs = bench.oracle_sample(wl, 0.2)
    assert steps > wl["nsteps"] and secs >= 0.2 and rate > 0


def test_hbm_peak_prefers_the_measured_value(tmp_path, monkeypatch):
    import bench
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.hbm_peak_gbs() == (bench.HBM_FALLBACK_GBS, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6502.2}))
    assert bench.hbm_peak_gbs() == (6502.2, "measured")


def test_traffic_needs_a_capture_of_the_current_sources(tmp_path):
    """A DRAM traffic figure is used only if it was captured on the kernel
    sources as they stand: any other digest reads as no figure (null)."""
    import bench
    path = tmp_path / "dram.csv"
    digest = bench.kernel_source_digest()
    path.write_text("workload,kernel,dram_read_bytes,dram_write_bytes,sources,command\n"
                    "heat_x,octahedron,100,28,%s,ncu ...\n"
                    "heat_x,bridges,7,1,0123456789abcdef,ncu ...\n" % digest)
    assert bench.traffic_per_launch("heat_x", "octahedron", str(path)) == 128
    assert bench.traffic_per_launch("heat_x", "bridges", str(path)) is None
    assert bench.traffic_per_launch("heat_y", "octahedron", str(path)) is None
    assert bench.traffic_per_launch("heat_x", "octahedron", str(tmp_path / "none.csv")) is None
    assert len(digest) == 16 and digest == bench.kernel_source_digest()


def test_default_workload_is_the_large_heat_grid():
    import bench
    assert bench.DEFAULT_WORKLOAD == "heat16384"


def test_roofline_of_the_dominant_kernel(monkeypatch):
    """achieved = algorithmic flops of one launch of the dominant kernel over its
    mean live launch time; frac = achieved over the measured FP64 peak."""
    import bench
    monkeypatch.setattr(bench, "traffic_per_launch", lambda name, kernel: None)
    wl = dict(name="heat_x", eqn="heat", nx=256, ny=256, tile=64, depth=30)
    prof = {"up_pyramid": (0.01, 1), "bridges": (2.0, 4), "octahedron": (3.0, 4),
            "down_pyramid": (0.2, 1), "standard": (0.0, 0)}
    fp64 = {"peak_tflops": 1.2}
    r = bench.roofline(wl, prof, fp64)
    assert r["kernel"] == "octahedron" and r["bound"] == "alu" and r["traffic"] is None
    flops = bench.shape_cells("heat", 64, 30, "octahedron", 16) * 7
    assert r["flops_per_launch"] == flops
    assert abs(r["achieved"] - flops / 0.75e-3 / 1e12) < 1e-4
    assert abs(r["frac"] - r["achieved"] / 1.2) < 1e-4
    assert "hbm" not in r


def test_sweep_plans_are_legal_geometries():
    """bench.py --sweep: every (grid, tile, depth, cluster) of a plan is a
    geometry sweep_create accepts; edges that do not divide 16384 run on the
    largest multiple of the edge below it."""
    import bench
    from paper_2105_10332_b300 import sweep as S
    S.lib()
    for name, nx, eqn in (("heat16384", 16384, "heat"), ("heat64", 64, "heat"),
                          ("euler256", 256, "euler")):
        cfgs = bench.sweep_configs(dict(nx=nx, eqn=eqn), bench.SWEEP_PLANS[name])
        assert cfgs
        for n, b, d, c in cfgs:
            assert n % b == 0 and n // b >= 2 and n <= nx
            h = S.sweep_create(S.SWEEP_HEAT if eqn == "heat" else S.SWEEP_EULER, n, n, 1e-6,
                               1.0 / n, b, d)
            S.sweep_destroy(h)
    tiles = {b: n for n, b, _, _ in bench.sweep_configs(dict(nx=16384, eqn="heat"),
                                                       bench.SWEEP_PLANS["heat16384"])}
    assert tiles[12] == 16380 and tiles[24] == 16368 and tiles[64] == 16384


def test_standard_edge_plans_are_legal():
    """bench.py --sweep --sweep-standard: every Standard block edge of a plan
    is one the library accepts on that workload's grid."""
    import bench
    from paper_2105_10332_b300 import sweep as S
    for name, plan in bench.SWEEP_PLANS.items():
        wl = bench.workload(name)
        s = S.Solver(wl["eqn"], wl["nx"], wl["ny"], wl["dt"], wl["dx"], wl["tile"], wl["depth"])
        assert int(s.get("standard_tile")) in plan["standard_tiles"], name
        for t in plan["standard_tiles"]:
            s.set("standard_tile", t)
            assert s.get("standard_tile") == t
    # --sides: the heat workload on other grid sides, every edge legal there
    wl = bench.workload("heat16384")
    for n in bench.HEAT_SIDE_STEPS:
        w = bench.side_workload(wl, n)
        assert w["state"].shape == (n, n) and w["nsteps"] == bench.HEAT_SIDE_STEPS[n]
        s = S.Solver("heat", n, n, w["dt"], w["dx"], w["tile"], w["depth"])
        assert abs(s.get("r") - 0.1) < 1e-15
        for t in bench.SWEEP_PLANS["heat16384"]["standard_tiles"]:
            s.set("standard_tile", t)
