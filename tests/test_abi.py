"""C-ABI checks that need no GPU: the library loads, exports every symbol the
header declares, validates arguments and sizes its workspace.  No call here
reaches a kernel."""
import ctypes
import os
import re

import pytest

from paper_2105_10332_b300 import build as sbuild
from paper_2105_10332_b300 import sweep as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    sbuild.build()
    return S.lib()


def header_functions():
    text = open(os.path.join(ROOT, "include", "sweep.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sweep_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(L):
    names = header_functions()
    assert "sweep_run_swept" in names and "sweep_create" in names
    for n in names:
        assert hasattr(L, n), n
        assert n in S.SIGNATURES, n


def test_create_validates_geometry(L):
    good = dict(eqn=S.SWEEP_HEAT, nx=64, ny=64, dt=1e-5, dx=1 / 64, tile=16, depth=6)
    h = S.sweep_create(**good)
    assert S.sweep_get_param(h, "depth") == 6
    S.sweep_destroy(h)
    bad = [dict(eqn=2), dict(tile=15), dict(tile=2), dict(tile=24), dict(nx=16),
           dict(depth=7), dict(depth=8), dict(depth=1), dict(dt=0.0), dict(dx=-1.0),
           dict(dt=float("nan")), dict(eqn=S.SWEEP_EULER, tile=8), dict(eqn=S.SWEEP_EULER, depth=4),
           dict(eqn=S.SWEEP_EULER, tile=64)]
    for b in bad:
        args = dict(good, **b)
        with pytest.raises(S.SweepError) as e:
            S.sweep_create(**args)
        assert e.value.status == S.SWEEP_EINVAL, b


def test_depth_zero_picks_largest_even(L):
    for eqn, tile, expect in ((S.SWEEP_HEAT, 16, 6), (S.SWEEP_HEAT, 32, 14), (S.SWEEP_HEAT, 12, 4),
                              (S.SWEEP_EULER, 32, 6), (S.SWEEP_EULER, 16, 2), (S.SWEEP_EULER, 20, 4)):
        h = S.sweep_create(eqn, 4 * tile, 2 * tile, 1e-4, 0.01, tile, 0)
        assert S.sweep_get_param(h, "depth") == expect
        S.sweep_destroy(h)


def test_params_and_workspace(L):
    h = S.sweep_create(S.SWEEP_EULER, 96, 64, 1e-3, 0.1, 32, 4)
    assert S.sweep_get_param(h, "gamma") == 1.4
    S.sweep_set_param(h, "gamma", 5.0 / 3.0)
    assert S.sweep_get_param(h, "gamma") == 5.0 / 3.0
    S.sweep_set_param(h, "limiter", 1)
    for key, val in (("gamma", 1.0), ("limiter", 3), ("nope", 1.0), ("standard_tile", 7),
                     ("standard_tile", 48)):
        with pytest.raises(S.SweepError):
            S.sweep_set_param(h, key, val)
    assert S.sweep_get_param(h, "ncomp") == 4 and S.sweep_get_param(h, "radius") == 2
    # (depth + 1) slots of one state, 256-byte padded, plus a 256-byte header
    slot = (4 * 96 * 64 * 8 + 255) // 256 * 256
    assert S.sweep_workspace_bytes(h) == 256 + 5 * slot
    S.sweep_destroy(h)


def test_run_rejects_bad_pointers_before_any_launch(L):
    h = S.sweep_create(S.SWEEP_HEAT, 64, 64, 1e-5, 1 / 64, 16, 6)
    for fn in (S.sweep_run_swept, S.sweep_run_standard):
        assert fn(h, None, 1, ctypes.c_void_p(4096), None) == S.SWEEP_EINVAL
        assert fn(h, ctypes.c_void_p(4096), 1, None, None) == S.SWEEP_EINVAL
        assert fn(h, ctypes.c_void_p(4104), 1, ctypes.c_void_p(4096), None) == S.SWEEP_EINVAL
        assert fn(h, ctypes.c_void_p(4096), 1, ctypes.c_void_p(4352 + 8), None) == S.SWEEP_EINVAL
        assert fn(h, ctypes.c_void_p(4096), -1, ctypes.c_void_p(4096), None) == S.SWEEP_EINVAL
    S.sweep_destroy(h)
    assert S.error_string(S.SWEEP_ETIMEOUT) == "device wait timed out"


def test_every_status_has_its_own_message(L):
    codes = (S.SWEEP_OK, S.SWEEP_EINVAL, S.SWEEP_ENOMEM, S.SWEEP_ECUDA, S.SWEEP_ETIMEOUT,
             S.SWEEP_EUNSUPPORTED, S.SWEEP_EDEVICE)
    msgs = [S.error_string(c) for c in codes]
    assert len(set(msgs)) == len(codes) and "unknown status" not in msgs
    assert S.error_string(99) == "unknown status"


def test_injected_host_allocation_failure(L):
    """sweep_create's handle allocation, made to fail on the host: SWEEP_ENOMEM,
    nothing is returned, and the next create succeeds (the fault disarms)."""
    live = S.sweep_live_cuda_objects()
    S.sweep_inject_fault(S.SWEEP_SITE_HOST_ALLOC, 2)
    h1 = S.sweep_create(S.SWEEP_HEAT, 64, 64, 1e-5, 1 / 64, 16, 6)  # first pass: fine
    with pytest.raises(S.SweepError) as e:
        S.sweep_create(S.SWEEP_HEAT, 64, 64, 1e-5, 1 / 64, 16, 6)   # second: fails
    assert e.value.status == S.SWEEP_ENOMEM
    h3 = S.sweep_create(S.SWEEP_EULER, 64, 64, 1e-3, 0.1, 32, 6)
    S.sweep_destroy(h1)
    S.sweep_destroy(h3)
    assert S.sweep_live_cuda_objects() == live
    for site, nth in ((7, 1), (S.SWEEP_SITE_EVENTS, -1)):
        with pytest.raises(S.SweepError):
            S.sweep_inject_fault(site, nth)
    S.sweep_inject_fault(0, 0)


def test_check_parameter(L):
    h = S.sweep_create(S.SWEEP_HEAT, 64, 64, 1e-5, 1 / 64, 16, 6)
    assert S.sweep_get_param(h, "check") == 0
    S.sweep_set_param(h, "check", 1)
    assert S.sweep_get_param(h, "check") == 1
    with pytest.raises(S.SweepError):
        S.sweep_set_param(h, "check", 2)
    for bad in (16, 48, 256, -32):
        with pytest.raises(S.SweepError) as e:
            S.sweep_set_param(h, "l2_fetch_bytes", bad)
        assert e.value.status == S.SWEEP_EINVAL
    S.sweep_set_param(h, "l2_fetch_bytes", 0)  # 0 leaves the context untouched: no CUDA call
    assert S.sweep_get_param(h, "l2_fetch_bytes") == 0
    S.sweep_destroy(h)
    assert S.sweep_check(None, None)[0] == S.SWEEP_EINVAL


def test_adjoint_workspace_and_argument_checks(L):
    h = S.sweep_create(S.SWEEP_EULER, 64, 64, 1e-3, 0.1, 32, 6)
    slot = (4 * 64 * 64 * 8 + 255) // 256 * 256
    # level store (7 slots) + 32 checkpoints + 64-step segment + its 64 first
    # stages Q* + mu* + per-cell pressure terms (4) + limiter terms (12) + faces
    # (per axis: 8 state gradients and 4 pressure adjoints)
    nseg = (2000 + 63) // 64
    plane = 64 * 64 * 8
    expect = (256 + slot * 7 + slot * nseg + slot * 64 + slot * 64 + slot + 4 * plane
              + 12 * plane + 24 * plane)
    assert S.sweep_adjoint_workspace_bytes(h, 2000, 64) == expect
    assert S.sweep_adjoint_workspace_bytes(h, 2000, 0) == 0
    p = ctypes.c_void_p(4096)
    assert S.sweep_adjoint(h, None, p, ctypes.c_void_p(8192), 5, 4, p, None) == S.SWEEP_EINVAL
    assert S.sweep_adjoint(h, p, p, p, 5, 4, p, None) == S.SWEEP_EINVAL  # lam0 aliases lamT
    assert S.sweep_adjoint(h, p, p, ctypes.c_void_p(8192), 5, 0, p, None) == S.SWEEP_EINVAL
    S.sweep_destroy(h)
    hh = S.sweep_create(S.SWEEP_HEAT, 64, 64, 1e-5, 1 / 64, 16, 6)
    assert S.sweep_adjoint_workspace_bytes(hh, 100, 64) == S.sweep_workspace_bytes(hh)
    S.sweep_destroy(hh)


def test_heat_coefficient_matches_the_oracle(L, oracle_lib):
    """The library's heat coefficient r = alpha dt / dx^2 (App. A) is the
    oracle's, bit for bit, for the workloads' sides (powers of two and not)
    and diffusivities other than 1: both evaluate the formula as written."""
    from paper_2105_10332_b300 import workloads as W
    for n, tile in ((64, 16), (48, 12), (72, 12), (80, 20), (96, 16), (4096, 64), (16384, 64)):
        for alpha, r in ((1.0, 0.1), (0.7, 0.2), (2.5, 0.05)):
            dt, dx = W.heat_dt(n, r, alpha)
            h = S.sweep_create(S.SWEEP_HEAT, n, n, dt, dx, tile, 0)
            S.sweep_set_param(h, "alpha", alpha)
            assert S.sweep_get_param(h, "r") == oracle_lib.heat_r(dt, dx, alpha), (n, alpha)
            S.sweep_destroy(h)


def test_autotune_candidates_are_legal():
    from paper_2105_10332_b300 import autotune
    for eqn in ("heat", "euler"):
        for side in (64, 96, 160, 512, 2048):
            c = autotune.candidates(eqn, side)
            assert c, (eqn, side)
            for cfg in c:
                assert side % cfg["tile"] == 0 and side // cfg["tile"] >= 2
                n = 1 if eqn == "heat" else 2
                assert 2 <= cfg["depth"] <= cfg["tile"] // (2 * n) - 1 and cfg["depth"] % 2 == 0
    assert autotune.size_class(96) == 128 and autotune.size_class(64) == 64


def test_autotuner_gives_every_batch_side_a_legal_config():
    """The 256 sides of the batched workload (multiples of 32 in [64, 2048]),
    both equations: a size class first tuned on a side that admits tile 64
    (e.g. 384) must not hand tile 64 to a later side of the class it does not
    divide (e.g. 352).  The timer is a stand-in that prefers the largest tile
    and cannot build one configuration in three; no GPU is used."""
    from paper_2105_10332_b300 import autotune, workloads as W
    calls = []

    def measure(cfg):
        calls.append(cfg)
        if (cfg["tile"] + cfg["depth"]) % 3 == 0:
            return None
        return 100.0 / cfg["tile"] + 0.01 * cfg["depth"]

    tuner = autotune.Autotuner()
    sides = W.batch_sides(256)
    for k, side in enumerate(sides):
        eqn = "heat" if k % 2 == 0 else "euler"
        cfg = tuner.select(eqn, side, measure)
        assert cfg in autotune.candidates(eqn, side), (eqn, side, cfg)
        assert side % cfg["tile"] == 0 and side // cfg["tile"] >= 2
    assert None not in tuner.cache.values()
    assert len(calls) < 4 * len(sides)  # classes reuse their ranking
    with pytest.raises(RuntimeError):
        autotune.Autotuner().select("heat", 384, lambda cfg: None)


def test_batch_workspace_is_sum_of_instances(L):
    hs = [S.sweep_create(S.SWEEP_HEAT, 64, 64, 1e-5, 1 / 64, 16, 6),
          S.sweep_create(S.SWEEP_EULER, 96, 96, 1e-3, 0.1, 32, 6)]
    total = sum((S.sweep_workspace_bytes(h) + 255) // 256 * 256 for h in hs)
    assert S.sweep_batch_workspace_bytes(hs) == total
    for h in hs:
        S.sweep_destroy(h)


def test_standard_tile_default_fills_the_sms(L):
    """The default Standard block edge is the first preferred edge giving at
    least its minimum number of blocks (heat: 64 and 32 from 1024 blocks,
    smaller edges from 148, one per B300 SM), else the edge giving the
    most."""
    for eqn, nx, tile, expect in ((S.SWEEP_HEAT, 64, 16, 8), (S.SWEEP_HEAT, 128, 16, 8),
                                  (S.SWEEP_HEAT, 256, 32, 16), (S.SWEEP_HEAT, 512, 32, 16),
                                  (S.SWEEP_HEAT, 1024, 64, 32), (S.SWEEP_HEAT, 2048, 64, 64),
                                  (S.SWEEP_HEAT, 4096, 64, 64), (S.SWEEP_HEAT, 16384, 64, 64),
                                  (S.SWEEP_EULER, 256, 32, 16), (S.SWEEP_EULER, 64, 32, 8),
                                  (S.SWEEP_EULER, 1024, 32, 16), (S.SWEEP_HEAT, 72, 12, 8)):
        h = S.sweep_create(eqn, nx, nx, 1e-6, 1.0 / nx, tile, 0)
        assert S.sweep_get_param(h, "standard_tile") == expect, (eqn, nx)
        S.sweep_destroy(h)
    # no edge of the preferred list divides 56 x 84: the smallest even one that does
    h = S.sweep_create(S.SWEEP_HEAT, 56, 84, 1e-6, 1.0 / 56, 14, 0)
    assert S.sweep_get_param(h, "standard_tile") == 14
    S.sweep_destroy(h)



def test_euler_octahedron_cluster_default(L):
    """Euler Octahedra default to 2-CTA clusters while 2 CTAs per block fit one
    per SM (at most 74 blocks), else to single CTAs; heat to single CTAs."""
    for eqn, nx, tile, expect in ((S.SWEEP_EULER, 256, 32, 2), (S.SWEEP_EULER, 1024, 32, 1),
                                  (S.SWEEP_EULER, 64, 32, 2), (S.SWEEP_EULER, 320, 32, 1),
                                  (S.SWEEP_HEAT, 64, 16, 1)):
        h = S.sweep_create(eqn, nx, nx, 1e-6, 1.0 / nx, tile, 0)
        assert S.sweep_get_param(h, "cluster_oct") == expect, (eqn, nx)
        assert S.sweep_get_param(h, "cluster_bridges") == 1
        S.sweep_destroy(h)
