"""The allocation-free swept run, sweep_run_swept_static.

It serves callers that cannot allocate device memory when they advance a
state (an application that owns all GPU memory through its own pool, or a
loop where an allocation and its possible failure are not acceptable): the
level store lives in a fixed array inside the library instead of a
caller-provided workspace.  Its output must equal sweep_run_swept's, bit for
bit (the bar every Swept comparison in this suite uses), over consecutive
calls that reuse the array whatever an earlier call left in it.
"""
import ctypes

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


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_static_scratch_run_matches_workspace_run(torch_cuda):
    torch = torch_cuda
    from paper_2105_10332_b300 import sweep as S
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    # Euler vortex 256^2, block 32, depth 6: the benchmark's solver (14 MiB of levels)
    q0, dx = W.vortex(256, xc=0.5, yc=-0.25)
    dt, _ = W.vortex_dt(q0, dx, 10.0)
    he = S.sweep_create(S.SWEEP_EULER, 256, 256, dt, dx, 32, 6)
    assert S.sweep_workspace_bytes(he) <= S.STATIC_SCRATCH_BYTES
    # heat 64^2, block 16, depth 6: a second problem that leaves other data in the array
    hd, hdx = W.heat_dt(64, 0.1)
    hh = S.sweep_create(S.SWEEP_HEAT, 64, 64, hd, hdx, 16, 6)
    try:
        a = torch.from_numpy(q0).cuda()
        b = a.clone()
        ws = torch.empty(S.sweep_workspace_bytes(he), dtype=torch.uint8, device="cuda")
        u0 = torch.from_numpy(W.heat_modes(64, 64, seed=5)).cuda()
        ua, ub = u0.clone(), u0.clone()
        wsh = torch.empty(S.sweep_workspace_bytes(hh), dtype=torch.uint8, device="cuda")
        for call in range(2):  # two calls in a row, each continuing the last state
            n = 37 + 4 * call  # 37 steps, then 41 (different leftover Standard steps)
            assert S.sweep_run_swept(he, _p(a), n, _p(ws), stream) == S.SWEEP_OK
            assert S.sweep_run_swept_static(he, _p(b), n, stream) == S.SWEEP_OK
            torch.cuda.synchronize()
            assert torch.equal(a, b), "call %d differs (max %.3g)" % (
                call, float((a - b).abs().max()))
            assert S.sweep_run_swept(hh, _p(ua), 29, _p(wsh), stream) == S.SWEEP_OK
            assert S.sweep_run_swept_static(hh, _p(ub), 29, stream) == S.SWEEP_OK
            torch.cuda.synchronize()
            assert torch.equal(ua, ub), "heat call %d differs" % call
        assert not torch.equal(a, torch.from_numpy(q0).cuda())
        # once the library's module is loaded (the calls above), further
        # calls leave the device's free memory exactly as it was
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(2):
            assert S.sweep_run_swept_static(he, _p(b), 7, stream) == S.SWEEP_OK
            assert S.sweep_run_swept_static(hh, _p(ub), 5, stream) == S.SWEEP_OK
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
    finally:
        S.sweep_destroy(he)
        S.sweep_destroy(hh)


def test_static_scratch_rejects_oversized_problems(torch_cuda):
    from paper_2105_10332_b300 import sweep as S
    torch = torch_cuda
    dt, dx = W.heat_dt(1024, 0.1)
    h = S.sweep_create(S.SWEEP_HEAT, 1024, 1024, dt, dx, 32, 14)  # 15 slots of 8 MiB
    try:
        assert S.sweep_workspace_bytes(h) > S.STATIC_SCRATCH_BYTES
        u = torch.zeros(1024, 1024, dtype=torch.float64, device="cuda")
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        assert S.sweep_run_swept_static(h, _p(u), 1, stream) == S.SWEEP_EINVAL
    finally:
        S.sweep_destroy(h)
