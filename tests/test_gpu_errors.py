"""Error reporting on the GPU, without a GPU fault.

The device error word: a state that holds a NaN makes the kernels that
write the state set SWEEP_DEV_NONFINITE, which sweep_check (or a run with
"check" set) reports as SWEEP_EDEVICE; a finite run leaves the word clear.
The batch stream pool: a stream or event creation made to fail on the host
returns SWEEP_ECUDA and leaves nothing behind, and the next call builds the
pool and runs.  The launch-geometry bit is not provoked: that would take a
deliberately wrong launch.  The L2 fetch-granularity setting (a
process-wide CUDA limit) runs in a fresh process of its own.
"""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2105_10332_b300 import workloads as W

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_10332_b300 import build
    build.build()
    return torch


@pytest.mark.parametrize("method", ["run_swept", "run_standard"])
def test_nonfinite_state_sets_the_error_word(torch_cuda, method):
    torch = torch_cuda
    from paper_2105_10332_b300 import sweep as S
    dt, dx = W.heat_dt(64, 0.1)
    s = S.Solver("heat", 64, 64, dt, dx, 16, 6)
    u0 = W.heat_modes(64, 64, seed=3)
    u = torch.from_numpy(u0).cuda()
    getattr(s, method)(u, 9)
    assert s.check() == 0
    bad = u0.copy()
    bad[17, 40] = np.nan
    u = torch.from_numpy(bad).cuda()
    getattr(s, method)(u, 9)
    assert s.check() & S.SWEEP_DEV_NONFINITE
    assert s.check() == 0  # sweep_check clears the word
    # with "check" set the run itself waits and reports
    s.set("check", 1)
    u = torch.from_numpy(bad).cuda()
    with pytest.raises(S.SweepError) as e:
        getattr(s, method)(u, 9)
    assert e.value.status == S.SWEEP_EDEVICE
    u = torch.from_numpy(u0).cuda()
    getattr(s, method)(u, 9)  # finite again: the run clears the word on entry


def test_euler_nan_reported_by_static_run(torch_cuda):
    torch = torch_cuda
    from paper_2105_10332_b300 import sweep as S
    q0, dx = W.vortex(64)
    dt, _ = W.vortex_dt(q0, dx, 1.0)
    h = S.sweep_create(S.SWEEP_EULER, 64, 64, dt, dx, 32, 6)
    try:
        S.sweep_set_param(h, "check", 1)
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        q = torch.from_numpy(q0).cuda()
        assert S.sweep_run_swept_static(h, ctypes.c_void_p(q.data_ptr()), 7, stream) == S.SWEEP_OK
        bad = q0.copy()
        bad[0, 5, 5] = -1.0  # negative density: the sound speed is a NaN
        q = torch.from_numpy(bad).cuda()
        rc = S.sweep_run_swept_static(h, ctypes.c_void_p(q.data_ptr()), 7, stream)
        assert rc == S.SWEEP_EDEVICE
    finally:
        S.sweep_destroy(h)


POOL_SCRIPT = r"""
import sys
sys.path.insert(0, %r)
import torch
from paper_2105_10332_b300 import sweep as S, workloads as W
dt, dx = W.heat_dt(64, 0.1)
solvers = [S.Solver("heat", 64, 64, dt, dx, 16, 6) for _ in range(3)]
init = torch.from_numpy(W.heat_modes(64, 64, seed=8)).cuda()
ref = init.clone()
solvers[0].run_swept(ref, 11)
states = [init.clone() for _ in solvers]
b = S.Batch(solvers, states, 11)
live = S.sweep_live_cuda_objects()
S.sweep_inject_fault(S.SWEEP_SITE_STREAM_POOL, 6)  # the 6th stream/event of the pool fails
try:
    b.run()
    raise SystemExit("no failure")
except S.SweepError as e:
    assert e.status == S.SWEEP_ECUDA, e
assert S.sweep_live_cuda_objects() == live, (S.sweep_live_cuda_objects(), live)
for st in states:
    st.copy_(init)
b.run()  # the pool is built this time
torch.cuda.synchronize()
assert S.sweep_live_cuda_objects() == live + 33
assert all(torch.equal(st, ref) for st in states)
print("pool ok")
"""


def test_batch_pool_failure_leaks_nothing(torch_cuda):
    """Run in a fresh process: the pool is built on a device's first batch."""
    out = subprocess.run([sys.executable, "-c", POOL_SCRIPT % ROOT], capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0 and "pool ok" in out.stdout, out.stdout + out.stderr


L2_SCRIPT = r"""
import sys
sys.path.insert(0, %r)
import torch
from paper_2105_10332_b300 import sweep as S, workloads as W
out = {}
for setting in (0, 32):
    dt, dx = W.heat_dt(256, 0.1)
    h = S.Solver("heat", 256, 256, dt, dx, 64, 30, l2_fetch_bytes=setting)
    u = torch.from_numpy(W.heat_modes(256, 256, seed=4)).cuda()
    h.run_swept(u, 23)
    q0, ex = W.vortex(128)
    edt, _ = W.vortex_dt(q0, ex, 1.0)
    e = S.Solver("euler", 128, 128, edt, ex, 32, 6, l2_fetch_bytes=setting)
    q = torch.from_numpy(q0).cuda()
    e.run_swept(q, 9)
    torch.cuda.synchronize()
    out[setting] = (u.cpu(), q.cpu())
    assert e.get("l2_fetch_bytes") == setting
assert torch.equal(out[0][0], out[32][0]) and torch.equal(out[0][1], out[32][1])
print("l2 ok")
"""


def test_l2_fetch_setting_keeps_the_bits(torch_cuda):
    out = subprocess.run([sys.executable, "-c", L2_SCRIPT % ROOT], capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0 and "l2 ok" in out.stdout, out.stdout + out.stderr


CHECKED_SCRIPT = r"""
import sys
sys.path.insert(0, %r)
import numpy as np, torch
import oracle
from paper_2105_10332_b300 import sweep as S, workloads as W
assert S.LIB_PATH.endswith("libsweep_checked.so")
dt, dx = W.heat_dt(64, 0.1)
h = S.Solver("heat", 64, 64, dt, dx, 16, 6, check=1)
u0 = W.heat_modes(64, 64, seed=9)
for method in ("run_swept", "run_standard"):
    u = torch.from_numpy(u0).cuda()
    getattr(h, method)(u, 13)
    assert np.array_equal(u.cpu().numpy(), oracle.heat_run(u0, 13, dt, dx)), method
q0, ex = W.vortex(64)
edt, _ = W.vortex_dt(q0, ex, 1.0)
e = S.Solver("euler", 64, 64, edt, ex, 32, 6, check=1)
for method in ("run_swept", "run_standard"):
    q = torch.from_numpy(q0).cuda()
    getattr(e, method)(q, 7)
    assert np.array_equal(q.cpu().numpy(), oracle.euler_run(q0, edt, ex, 7)), method
print("checked ok")
"""


def test_checked_build_verifies_its_launches(torch_cuda):
    """The checked build (every kernel verifies its grid, block and shared
    memory at entry) runs the same bits as the oracle with "check" set, so
    every run reads back a clear device error word."""
    from paper_2105_10332_b300 import build
    env = dict(os.environ, SWEEP_LIBRARY=build.LIB_CHECKED)
    out = subprocess.run([sys.executable, "-c", CHECKED_SCRIPT % ROOT], capture_output=True,
                         text=True, timeout=300, env=env)
    assert out.returncode == 0 and "checked ok" in out.stdout, out.stdout + out.stderr
