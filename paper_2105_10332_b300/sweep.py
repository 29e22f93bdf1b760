"""Python binding of the C ABI in include/sweep.h (libsweep.so).

Argument marshalling only: every step of the solver runs in the CUDA kernels
of libsweep.so.  There is no CPU fallback -- if the library is missing this
module raises.  PyTorch supplies device memory and streams.

Low-level functions carry the C names (``sweep_create``, ``sweep_run_swept``
...); ``Solver`` wraps a handle and its workspace.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# SWEEP_LIBRARY may name another build of the same library, e.g. the checked
# build libsweep_checked.so (kernels that also verify their launch geometry)
LIB_PATH = os.environ.get("SWEEP_LIBRARY") or os.path.join(HERE, "libsweep.so")

SWEEP_HEAT = 0
SWEEP_EULER = 1

SWEEP_OK = 0
SWEEP_EINVAL = 1
SWEEP_ENOMEM = 2
SWEEP_ECUDA = 3
SWEEP_ETIMEOUT = 4
SWEEP_EUNSUPPORTED = 5
SWEEP_EDEVICE = 6

SWEEP_DEV_LAUNCH = 1
SWEEP_DEV_NONFINITE = 2

SWEEP_SITE_HOST_ALLOC = 1
SWEEP_SITE_STREAM_POOL = 2
SWEEP_SITE_EVENTS = 3

# every symbol include/sweep.h declares: name -> (restype, argtypes)
_c_int, _c_i64, _c_dbl, _vp = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
SIGNATURES = {
    "sweep_create": (_c_int, [_c_int, _c_i64, _c_i64, _c_dbl, _c_dbl, _c_int, _c_int,
                              ctypes.POINTER(_vp)]),
    "sweep_set_param": (_c_int, [_vp, ctypes.c_char_p, _c_dbl]),
    "sweep_get_param": (_c_int, [_vp, ctypes.c_char_p, ctypes.POINTER(_c_dbl)]),
    "sweep_workspace_bytes": (ctypes.c_size_t, [_vp]),
    "sweep_run_swept": (_c_int, [_vp, _vp, _c_i64, _vp, _vp]),
    "sweep_run_standard": (_c_int, [_vp, _vp, _c_i64, _vp, _vp]),
    "sweep_run_swept_static": (_c_int, [_vp, _vp, _c_i64, _vp]),
    "sweep_adjoint_workspace_bytes": (ctypes.c_size_t, [_vp, _c_i64, _c_int]),
    "sweep_batch_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(_vp), _c_int]),
    "sweep_batch_run": (_c_int, [ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_c_i64),
                                 _c_int, _vp, _vp]),
    "sweep_adjoint": (_c_int, [_vp, _vp, _vp, _vp, _c_i64, _c_int, _vp, _vp]),
    "sweep_profile_read": (_c_int, [_vp, ctypes.POINTER(_c_dbl), ctypes.POINTER(_c_i64), _c_int]),
    "sweep_fp64_probe": (_c_int, [_vp, _c_i64, _c_int, _c_int, _vp]),
    "sweep_check": (_c_int, [_vp, ctypes.POINTER(ctypes.c_uint), _vp]),
    "sweep_inject_fault": (_c_int, [_c_int, _c_int]),
    "sweep_live_cuda_objects": (_c_int, []),
    "sweep_destroy": (None, [_vp]),
    "sweep_error_string": (ctypes.c_char_p, [_c_int]),
}

_lib = None


class SweepError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__("%s: %s (status %d)" % (what, error_string(status), status))


def lib():
    """Load libsweep.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libsweep.so is not built; run `python -m paper_2105_10332_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def error_string(status):
    return lib().sweep_error_string(int(status)).decode()


def _check(status, what):
    if status != SWEEP_OK:
        raise SweepError(status, what)


# ------------------------------------------------------------ C-named wrappers

def sweep_create(eqn, nx, ny, dt, dx, tile, depth=0):
    h = ctypes.c_void_p()
    _check(lib().sweep_create(int(eqn), int(nx), int(ny), float(dt), float(dx), int(tile),
                              int(depth), ctypes.byref(h)), "sweep_create")
    return h


def sweep_set_param(h, key, value):
    _check(lib().sweep_set_param(h, key.encode(), float(value)), "sweep_set_param(%s)" % key)


def sweep_get_param(h, key):
    v = ctypes.c_double()
    _check(lib().sweep_get_param(h, key.encode(), ctypes.byref(v)), "sweep_get_param(%s)" % key)
    return v.value


def sweep_workspace_bytes(h):
    return int(lib().sweep_workspace_bytes(h))


def sweep_run_swept(h, state_ptr, nsteps, ws_ptr, stream_ptr):
    return int(lib().sweep_run_swept(h, state_ptr, int(nsteps), ws_ptr, stream_ptr))


def sweep_run_standard(h, state_ptr, nsteps, ws_ptr, stream_ptr):
    return int(lib().sweep_run_standard(h, state_ptr, int(nsteps), ws_ptr, stream_ptr))


def sweep_run_swept_static(h, state_ptr, nsteps, stream_ptr):
    """Swept run with the library's fixed device scratch (no workspace, no allocation)."""
    return int(lib().sweep_run_swept_static(h, state_ptr, int(nsteps), stream_ptr))


STATIC_SCRATCH_BYTES = 16 << 20


def sweep_adjoint_workspace_bytes(h, nsteps, ckpt_every):
    return int(lib().sweep_adjoint_workspace_bytes(h, int(nsteps), int(ckpt_every)))


def sweep_adjoint(h, q0_ptr, lamT_ptr, lam0_ptr, nsteps, ckpt_every, ws_ptr, stream_ptr):
    return int(lib().sweep_adjoint(h, q0_ptr, lamT_ptr, lam0_ptr, int(nsteps), int(ckpt_every),
                                   ws_ptr, stream_ptr))


def sweep_profile_read(h, nkinds=5):
    ms = (ctypes.c_double * nkinds)()
    n = (ctypes.c_int64 * nkinds)()
    _check(lib().sweep_profile_read(h, ms, n, int(nkinds)), "sweep_profile_read")
    return list(ms), list(n)


def sweep_fp64_probe(out_ptr, iters, blocks, threads, stream_ptr):
    """Enqueue the FP64 fma-throughput probe (16 * iters * blocks * threads flops)."""
    return int(lib().sweep_fp64_probe(out_ptr, int(iters), int(blocks), int(threads), stream_ptr))


def sweep_check(ws_ptr, stream_ptr):
    """(status, bits) of the device error word of a workspace (waits for the stream)."""
    bits = ctypes.c_uint(0)
    rc = int(lib().sweep_check(ws_ptr, ctypes.byref(bits), stream_ptr))
    return rc, int(bits.value)


def sweep_inject_fault(site, nth):
    _check(lib().sweep_inject_fault(int(site), int(nth)), "sweep_inject_fault")


def sweep_live_cuda_objects():
    return int(lib().sweep_live_cuda_objects())


def sweep_destroy(h):
    lib().sweep_destroy(h)


KERNEL_KINDS = ("up_pyramid", "bridges", "octahedron", "down_pyramid", "standard")


# ------------------------------------------------------------------ Solver

class Solver:
    """A swept-rule solver for one grid.

    eqn: "heat" or "euler" (or SWEEP_HEAT / SWEEP_EULER).  States are torch
    float64 tensors of shape [ny, nx] (heat) or [4, ny, nx] (Euler), advanced
    in place.  Device tensors run on the current torch stream; host tensors
    are copied to the device and back (the end-to-end path).
    """

    def __init__(self, eqn, nx, ny, dt, dx, tile, depth=0, **params):
        if isinstance(eqn, str):
            eqn = {"heat": SWEEP_HEAT, "euler": SWEEP_EULER}[eqn]
        self.eqn = eqn
        self.nx, self.ny = int(nx), int(ny)
        self._h = sweep_create(eqn, nx, ny, dt, dx, tile, depth)
        for k, v in params.items():
            sweep_set_param(self._h, k, v)
        self.tile = int(self.get("tile"))
        self.depth = int(self.get("depth"))
        self.ncomp = int(self.get("ncomp"))
        self._ws = None

    def get(self, key):
        return sweep_get_param(self._h, key)

    def set(self, key, value):
        sweep_set_param(self._h, key, value)

    @property
    def workspace_bytes(self):
        return sweep_workspace_bytes(self._h)

    def workspace(self, device):
        import torch
        if self._ws is None or self._ws.device != torch.device(device):
            self._ws = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=device)
        return self._ws

    def _shape(self):
        return (self.ny, self.nx) if self.ncomp == 1 else (self.ncomp, self.ny, self.nx)

    def _run(self, fn, state, nsteps, ws=None):
        import torch
        if tuple(state.shape) != self._shape() or state.dtype != torch.float64:
            raise ValueError("state must be float64 of shape %s" % (self._shape(),))
        if not state.is_cuda:
            dev = state.new_empty(state.shape, device="cuda")
            dev.copy_(state, non_blocking=True)
            self._run(fn, dev, nsteps, ws)
            state.copy_(dev, non_blocking=False)
            return state
        if not state.is_contiguous():
            raise ValueError("state must be contiguous")
        ws = self.workspace(state.device) if ws is None else ws
        stream = torch.cuda.current_stream(state.device).cuda_stream
        rc = fn(self._h, ctypes.c_void_p(state.data_ptr()), nsteps, ctypes.c_void_p(ws.data_ptr()),
                ctypes.c_void_p(stream))
        _check(rc, fn.__name__)
        return state

    def run_swept(self, state, nsteps, ws=None):
        """Advance `state` by nsteps with the swept rule (bit-identical to run_standard)."""
        return self._run(sweep_run_swept, state, nsteps, ws)

    def run_standard(self, state, nsteps, ws=None):
        """Advance `state` by nsteps with one kernel per RK2 step."""
        return self._run(sweep_run_standard, state, nsteps, ws)

    def adjoint(self, q0, lamT, nsteps, ckpt_every=64):
        """dL/dQ^0 given lamT = dL/dQ^N (device tensors of the state shape); returns a
        new tensor.  q0 is the initial state (not read for heat)."""
        import torch
        if tuple(lamT.shape) != self._shape() or lamT.dtype != torch.float64 or not lamT.is_cuda:
            raise ValueError("lamT must be a float64 CUDA tensor of shape %s" % (self._shape(),))
        lamT = lamT.contiguous()
        q0 = lamT if q0 is None else q0.contiguous()
        lam0 = torch.empty_like(lamT)
        nbytes = sweep_adjoint_workspace_bytes(self._h, nsteps, ckpt_every)
        ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=lamT.device)
        stream = torch.cuda.current_stream(lamT.device).cuda_stream
        rc = sweep_adjoint(self._h, ctypes.c_void_p(q0.data_ptr()), ctypes.c_void_p(lamT.data_ptr()),
                           ctypes.c_void_p(lam0.data_ptr()), nsteps, ckpt_every,
                           ctypes.c_void_p(ws.data_ptr()), ctypes.c_void_p(stream))
        _check(rc, "sweep_adjoint")
        return lam0

    def check(self, ws=None):
        """Bits of the device error word of this solver's workspace (0: none);
        waits for the current stream and clears the word."""
        import torch
        ws = self._ws if ws is None else ws
        if ws is None:
            return 0
        stream = torch.cuda.current_stream(ws.device).cuda_stream
        rc, bits = sweep_check(ctypes.c_void_p(ws.data_ptr()), ctypes.c_void_p(stream))
        if rc not in (SWEEP_OK, SWEEP_EDEVICE):
            _check(rc, "sweep_check")
        return bits

    def profile(self):
        """{kind: (total ms, launches)} of the launches recorded since profiling was enabled."""
        ms, n = sweep_profile_read(self._h, len(KERNEL_KINDS))
        return {k: (ms[i], n[i]) for i, k in enumerate(KERNEL_KINDS)}

    def close(self):
        if getattr(self, "_h", None) is not None:
            sweep_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sweep_batch_workspace_bytes(handles):
    arr = (ctypes.c_void_p * len(handles))(*[h.value for h in handles])
    return int(lib().sweep_batch_workspace_bytes(arr, len(handles)))


def sweep_batch_run(handles, state_ptrs, nsteps, ws_ptr, stream_ptr):
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*[h.value for h in handles])
    ps = (ctypes.c_void_p * n)(*state_ptrs)
    ns = (ctypes.c_int64 * n)(*[int(x) for x in nsteps])
    return int(lib().sweep_batch_run(hs, ps, ns, n, ws_ptr, stream_ptr))


class Batch:
    """Many independent solvers advanced together (sweep_batch_run), optionally
    captured once into a CUDA graph and replayed."""

    def __init__(self, solvers, states, nsteps):
        import torch
        self.solvers = list(solvers)
        self.states = list(states)
        self.nsteps = [int(n) for n in (nsteps if hasattr(nsteps, "__len__") else
                                          [nsteps] * len(self.solvers))]
        for s, st in zip(self.solvers, self.states):
            if tuple(st.shape) != s._shape() or st.dtype != torch.float64 or not st.is_cuda:
                raise ValueError("each state must be a float64 CUDA tensor of its solver's shape")
        self._handles = [s._h for s in self.solvers]
        nbytes = sweep_batch_workspace_bytes(self._handles)
        self.ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.states[0].device)
        self.graph = None

    def _launch(self, stream):
        rc = sweep_batch_run(self._handles, [t.data_ptr() for t in self.states], self.nsteps,
                             ctypes.c_void_p(self.ws.data_ptr()), ctypes.c_void_p(stream))
        _check(rc, "sweep_batch_run")

    def run(self):
        import torch
        self._launch(torch.cuda.current_stream(self.states[0].device).cuda_stream)

    def capture(self):
        """Record one batch into a CUDA graph (replay() then runs it with one launch)."""
        import torch
        self.run()  # first call creates the stream pool and sets kernel attributes
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._launch(torch.cuda.current_stream().cuda_stream)
        return self.graph

    def replay(self):
        self.graph.replay()


def _autograd_function():
    import torch

    class SweptRun(torch.autograd.Function):
        """Q^N = swept(Q^0, nsteps); backward runs the discrete adjoint."""

        @staticmethod
        def forward(ctx, q0, solver, nsteps, ckpt_every):
            ctx.solver, ctx.nsteps, ctx.ckpt = solver, int(nsteps), int(ckpt_every)
            ctx.save_for_backward(q0)
            q = q0.detach().clone().contiguous()
            solver.run_swept(q, nsteps)
            return q

        @staticmethod
        def backward(ctx, grad):
            (q0,) = ctx.saved_tensors
            g = ctx.solver.adjoint(q0.detach(), grad.contiguous(), ctx.nsteps, ctx.ckpt)
            return g, None, None, None

    return SweptRun


_SweptRun = None


def swept_run(q0, solver, nsteps, ckpt_every=64):
    """Differentiable swept run: gradients of any loss of the result with
    respect to q0 come from the discrete adjoint (sweep_adjoint)."""
    global _SweptRun
    if _SweptRun is None:
        _SweptRun = _autograd_function()
    return _SweptRun.apply(q0, solver, nsteps, ckpt_every)
