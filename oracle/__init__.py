"""CPU oracle for the swept-rule solver -- TEST INFRASTRUCTURE ONLY.

A plain, slow fp64 C reference (``sweep_oracle.c``) loaded through ctypes.
Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the product path never does.  It shares
no code with the CUDA library.

Functions (each follows the passage cited in the C source):
  heat_r         -- App. A mesh ratio r = alpha dt / dx^2 from the physical inputs
  heat_run       -- App. A heat update, RK2 midpoint (scheme 0) or forward Euler (1)
  euler_run      -- App. B Euler scheme: pressure minmod, Rusanov-form flux, RK2
  swept_replay   -- the Sec. 3.3 phase schedule replayed cell by cell with
                    dependency checks (Eq. 1 bounds the depth)
  heat_adjoint, euler_adjoint -- discrete adjoints (reverse mode) of the two
                    schemes, with checkpointing for Euler
  face_flux, limiter, state_flux, cell_pressure -- single-face and single-cell
                    pieces used by the pins
"""
import ctypes

import numpy as np

from . import build as _build

_lib = None

ERRORS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "read of an unavailable value",
          4: "value computed twice", 5: "value never computed"}


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        i64 = ctypes.c_int64
        dbl = ctypes.c_double
        L.oracle_heat_r.argtypes = [dbl, dbl, dbl]
        L.oracle_heat_r.restype = dbl
        L.oracle_heat_run.argtypes = [i64, i64, dbl, dbl, dbl, ctypes.c_int, dp, i64]
        L.oracle_heat_run.restype = ctypes.c_int
        L.oracle_euler_run.argtypes = [i64, i64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int, dp, i64]
        L.oracle_euler_run.restype = ctypes.c_int
        L.oracle_face_flux.argtypes = [dp, dp, dp, dp, ctypes.c_double, ctypes.c_int, dp]
        L.oracle_face_flux.restype = None
        L.oracle_limiter.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, dp, dp]
        L.oracle_limiter.restype = None
        L.oracle_state_flux.argtypes = [dp, ctypes.c_double, dp, dp]
        L.oracle_state_flux.restype = None
        L.oracle_swept_replay.argtypes = [ctypes.c_int, i64, i64, i64, ctypes.c_int, i64,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_int, dp, ctypes.POINTER(ctypes.c_int64),
                                          ctypes.c_int]
        L.oracle_swept_replay.restype = ctypes.c_int
        L.oracle_heat_adjoint.argtypes = [i64, i64, dbl, dbl, dbl, dp, i64]
        L.oracle_heat_adjoint.restype = ctypes.c_int
        L.oracle_euler_adjoint.argtypes = [i64, i64, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int, dp, dp, i64, i64]
        L.oracle_euler_adjoint.restype = ctypes.c_int
        L.oracle_cell_pressure.argtypes = [dp, dbl]
        L.oracle_cell_pressure.restype = dbl
        _lib = L
    return _lib


def _dptr(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("oracle %s failed: %s (%d)" % (what, ERRORS.get(rc, "?"), rc))


def heat_r(dt, dx, alpha=1.0):
    """App. A mesh ratio r = alpha dt / dx^2, as the oracle evaluates it."""
    return float(lib().oracle_heat_r(float(alpha), float(dt), float(dx)))


def heat_run(u0, nsteps, dt, dx, alpha=1.0, scheme=0):
    """Advance the periodic heat field u0 [ny, nx] by nsteps time steps of size dt
    on a grid of spacing dx (dy = dx) with diffusivity alpha (App. A); returns a
    new array.  The oracle forms r = alpha dt / dx^2 itself."""
    u = np.ascontiguousarray(u0, dtype=np.float64).copy()
    ny, nx = u.shape
    _check(lib().oracle_heat_run(nx, ny, float(alpha), float(dt), float(dx), int(scheme), _dptr(u),
                                 int(nsteps)), "heat_run")
    return u


def euler_run(q0, dt, dx, nsteps, gamma=1.4, limiter=0):
    """Advance the periodic Euler state q0 [4, ny, nx] = (rho, rho u, rho v, E) by nsteps (App. B)."""
    q = np.ascontiguousarray(q0, dtype=np.float64).copy()
    _, ny, nx = q.shape
    _check(lib().oracle_euler_run(nx, ny, float(dt), float(dx), float(gamma), int(limiter),
                                  _dptr(q), int(nsteps)), "euler_run")
    return q


def swept_replay(eqn, state0, tile, depth, nsteps, c1, c2, gamma=1.4, limiter=0, plant=0):
    """Replay the swept schedule cell by cell (Sec. 3.3).

    eqn 0: heat, state0 [ny, nx], c1 = r/2, c2 = r.  eqn 1: Euler, state0
    [4, ny, nx], c1 = dt/(2 dx), c2 = dt/dx.  Returns (final state, stats dict).
    Raises on a dependency violation, a duplicate or a gap.  ``plant`` != 0
    plants a known schedule mistake (1: Octahedron before Bridges, 2: one
    level beyond Eq. 1) so a test can show the checker catches it.
    """
    s = np.ascontiguousarray(state0, dtype=np.float64).copy()
    nx, ny = s.shape[-1], s.shape[-2]
    st = (ctypes.c_int64 * 8)()
    rc = lib().oracle_swept_replay(int(eqn), nx, ny, int(tile), int(depth), int(nsteps),
                                   float(c1), float(c2), float(gamma), int(limiter), _dptr(s), st,
                                   int(plant))
    stats = {"cells": st[0], "cross_reads": st[1], "error": st[2], "where": (st[3], st[4], st[5]),
             "swept_levels": st[6], "phases": st[7]}
    if rc != 0:
        raise RuntimeError("swept replay failed: %s at level %d cell (%d, %d)"
                           % (ERRORS.get(rc, "?"), st[3], st[4], st[5]))
    return s, stats


def heat_adjoint(lamT, nsteps, dt, dx, alpha=1.0):
    """(A^T)^N lamT for the RK2 heat step A (App. A) with r = alpha dt / dx^2:
    the gradient of <u_N, lamT> with respect to u_0."""
    lam = np.ascontiguousarray(lamT, dtype=np.float64).copy()
    ny, nx = lam.shape
    _check(lib().oracle_heat_adjoint(nx, ny, float(alpha), float(dt), float(dx), _dptr(lam),
                                     int(nsteps)), "heat_adjoint")
    return lam


def euler_adjoint(q0, lamT, dt, dx, nsteps, ckpt=64, gamma=1.4, limiter=0):
    """dL/dQ^0 given lamT = dL/dQ^N for the App. B scheme (checkpoints every ckpt steps)."""
    q = np.ascontiguousarray(q0, dtype=np.float64)
    lam = np.ascontiguousarray(lamT, dtype=np.float64).copy()
    _, ny, nx = q.shape
    _check(lib().oracle_euler_adjoint(nx, ny, float(dt), float(dx), float(gamma), int(limiter),
                                      _dptr(q), _dptr(lam), int(nsteps), int(ckpt)),
           "euler_adjoint")
    return lam


def face_flux(qm1, q0, q1, q2, gamma=1.4, limiter=0):
    """Numerical flux (face-normal frame) at the face between q0 and q1."""
    arrs = [np.ascontiguousarray(x, dtype=np.float64) for x in (qm1, q0, q1, q2)]
    out = np.zeros(4)
    lib().oracle_face_flux(*[_dptr(a) for a in arrs], float(gamma), int(limiter), _dptr(out))
    return out


def limiter(dm, dp, kind=0):
    """(phi towards the + face, phi towards the - face) for one cell."""
    a = np.zeros(1)
    b = np.zeros(1)
    lib().oracle_limiter(float(dm), float(dp), int(kind), _dptr(a), _dptr(b))
    return float(a[0]), float(b[0])


def cell_pressure(q, gamma=1.4):
    """Pressure of one conserved state (rho, rho u, rho v, E) as the limiter forms it."""
    qa = np.ascontiguousarray(q, dtype=np.float64)
    return float(lib().oracle_cell_pressure(_dptr(qa), float(gamma)))


def state_flux(q, gamma=1.4):
    """Physical flux and |u_n| + c of one state in the face-normal frame."""
    qa = np.ascontiguousarray(q, dtype=np.float64)
    f = np.zeros(4)
    lam = np.zeros(1)
    lib().oracle_state_flux(_dptr(qa), float(gamma), _dptr(f), _dptr(lam))
    return f, float(lam[0])
