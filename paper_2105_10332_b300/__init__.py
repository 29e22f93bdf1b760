"""B300-native swept-rule solver for explicit 2D stencil PDEs (heat, Euler; RK2; FP64).

Python binding over the C ABI in ``include/sweep.h`` (``libsweep.so``):
``from paper_2105_10332_b300 import sweep``.  ``workloads`` builds the
seeded synthetic inputs (heat modes, isentropic vortex).
"""
__all__ = ["sweep", "workloads"]
