"""Autotuner for the swept solver's knobs: block edge (tile), depth (levels per
phase) and, for Euler, the cluster sizes of the Octahedron and Bridge
kernels -- the tuning the paper does by sweeping the block size (Sec. 4).

For a (equation, grid side) pair it times each candidate configuration on a
short run of a representative instance with CUDA events and keeps the
fastest; results are cached per (equation, size class), the size class being
the side rounded up to a power of two.
"""
import math

from . import sweep as S

HEAT_TILES = (16, 32, 64)
EULER_TILES = (16, 32)


def size_class(side):
    return 1 << max(0, math.ceil(math.log2(side)))


def candidates(eqn, side):
    """Legal configurations for a square grid of this side: dicts of Solver kwargs."""
    out = []
    tiles = HEAT_TILES if eqn == "heat" else EULER_TILES
    n = 1 if eqn == "heat" else 2
    for b in tiles:
        if side % b or side // b < 2:
            continue
        k = b // (2 * n) - 1
        depths = sorted({d for d in (k - (k % 2), (k // 2) - ((k // 2) % 2)) if d >= 2})
        for d in depths:
            if eqn == "heat":
                out.append(dict(tile=b, depth=d))
            else:
                for co, cb in ((2, 1), (1, 1)):
                    out.append(dict(tile=b, depth=d, cluster_oct=co, cluster_bridges=cb))
    return out


class Autotuner:
    def __init__(self, steps=None):
        self.steps = steps
        self.cache = {}
        self.log = []

    def best(self, eqn, side, dt, dx, state):
        """Fastest configuration for (eqn, size class of side); `state` is a CUDA
        tensor of the instance used for timing (left unchanged)."""
        import torch
        key = (eqn, size_class(side))
        if key in self.cache:
            return self.cache[key]
        best, best_ms = None, None
        for cfg in candidates(eqn, side):
            kw = dict(cfg)
            tile, depth = kw.pop("tile"), kw.pop("depth")
            try:
                solver = S.Solver(eqn, side, side, dt, dx, tile, depth, **kw)
            except S.SweepError:
                continue
            steps = self.steps or max(2 * depth, 8)
            work = state.clone()
            solver.run_swept(work, steps)  # warm-up
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            work.copy_(state)
            e0.record()
            solver.run_swept(work, steps)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            self.log.append((eqn, side, cfg, ms))
            if best_ms is None or ms < best_ms:
                best, best_ms = cfg, ms
            solver.close()
        self.cache[key] = best
        return best
