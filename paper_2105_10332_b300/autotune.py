"""Autotuner for the swept solver's knobs: block edge (tile), depth (levels per
phase) and, for Euler, the cluster sizes of the Octahedron and Bridge
kernels -- the tuning the paper does by sweeping the block size (Sec. 4).

For an (equation, grid side) pair it times each legal configuration on a
short run of a representative instance with CUDA events.  Timings are kept
per (equation, size class), the size class being the side rounded up to a
power of two: a later side of the same class takes the fastest configuration
of that class's ranking that is legal for it (its tile must divide the side),
and only a side for which no ranked configuration is legal is timed afresh.
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
    """ranking[(eqn, class)]: configurations fastest first, as timed on the
    first side of the class that needed tuning (later sides that needed a
    fresh timing add theirs after).  cache[(eqn, class)]: the fastest of the
    first timing.  chosen[(eqn, side)]: what each side was given."""

    def __init__(self, steps=None):
        self.steps = steps
        self.ranking = {}
        self.cache = {}
        self.chosen = {}
        self.log = []

    def select(self, eqn, side, measure):
        """Configuration for (eqn, side).  measure(cfg) -> milliseconds per step,
        or None when that configuration cannot be built; it is called only when
        the class's ranking holds no configuration legal for this side."""
        key = (eqn, size_class(side))
        legal = candidates(eqn, side)
        for cfg in self.ranking.get(key, []):
            if cfg in legal:
                self.chosen[(eqn, side)] = cfg
                return cfg
        timed = []
        for cfg in legal:
            ms = measure(cfg)
            if ms is None:
                continue
            self.log.append((eqn, side, cfg, ms))
            timed.append((ms, len(timed), cfg))
        if not timed:
            raise RuntimeError("no legal swept configuration runs for %s at side %d" % (eqn, side))
        timed.sort()
        fresh = [cfg for _, _, cfg in timed]
        self.ranking[key] = self.ranking.get(key, []) + [c for c in fresh
                                                           if c not in self.ranking.get(key, [])]
        self.cache.setdefault(key, fresh[0])
        self.chosen[(eqn, side)] = fresh[0]
        return fresh[0]

    def best(self, eqn, side, dt, dx, state):
        """Fastest legal configuration for (eqn, side); `state` is a CUDA tensor
        of the instance used for timing (left unchanged)."""
        import torch

        def measure(cfg):
            kw = dict(cfg)
            tile, depth = kw.pop("tile"), kw.pop("depth")
            try:
                solver = S.Solver(eqn, side, side, dt, dx, tile, depth, **kw)
            except S.SweepError:
                return None
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
            solver.close()
            return e0.elapsed_time(e1) / steps

        return self.select(eqn, side, measure)
