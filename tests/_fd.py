"""Central differences of the FP64 oracle's smoothed objective for the GPU
gradient tests, evaluated in worker processes (each builds the seeded
workload once).  Tests only; the pool is started with the 'spawn' method."""
from __future__ import annotations

import numpy as np

_D = None


def init(workload: str, seed: int, period_ns: float):
    global _D
    from paper_2511_11660_b300 import synth
    _D = synth.workload(workload, seed=seed)
    _D["period_ns"] = period_ns


def objective_at(task):
    """J with cell coordinate (cell, axis) moved by delta um (0: unmoved).
    Returns (J, the coordinate actually used, in FP32)."""
    import oracle
    cell, axis, delta = task
    dd = dict(_D)
    xy = np.asarray(_D["cell_xy"], np.float32).copy()
    xy[2 * cell + axis] = np.float32(np.float64(xy[2 * cell + axis]) + delta)
    dd["cell_xy"] = xy
    return oracle.objective(dd), float(xy[2 * cell + axis])
