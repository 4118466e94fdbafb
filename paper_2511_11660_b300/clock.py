"""Clock period selection for benchmark workloads (host logic only).

Given every endpoint's setup requirement q_e (its late arrival plus setup,
i.e. minus its slack at period 0), place the period in the widest gap
between consecutive requirements inside a quantile band around 90%, so that
about 10% of the endpoints violate and no endpoint slack sits within half
that gap of zero."""
from __future__ import annotations

import numpy as np


def period_in_gap(requirements, bands=((0.89, 0.91), (0.88, 0.92), (0.87, 0.93), (0.85, 0.95)),
                  min_half_gap: float = 1e-4):
    q = np.sort(np.asarray(requirements, np.float64).reshape(-1))
    n = len(q)
    if n < 2:
        return float(q[0] if n else 1.0) + 1.0, float("inf")
    best = None
    for lo, hi in bands:
        i0, i1 = int(np.floor(lo * (n - 1))), int(np.ceil(hi * (n - 1)))
        i1 = max(i1, i0 + 1)
        g = np.diff(q[i0:i1 + 1])
        k = int(np.argmax(g))
        best = (0.5 * (q[i0 + k] + q[i0 + k + 1]), 0.5 * float(g[k]))
        if best[1] > min_half_gap:
            break
    return float(best[0]), float(best[1])
