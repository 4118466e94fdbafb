"""Shared parity helpers for the GPU tests: tolerance checks and the clock
period chosen from the oracle so that endpoint violation sets are well
defined (no endpoint slack closer to zero than the GPU's error bound)."""
from __future__ import annotations

import numpy as np

import oracle

ABS_TOL = 1e-4   # ns
REL_TOL = 1e-5


def close(gpu, ref, abs_tol=ABS_TOL, rel_tol=REL_TOL):
    """Per element: infinities must match exactly; finite values must be
    within abs_tol OR within rel_tol * |ref|.  Returns (ok, max_abs, max_rel)."""
    g = np.asarray(gpu, np.float64)
    r = np.asarray(ref, np.float64)
    assert g.shape == r.shape, (g.shape, r.shape)
    fin = np.isfinite(r)
    ok_inf = np.array_equal(g[~fin], r[~fin])
    err = np.abs(g[fin] - r[fin])
    rel = err / np.maximum(np.abs(r[fin]), 1e-30)
    ok = ok_inf and bool(np.all((err <= abs_tol) | (rel <= rel_tol))) and bool(np.all(np.isfinite(g[fin])))
    return ok, (float(err.max()) if err.size else 0.0), (float(rel.max()) if rel.size else 0.0)


def assert_close(name, gpu, ref, abs_tol=ABS_TOL, rel_tol=REL_TOL):
    ok, ea, er = close(gpu, ref, abs_tol, rel_tol)
    if not ok:
        g = np.asarray(gpu, np.float64)
        r = np.asarray(ref, np.float64)
        bad = np.argwhere(~((np.abs(g - r) <= abs_tol) | (np.abs(g - r) <= rel_tol * np.abs(r)) | (g == r)))
        raise AssertionError("%s: max abs err %.3g, max rel err %.3g; first bad %s: gpu %r ref %r"
                             % (name, ea, er, bad[:3].tolist(), g[tuple(bad[0])] if len(bad) else None,
                                r[tuple(bad[0])] if len(bad) else None))
    return ea, er


VIOL_MARGIN = ABS_TOL   # ns


def assert_viol_defined(ref, margin: float = VIOL_MARGIN):
    """Endpoint violation sets are well defined when every finite endpoint
    slack of the oracle lies farther than the tolerance from zero: a GPU
    value within tolerance then has the same sign (|err| <= max(1e-4, 1e-5
    |ref|) < |ref|), so the sets must agree bit for bit.  Fails (it does not
    skip) when a design or clock period breaks that."""
    for key in ("ep_setup", "ep_hold"):
        v = np.asarray(ref[key], np.float64)
        v = v[np.isfinite(v)]
        if v.size:
            worst = float(np.abs(v).min())
            assert worst > margin, ("%s: an endpoint slack %.3g ns from zero, within the %.0e ns tolerance: "
                                    "the violation set is not well defined for this design" % (key, worst, margin))


def tune_period(d: dict, bands=((0.89, 0.91), (0.88, 0.92), (0.87, 0.93), (0.85, 0.95)),
                min_half_gap: float = 1e-4):
    """Clock period in the widest gap between consecutive endpoint setup
    requirements inside a quantile band around 90% (so about 10% of the
    endpoints violate), taking the narrowest band of ``bands`` whose widest
    gap exceeds twice ``min_half_gap`` -- the tolerance -- so that violation
    sets are well defined.  Uses the oracle with T = 0, where each endpoint
    slack is minus its requirement.  Returns (period, half_gap)."""
    d0 = dict(d)
    d0["period_ns"] = 0.0
    r = oracle.sta(d0)
    q = np.sort(-r["ep_setup"][:, 0])
    n = len(q)
    best = None
    for lo_q, hi_q in bands:
        i0, i1 = int(np.floor(lo_q * (n - 1))), int(np.ceil(hi_q * (n - 1)))
        i1 = max(i1, i0 + 1)
        gaps = np.diff(q[i0:i1 + 1])
        k = int(np.argmax(gaps))
        best = (0.5 * (q[i0 + k] + q[i0 + k + 1]), 0.5 * float(gaps[k]))
        if best[1] > min_half_gap:
            break
    T, half = best
    assert half > min_half_gap, "no clean gap for the clock period (half gap %.3g)" % half
    return float(T), half
