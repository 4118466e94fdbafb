"""GPU timing exceptions (false paths, multicycle paths and max/min delays by
startpoint group, ordered -through sets of gate inputs and endpoint list)
against the FP64 oracle.

Every per-pin array holds one state per (corner, exception tag) and is
compared element by element (infinities equal: an absent tag's arrival is
-inf late / +inf early); endpoint slacks are the minimum over tags and
violation flags are bit-exact wherever the oracle's slack is clear of zero by
more than twice the tolerance."""
import numpy as np
import pytest

import oracle
from paper_2511_11660_b300 import sta, synth
from tests._parity import ABS_TOL, assert_close, tune_period
from tests.test_gpu_paths import check_paths

pytestmark = pytest.mark.gpu

SCHEDULES = [sta.SCHED_LEVEL, sta.SCHED_DATAFLOW, sta.SCHED_COOP, sta.SCHED_TILE]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    sta.load()


def _design(case, seed, n_groups, max_thru=0, actions=None):
    rng = np.random.default_rng(100 + seed)
    if case == "corners":
        ls, rs = synth.lut_corners()
        d = synth.make_design(3000, 20, seed=seed, n_corners=4, lut_scale=ls, rc_scale=rs, period_ns=1.7)
    elif case == "placed":
        d = synth.make_design(3000, 20, seed=seed, placed=True)
        d["period_ns"], _ = tune_period(d)
    else:
        d = synth.workload("tiny", seed=seed)
        d["period_ns"], _ = tune_period(d)
    d.update(synth.exception_groups(d, rng, n_groups, max_thru=max_thru, actions=actions))
    return d


def _gpu(ctx):
    out = {k: ctx.get_pin_state(w) for k, w in (("at", sta.AT), ("slew", sta.SLEW), ("rat", sta.RAT),
                                                  ("slack", sta.SLACK))}
    out["ep_setup"], out["ep_hold"], out["viol_setup"], out["viol_hold"] = ctx.get_endpoint_slack()
    out["report"] = ctx.report_slack()
    return out


def check(d, g, ref):
    K = int(d.get("n_corners", 1))
    Tg = oracle.n_tags(d)
    for k in ("at", "slew", "rat", "slack"):
        assert g[k].shape == ref[k].shape == (d["n_pins"], K * Tg, 4)
        assert_close(k, g[k], ref[k])
    assert_close("ep_setup", g["ep_setup"], ref["ep_setup"])
    assert_close("ep_hold", g["ep_hold"], ref["ep_hold"])
    margin = 2 * ABS_TOL
    for name, vname in (("ep_setup", "viol_setup"), ("ep_hold", "viol_hold")):
        r = ref[name]
        clear = ~(np.abs(r) <= margin)
        np.testing.assert_array_equal(g[vname][clear], (r[clear] < 0).astype(np.uint8))
    for k in range(K):
        rep = g["report"][k]
        es = g["ep_setup"][:, k].astype(np.float64)
        assert rep["tns_setup"] == pytest.approx(np.minimum(es, 0).sum(), rel=1e-12, abs=1e-12)
        nv = max(int(ref["n_viol_setup"][k]), 1)
        assert abs(rep["tns_setup"] - ref["tns_setup"][k]) <= nv * 1e-4 + 1e-5 * abs(ref["tns_setup"][k])
        assert abs(rep["wns_setup"] - ref["wns_setup"][k]) <= 1e-4 + 1e-5 * abs(ref["wns_setup"][k])
        assert abs(rep["tns_hold"] - ref["tns_hold"][k]) <= max(int(ref["n_viol_hold"][k]), 1) * 1e-4 + \
            1e-5 * abs(ref["tns_hold"][k])


ALL_ACTIONS = (0, 1, 2, 3)   # false path, multicycle, max delay, min delay


@pytest.mark.parametrize("case,seed,n_groups,max_thru,actions",
                         [("tiny", 0, 1, 0, None), ("tiny", 1, 3, 0, None), ("tiny", 2, 7, 0, None),
                          ("corners", 4, 3, 0, None), ("placed", 5, 2, 0, None),
                          ("tiny", 6, 3, 2, None), ("tiny", 7, 5, 3, None),
                          ("corners", 8, 2, 2, None), ("tiny", 9, 6, 0, ALL_ACTIONS),
                          ("corners", 10, 4, 1, ALL_ACTIONS), ("tiny", 11, 4, 2, (2, 3))])
def test_exceptions_parity_all_schedules(case, seed, n_groups, max_thru, actions):
    d = _design(case, seed, n_groups, max_thru, actions)
    ref = oracle.sta(d)
    # the groups must change something: some endpoint's slack differs from the unconstrained analysis
    plain = {k: v for k, v in d.items() if not k.startswith("exc_")}
    assert not np.allclose(oracle.sta(plain)["ep_setup"], ref["ep_setup"])
    ctx = sta.Context(d)
    assert ctx.stats()["n_tags"] == oracle.n_tags(d)
    for sch in SCHEDULES:
        ctx.set_schedule(sch)
        ctx.update_timing()
        check(d, _gpu(ctx), ref)
    ctx.close()


def test_exceptions_corner_and_clock_updates():
    d = _design("corners", 7, 4)
    ctx = sta.Context(d)
    ctx.update_timing()
    check(d, _gpu(ctx), oracle.sta(d))
    ls = np.array([1.0, 1.1, 0.95, 1.3], np.float32)
    rs = np.array([1.0, 0.9, 1.2, 1.25], np.float32)
    ctx.set_corners(ls, rs)
    ctx.set_clock(1.9)
    ctx.update_timing()
    d2 = dict(d, lut_scale=ls, rc_scale=rs, period_ns=1.9)
    check(d2, _gpu(ctx), oracle.sta(d2))
    ctx.close()


def test_exceptions_all_false_paths_leave_no_checks():
    """One false-path group from every startpoint to every endpoint: tag 0
    carries no arrival, so every endpoint slack is +inf and nothing violates."""
    d = synth.workload("tiny", seed=3)
    d["period_ns"], _ = tune_period(d)
    role = np.asarray(d["pin_role"])
    starts = np.nonzero((role == synth.PI) | (role == synth.CK))[0].astype(np.int32)
    d.update(exc_from_ptr=np.array([0, len(starts)], np.int32), exc_from=starts,
             exc_to_ptr=np.array([0, 0], np.int32), exc_to=np.zeros(0, np.int32),
             exc_action=np.array([0], np.int32), exc_mult=np.array([1.0], np.float32))
    ctx = sta.Context(d)
    ctx.update_timing()
    g = _gpu(ctx)
    assert np.all(np.isposinf(g["ep_setup"])) and np.all(np.isposinf(g["ep_hold"]))
    assert not g["viol_setup"].any() and not g["viol_hold"].any()
    rep = g["report"][0]
    assert rep["wns_setup"] == 0.0 and rep["tns_setup"] == 0.0 and rep["n_viol_setup"] == 0
    check(d, g, oracle.sta(d))
    ctx.close()


@pytest.mark.parametrize("case,seed,n_groups,corner,max_thru", [("tiny", 1, 3, 0, 0), ("corners", 4, 3, 2, 0),
                                                                ("tiny", 6, 3, 0, 2), ("corners", 8, 2, 1, 2)])
def test_exceptions_paths(case, seed, n_groups, corner, max_thru):
    d = _design(case, seed, n_groups, max_thru)
    res = oracle.sta(d)
    ctx = sta.Context(d)
    ctx.update_timing()
    for k in (1, 40, 400):
        gpu = ctx.report_paths(k, corner=corner)
        check_paths(d, gpu, res, k, corner=corner)
        want = oracle.report_paths(d, k, corner=corner, res=res)
        assert len(gpu) == len(want)
    ctx.close()


@pytest.mark.parametrize("max_thru,actions", [(0, None), (2, None), (0, ALL_ACTIONS)])
def test_exceptions_full_size(max_thru, actions):
    """The 1M-cell workload with three exception groups (four tags; with
    through sets of 1/64 of the gate inputs, up to ten), also with max/min
    delay actions."""
    d = synth.workload("scale", seed=0)
    d["period_ns"], _ = tune_period(d)
    d.update(synth.exception_groups(d, np.random.default_rng(9), 3, div_from=5, div_to=4, max_thru=max_thru,
                                    div_thru=64, actions=actions))
    ref = oracle.sta(d)
    ctx = sta.Context(d)
    ctx.update_timing()
    check(d, _gpu(ctx), ref)
    ctx.close()
