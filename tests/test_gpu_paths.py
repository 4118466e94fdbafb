"""GPU top-k path report (sta_report_paths) against the FP64 oracle.

What is unique is compared: the reported endpoints are the k worst below the
threshold (up to near-ties of the FP32 slacks), in non-decreasing slack.  Where
several answers are correct (a near-tie between two fan-ins), the rest is
checked for validity: each path is a chain of timing arcs from a startpoint
to its endpoint with consistent edges, its arrivals match the oracle's, and
every step is critical under the oracle's FP64 numbers (the chosen input's
arrival + arc delay is within tolerance of the best candidate)."""
import numpy as np
import pytest

import oracle
from paper_2511_11660_b300 import sta, synth
from tests import _indep
from tests._parity import ABS_TOL, REL_TOL, tune_period

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    sta.load()


def tol(x):
    return ABS_TOL + REL_TOL * abs(x)


def check_paths(d, gpu, res, k, slack_lt=np.inf, corner=0):
    """With timing exceptions each path is checked in the (corner, tag)
    states whose late slack at its endpoint is within tolerance of the
    smallest: it must be valid and critical in one of them."""
    net = _indep.Net(d, corner)
    Tg = oracle.n_tags(d)
    _, adv = oracle.tag_layout(d)
    role = np.asarray(d["pin_role"])
    K = int(d.get("n_corners", 1))
    sc = float(np.asarray(d["lut_scale"] if d.get("lut_scale") is not None else np.ones(K))[corner])
    i1 = np.asarray(d["lut_idx1"]).reshape(-1, 3, 4, 7)
    i2 = np.asarray(d["lut_idx2"]).reshape(-1, 3, 4, 7)
    vv = np.asarray(d["lut_val"]).reshape(-1, 3, 4, 49)
    sense = np.asarray(d["arc_sense"]).reshape(-1, 3)
    cpp, cp = np.asarray(d["cell_pin_ptr"]), np.asarray(d["cell_pin"])
    eps, es = res["endpoints"], res["ep_setup"][:, corner]
    eligible = sorted((e for e in range(len(eps)) if es[e] < slack_lt), key=lambda e: (es[e], e))
    assert len(gpu) == min(k, len(eligible))
    ep_index = {int(p): e for e, p in enumerate(eps)}
    if gpu:
        kth = es[eligible[len(gpu) - 1]]
        for p in gpu:
            e = ep_index[p["endpoint"]]
            assert abs(p["slack"] - es[e]) <= tol(es[e])
            assert es[e] <= kth + 2 * tol(kth)           # among the k worst up to near-ties
        s = [p["slack"] for p in gpu]
        assert all(a <= b for a, b in zip(s, s[1:]))

    def check_one(p, st_end):
        pins, rfs, ats = p["pins"], p["rf"], p["at"]
        # the state at every pin: it changes only at -through pins, to the
        # previous tag's state when that one carries the larger late arrival
        sts = [st_end] * len(pins)
        for i in range(len(pins) - 1, 0, -1):
            st = sts[i]
            v, u = int(pins[i]), int(pins[i - 1])
            if net.driver.get(v) == u:
                tg = st - corner * Tg
                a = adv.get(v, 0)
                stay, inflow = not (a >> tg) & 1, tg >= 1 and (a >> (tg - 1)) & 1
                r = 2 + int(rfs[i])
                a_st, a_prev = res["at"][u, st, r], res["at"][u, st - 1, r]
                if inflow and (not stay or a_prev > a_st + (tol(a_st) if np.isfinite(a_st) else 0.0)):
                    st -= 1
            sts[i - 1] = st

        def cand(v, rv, u, ru, st):
            at, slew = res["at"][:, st], res["slew"][:, st]
            c = net.cell_of[v]
            t = d["cell_type"][c]
            j = net.slot_of[u]
            dl = oracle.lut_eval(i1[t, j, rv], i2[t, j, rv], vv[t, j, rv], slew[u, 2 + ru], net.load[v])[0]
            return at[u, 2 + ru] + sc * dl

        assert pins[-1] == p["endpoint"]
        assert role[pins[0]] in (synth.PI, synth.CK)
        for q, r, a, st in zip(pins, rfs, ats, sts):
            ref = res["at"][q, st, 2 + r]
            assert abs(a - ref) <= tol(ref)
        for i in range(1, len(pins)):
            u, ru, v, rv = int(pins[i - 1]), int(rfs[i - 1]), int(pins[i]), int(rfs[i])
            st = sts[i]
            if net.driver.get(v) == u:
                assert ru == rv
                continue
            c = net.cell_of[v]
            assert c >= 0 and net.cell_of[u] == c
            t = d["cell_type"][c]
            if role[v] == synth.Q:
                assert ru == 0 and sense[t, net.slot_of[u]] == _indep.RISE
                continue
            assert ru in _indep.rf_in_of(sense[t, net.slot_of[u]], rv)
            best = max(cand(v, rv, int(cp[cpp[c] + j]), r2, st) for j in range(d["type_nin"][t])
                       for r2 in _indep.rf_in_of(sense[t, j], rv))
            assert cand(v, rv, u, ru, st) >= best - 2 * tol(best)

    for p in gpu:
        e = int(p["endpoint"])
        late = [float(np.min(res["slack"][e, corner * Tg + g, 2:])) for g in range(Tg)]
        worst = min(late)
        states = [corner * Tg + g for g in range(Tg) if late[g] <= worst + 2 * tol(worst)]
        errors = []
        for st in states:
            try:
                check_one(p, st)
                break
            except AssertionError as ex:
                errors.append(ex)
        else:
            raise errors[0]


@pytest.mark.parametrize("case", ["tiny", "corners", "smooth", "threshold"])
def test_paths_match_oracle(case):
    corner = 0
    slack_lt = np.inf
    if case == "corners":
        ls, rs = synth.lut_corners()
        d = synth.make_design(3000, 20, seed=4, n_corners=4, lut_scale=ls, rc_scale=rs, period_ns=1.7)
        corner = 3
    elif case == "smooth":
        d = synth.make_design(3000, 15, seed=6, gamma_ns=0.01)
        d["period_ns"], _ = tune_period(d)
    else:
        d = synth.workload("tiny", seed=1)
        d["period_ns"], _ = tune_period(d)
        if case == "threshold":
            slack_lt = -0.05
    res = oracle.sta(d)
    ctx = sta.Context(d)
    for sch in (sta.SCHED_DATAFLOW, sta.SCHED_LEVEL):
        ctx.set_schedule(sch)
        ctx.update_timing()
        for k in (1, 25, 300):
            gpu = ctx.report_paths(k, slack_lt=slack_lt, corner=corner)
            check_paths(d, gpu, res, k, slack_lt, corner)
    ctx.close()


def test_paths_edge_cases():
    d = synth.workload("tiny", seed=2)
    d["period_ns"], _ = tune_period(d)
    ctx = sta.Context(d)
    ctx.update_timing()
    assert ctx.report_paths(0) == []
    assert ctx.report_paths(50, slack_lt=-1e6) == []
    E = ctx.E
    allp = ctx.report_paths(4096)
    assert len(allp) == min(E, 4096)
    assert [p["endpoint"] for p in allp[:30]] == [p["endpoint"] for p in ctx.report_paths(30)]
    with pytest.raises(sta.StaError):
        ctx.report_paths(4097)
    with pytest.raises(sta.StaError):
        ctx.report_paths(5, corner=1)
    ctx.close()


def test_batch_design_paths_equal_separate_context():
    ds = synth.batch_workload(seed=1, n_designs=3, lo=800, hi=3000, depth=12)
    b = sta.Context(None, batch=ds)
    b.update_timing()
    off = 0
    for i, d in enumerate(ds):
        c = sta.Context(d)
        c.update_timing()
        for corner in (0, 2):
            want = c.report_paths(40, corner=corner)
            got = b.report_paths(40, corner=corner, design=i)
            assert len(got) == len(want)
            for g, w in zip(got, want):
                assert g["endpoint"] == w["endpoint"] + off
                np.testing.assert_array_equal(g["pins"], w["pins"] + off)
                np.testing.assert_array_equal(g["rf"], w["rf"])
                np.testing.assert_array_equal(g["at"], w["at"])
        c.close()
        off += d["n_pins"]
    b.close()


def test_paths_full_size():
    """The 1M-cell workload: the 200 worst endpoints' paths against the oracle."""
    d = synth.workload("scale", seed=0)
    d["period_ns"], _ = tune_period(d)
    res = oracle.sta(d)
    ctx = sta.Context(d)
    ctx.update_timing()
    check_paths(d, ctx.report_paths(200), res, 200)
    ctx.close()
