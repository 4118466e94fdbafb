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


# ------------------------------------------- per-endpoint limit above 1

def check_nworst(d, gpu, want, L, res, corner=0):
    """The report with a per-endpoint limit against the oracle's: the path
    slacks, in order, agree within tolerance (near-ties may swap which of two
    equally critical paths is reported, never the slack at a rank); every GPU
    path is a chain of timing arcs with consistent edges from a startpoint to
    its endpoint, distinct from the others, at most L per endpoint, and its
    arrivals and slack are its own FP64 prefix sums under the oracle's
    analysis (cell arc delays at the analysis' slews and loads)."""
    net = _indep.Net(d, corner)
    role = np.asarray(d["pin_role"])
    K = int(d.get("n_corners", 1))
    sc = float(np.asarray(d["lut_scale"] if d.get("lut_scale") is not None else np.ones(K))[corner])
    i1 = np.asarray(d["lut_idx1"]).reshape(-1, 3, 4, 7)
    i2 = np.asarray(d["lut_idx2"]).reshape(-1, 3, 4, 7)
    vv = np.asarray(d["lut_val"]).reshape(-1, 3, 4, 49)
    sense = np.asarray(d["arc_sense"]).reshape(-1, 3)
    assert len(gpu) == len(want)
    gs = np.array([p["slack"] for p in gpu])
    ws = np.array([p["slack"] for p in want])
    assert np.all(np.diff(gs) >= 0)
    assert np.all(np.abs(gs - ws) <= ABS_TOL + REL_TOL * np.abs(ws)), np.abs(gs - ws).max()
    seen, per_ep = set(), {}
    for p in gpu:
        pins, rfs, ats = p["pins"], p["rf"], p["at"]
        key = (tuple(pins.tolist()), tuple(rfs.tolist()))
        assert key not in seen
        seen.add(key)
        per_ep[p["endpoint"]] = per_ep.get(p["endpoint"], 0) + 1
        assert pins[-1] == p["endpoint"]
        assert role[pins[0]] in (synth.PI, synth.CK)
        arr = float(res["at"][pins[0], corner, 2 + rfs[0]])
        assert abs(ats[0] - arr) <= tol(arr)
        for i in range(1, len(pins)):
            u, ru, v, rv = int(pins[i - 1]), int(rfs[i - 1]), int(pins[i]), int(rfs[i])
            if net.driver.get(v) == u:
                assert ru == rv
                arr += net.Dns[v]
            else:
                c = net.cell_of[v]
                assert c >= 0 and net.cell_of[u] == c
                t = d["cell_type"][c]
                j = net.slot_of[u]
                if role[v] == synth.Q:
                    assert ru == 0 and sense[t, j] == _indep.RISE
                else:
                    assert ru in _indep.rf_in_of(sense[t, j], rv)
                dl = oracle.lut_eval(i1[t, j, rv], i2[t, j, rv], vv[t, j, rv], res["slew"][u, corner, 2 + ru],
                                     net.load[v])[0]
                arr += sc * dl
            assert abs(ats[i] - arr) <= tol(arr), (i, ats[i], arr)
        ref = float(res["rat"][pins[-1], corner, 2 + rfs[-1]]) - arr
        assert abs(p["slack"] - ref) <= tol(ref)
    assert max(per_ep.values(), default=0) <= L


@pytest.mark.parametrize("case", ["tiny", "corners", "threshold"])
def test_nworst_paths_match_oracle(case):
    corner, slack_lt = 0, np.inf
    if case == "corners":
        ls, rs = synth.lut_corners()
        d = synth.make_design(3000, 20, seed=4, n_corners=4, lut_scale=ls, rc_scale=rs, period_ns=1.7)
        corner = 3
    else:
        d = synth.workload("tiny", seed=1)
        d["period_ns"], _ = tune_period(d)
        if case == "threshold":
            slack_lt = -0.05
    res = oracle.sta(d)
    ctx = sta.Context(d)
    ctx.update_timing()
    for k, L in ((1, 2), (40, 5), (300, 3), (64, 32)):
        gpu = ctx.report_paths(k, slack_lt=slack_lt, corner=corner, per_endpoint=L)
        want = oracle.report_paths_nworst(d, k, L, slack_lt=slack_lt, corner=corner, res=res)
        check_nworst(d, gpu, want, L, res, corner)
        assert len(gpu) > 0
    # more paths than endpoints at the limit: some endpoint holds several
    gpu = ctx.report_paths(100, per_endpoint=8, corner=corner, slack_lt=slack_lt)
    assert len({p["endpoint"] for p in gpu}) < len(gpu)
    ctx.close()


def test_nworst_limit_one_and_errors():
    d = synth.workload("tiny", seed=2)
    d["period_ns"], _ = tune_period(d)
    ctx = sta.Context(d)
    ctx.update_timing()
    a = ctx.report_paths(50)
    b = ctx.report_paths(50, per_endpoint=1)
    assert [p["endpoint"] for p in a] == [p["endpoint"] for p in b]
    assert ctx.report_paths(0, per_endpoint=4) == []
    assert ctx.report_paths(20, per_endpoint=4, slack_lt=-1e6) == []
    for k, L in ((10, 0), (10, 33), (4096, 5)):
        with pytest.raises(sta.StaError) as ei:
            ctx.report_paths(k, per_endpoint=L)
        assert ei.value.status == sta.EINVAL
    ctx.close()
    dx = dict(d, **synth.exception_groups(d, np.random.default_rng(0), 2))
    ctx = sta.Context(dx)
    ctx.update_timing()
    with pytest.raises(sta.StaError) as ei:
        ctx.report_paths(10, per_endpoint=2)
    assert ei.value.status == sta.EINVAL
    assert len(ctx.report_paths(10, per_endpoint=1)) == 10
    ctx.close()


def test_nworst_batch_design_equals_separate_context():
    ds = synth.batch_workload(seed=1, n_designs=3, lo=800, hi=3000, depth=12)
    b = sta.Context(None, batch=ds)
    b.update_timing()
    off = 0
    for i, d in enumerate(ds):
        c = sta.Context(d)
        c.update_timing()
        want = c.report_paths(60, corner=1, per_endpoint=4)
        got = b.report_paths(60, corner=1, design=i, per_endpoint=4)
        assert len(got) == len(want)
        for g, w in zip(got, want):
            assert g["endpoint"] == w["endpoint"] + off
            np.testing.assert_array_equal(g["pins"], w["pins"] + off)
            np.testing.assert_array_equal(g["at"], w["at"])
        c.close()
        off += d["n_pins"]
    b.close()


def test_nworst_paths_full_size():
    """The 1M-cell workload: the 100 worst paths, up to 4 per endpoint."""
    d = synth.workload("scale", seed=0)
    d["period_ns"], _ = tune_period(d)
    res = oracle.sta(d)
    ctx = sta.Context(d)
    ctx.update_timing()
    gpu = ctx.report_paths(100, per_endpoint=4)
    check_nworst(d, gpu, oracle.report_paths_nworst(d, 100, 4, res=res), 4, res)
    ctx.close()
