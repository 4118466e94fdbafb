"""Batched designs: one context over several independent designs of uneven
size and several corners (sta_create_batch) gives, design by design, the
results of separate contexts bit for bit, and the FP64 oracle's within the
parity tolerance; per-design reports come from per-design reductions."""
import numpy as np
import pytest

import oracle
from paper_2511_11660_b300 import sta, synth
from tests._parity import assert_close

pytestmark = pytest.mark.gpu

ARRAYS = (("at", sta.AT), ("slew", sta.SLEW), ("rat", sta.RAT), ("slack", sta.SLACK))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    sta.load()


def designs(corners=2):
    lib = synth.make_library(7)
    ls, rs = synth.lut_corners()
    return [synth.make_design(n, dep, seed=30 + i, lib=lib, n_corners=corners, lut_scale=ls[:corners],
                              rc_scale=rs[:corners], period_ns=1.6)
            for i, (n, dep) in enumerate([(300, 8), (2000, 25), (800, 12), (5000, 30), (40, 3)])]


@pytest.mark.parametrize("schedule", [sta.SCHED_LEVEL, sta.SCHED_DATAFLOW, sta.SCHED_COOP, sta.SCHED_TILE])
def test_batch_equals_separate_contexts(schedule):
    ds = designs()
    bctx = sta.Context(None, batch=ds)
    bctx.set_schedule(schedule)
    bctx.update_timing()
    got = {k: bctx.get_pin_state(w) for k, w in ARRAYS}
    es, eh, vs, vh = bctx.get_endpoint_slack()
    p0 = e0 = 0
    for i, d in enumerate(ds):
        ctx = sta.Context(d)
        ctx.set_schedule(schedule)
        ctx.update_timing()
        P = d["n_pins"]
        for k, w in ARRAYS:
            np.testing.assert_array_equal(got[k][p0:p0 + P], ctx.get_pin_state(w), err_msg="%d %s" % (i, k))
        s1, h1, _, _ = ctx.get_endpoint_slack()
        E = len(s1)
        np.testing.assert_array_equal(es[e0:e0 + E], s1)
        np.testing.assert_array_equal(eh[e0:e0 + E], h1)
        assert bctx.report_slack(design=i) == ctx.report_slack()
        ref = oracle.sta(d)
        assert_close("at", got["at"][p0:p0 + P], ref["at"])
        assert_close("slack", got["slack"][p0:p0 + P], ref["slack"])
        ctx.close()
        p0 += P
        e0 += E
    assert p0 == bctx.P and e0 == bctx.E
    bctx.close()


def test_batch_rejects_mismatched_designs():
    a, b = designs()[:2]
    b = dict(b)
    b["period_ns"] = 2.0
    with pytest.raises(sta.StaError) as ei:
        sta.Context(None, batch=[a, b])
    assert ei.value.status == sta.EINVAL


def test_set_corners_matches_fresh_context():
    d = designs(corners=2)[1]
    ctx = sta.Context(d)
    ctx.set_corners([1.25, 0.9], [1.15, 0.95])
    ctx.update_timing()
    d2 = dict(d)
    d2["lut_scale"] = np.array([1.25, 0.9], np.float32)
    d2["rc_scale"] = np.array([1.15, 0.95], np.float32)
    ref = oracle.sta(d2)
    assert_close("at", ctx.get_pin_state(sta.AT), ref["at"])
    assert_close("rat", ctx.get_pin_state(sta.RAT), ref["rat"])
    ctx.close()


def test_batch_with_exceptions_equals_separate_contexts():
    """Designs with their own timing-exception groups (false, multicycle,
    max/min delay, -through sets) batched together: endpoint slacks and
    flags, the per-design report and the oracle's values agree with separate
    contexts; each group acts on its own design's paths only."""
    ds = designs()[:3]
    rng = np.random.default_rng(4)
    ds[0] = dict(ds[0], **synth.exception_groups(ds[0], rng, 2, actions=(0, 1, 2, 3)))
    ds[2] = dict(ds[2], **synth.exception_groups(ds[2], rng, 3, max_thru=2, actions=(0, 1, 2, 3)))
    bctx = sta.Context(None, batch=ds)
    assert bctx.stats()["n_tags"] == 1 + sum(len(d.get("exc_action", [])) for d in ds) + \
        int(ds[2].get("exc_thru_ptr", [0])[-1])
    for schedule in (sta.SCHED_DATAFLOW, sta.SCHED_COOP, sta.SCHED_TILE):
        bctx.set_schedule(schedule)
        bctx.update_timing()
        es, eh, vs, vh = bctx.get_endpoint_slack()
        e0 = 0
        for i, d in enumerate(ds):
            ctx = sta.Context(d)
            ctx.set_schedule(schedule)
            ctx.update_timing()
            s1, h1, v1, w1 = ctx.get_endpoint_slack()
            E = len(s1)
            np.testing.assert_array_equal(es[e0:e0 + E], s1)
            np.testing.assert_array_equal(eh[e0:e0 + E], h1)
            np.testing.assert_array_equal(vs[e0:e0 + E], v1)
            assert bctx.report_slack(design=i) == ctx.report_slack()
            ref = oracle.sta(d)
            assert_close("ep_setup", es[e0:e0 + E], ref["ep_setup"])
            assert_close("ep_hold", eh[e0:e0 + E], ref["ep_hold"])
            ctx.close()
            e0 += E
    bctx.close()
    many = [dict(d, **synth.exception_groups(d, rng, 3)) for d in designs()[:3]]   # 9 groups
    with pytest.raises(sta.StaError) as ei:
        sta.Context(None, batch=many)
    assert ei.value.status == sta.EINVAL
