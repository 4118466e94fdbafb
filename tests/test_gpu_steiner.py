"""GPU Steiner-tree RC from positions (STA_WIRE_STEINER) against the oracle.

The tree construction is integer work on nm coordinates: every net's tree
length must equal the oracle's exactly.  Delays, slews, required times and
slacks built on the trees follow the usual tolerance (1e-4 ns or 1e-5
relative), endpoint violation sets bit-exact."""
import numpy as np
import pytest

import oracle
from paper_2511_11660_b300 import sta, synth
from tests._parity import tune_period
from tests.test_gpu_parity import check_all

pytestmark = pytest.mark.gpu

SCHEDULES = [sta.SCHED_LEVEL, sta.SCHED_DATAFLOW, sta.SCHED_COOP, sta.SCHED_TILE]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    sta.load()


def _steiner(d, ry=0.13, cy=0.25):
    d.update(wire_model=sta.WIRE_STEINER, r_per_um_y=ry, c_per_um_y=cy)
    return d


def _gpu(ctx):
    out = {k: ctx.get_pin_state(w) for k, w in (("at", sta.AT), ("slew", sta.SLEW), ("rat", sta.RAT),
                                                  ("slack", sta.SLACK))}
    out["ep_setup"], out["ep_hold"], out["viol_setup"], out["viol_hold"] = ctx.get_endpoint_slack()
    out["report"] = ctx.report_slack()
    return out


def _fanout_design(seed):
    """Nets of every size class: a PI driving 80 POs (> 64 pins: MST only),
    buffers driving 20-63 sinks (bitsets over several words), and a random
    placed logic cloud; positions in a 1000 um die."""
    rng = np.random.default_rng(seed)
    lib = synth.make_library(0)
    b = synth.Builder(lib)
    xy = lambda: tuple(float(v) for v in rng.uniform(0, 1000, 2))  # noqa: E731
    a = b.pi(xy=xy())
    for _ in range(80):
        b.po(a, xy=xy())
    for k in (20, 40, 63):
        x = b.cell("BUF", [a], xy=xy())
        for _ in range(k):
            y = b.cell("INV", [x], xy=xy())
            b.po(y, xy=xy())
    return b.design(placed=True)


@pytest.mark.parametrize("case", ["tiny", "corners", "fanout", "arnoldi"])
def test_steiner_parity_all_schedules(case):
    if case == "corners":
        ls, rs = synth.lut_corners()
        d = synth.make_design(3000, 20, seed=5, placed=True, n_corners=4, lut_scale=ls, rc_scale=rs)
    elif case == "fanout":
        d = _fanout_design(1)
    else:
        d = synth.make_design(3000, 20, seed=3, placed=True)
    _steiner(d)
    if case == "arnoldi":
        d.update(net_model=sta.NET_ARNOLDI, arnoldi_order=3)
    d["period_ns"], _ = tune_period(d)
    ref = oracle.sta(d)
    wl = oracle.net_wirelengths(d)
    ctx = sta.Context(d)
    for sch in SCHEDULES:
        ctx.set_schedule(sch)
        ctx.update_timing()
        np.testing.assert_array_equal(ctx.get_net_wirelength(), wl)
        check_all(d, _gpu(ctx), ref)
    ctx.close()


def test_steiner_differs_from_star_and_is_shorter():
    """The Steiner trees change the timing against the star, and every net's
    tree is no longer than the star's total segment length."""
    d = _steiner(synth.make_design(3000, 20, seed=7, placed=True), ry=0.0, cy=0.0)
    star = dict(d, wire_model=sta.WIRE_STAR)
    ctx = sta.Context(d)
    ctx.update_timing()
    wl = ctx.get_net_wirelength()
    s_st = ctx.get_endpoint_slack()[0]
    ctx.close()
    c2 = sta.Context(star)
    c2.update_timing()
    s_star = c2.get_endpoint_slack()[0]
    c2.close()
    assert not np.allclose(s_st, s_star)
    from tests import _indep
    net = _indep.Net(star)
    npp, npn = d["net_pin_ptr"], d["net_pin"]
    for m in range(0, d["n_nets"], 7):
        pins = npn[npp[m]:npp[m + 1]]
        dx, dy = net.pos(int(pins[0]))
        star_nm = sum(abs(oracle.nm(net.pos(int(p))[0]) - oracle.nm(dx)) +
                      abs(oracle.nm(net.pos(int(p))[1]) - oracle.nm(dy)) for p in pins[1:])
        assert wl[m] <= star_nm


def test_steiner_positions_update_and_device_output():
    """sta_set_positions rebuilds the trees at the next update; the
    wirelength also lands in a device tensor."""
    import torch
    d = _steiner(synth.make_design(2000, 15, seed=9, placed=True))
    d["period_ns"], _ = tune_period(d)
    ctx = sta.Context(d)
    ctx.update_timing()
    rng = np.random.default_rng(4)
    xy = (np.asarray(d["cell_xy"], np.float32) + rng.normal(0, 20, len(d["cell_xy"])).astype(np.float32))
    xy = np.clip(xy, 0, 1000).astype(np.float32)
    ctx.set_positions(torch.tensor(xy, device="cuda"))
    ctx.update_timing()
    d2 = dict(d, cell_xy=xy)
    np.testing.assert_array_equal(ctx.get_net_wirelength(device=True).cpu().numpy(), oracle.net_wirelengths(d2))
    # randomly moved cells: a position-update test, whose endpoint slacks are
    # not placed in a gap, so the flags are left out
    check_all(d2, _gpu(ctx), oracle.sta(d2), exact_viol=False)
    ctx.close()


def test_steiner_batch_equals_separate_contexts():
    lib = synth.make_library(0)
    ds = [_steiner(synth.make_design(n, 12, seed=s, lib=lib, placed=True)) for s, n in enumerate([900, 2500, 1600])]
    b = sta.Context(None, batch=ds)
    b.update_timing()
    wl = b.get_net_wirelength()
    off = 0
    for i, d in enumerate(ds):
        c = sta.Context(d)
        c.update_timing()
        np.testing.assert_array_equal(wl[off:off + d["n_nets"]], c.get_net_wirelength())
        assert b.report_slack(design=i) == c.report_slack()
        c.close()
        off += d["n_nets"]
    b.close()


def test_steiner_errors():
    d = synth.make_design(500, 8, seed=1, placed=True)
    ctx = sta.Context(d)   # star
    ctx.update_timing()
    with pytest.raises(sta.StaError):
        ctx.get_net_wirelength()
    ctx.close()
    ctx = sta.Context(_steiner(dict(d)))
    with pytest.raises(sta.StaError):
        ctx.get_net_wirelength()   # before the first update
    ctx.update_timing()
    assert len(ctx.get_net_wirelength()) == d["n_nets"]
    with pytest.raises(sta.StaError):
        ctx.backward(1.0, 1.0)
    ctx.close()


def test_steiner_full_size():
    """1M placed cells: every net's tree length exact, endpoint slacks and
    WNS/TNS against the oracle."""
    d = _steiner(synth.make_design(1_000_000, 150, seed=0, placed=True))
    d["period_ns"], _ = tune_period(d)
    ref = oracle.sta(d)
    ctx = sta.Context(d)
    ctx.update_timing()
    np.testing.assert_array_equal(ctx.get_net_wirelength(), oracle.net_wirelengths(d))
    g = _gpu(ctx)
    from tests._parity import assert_close
    assert_close("ep_setup", g["ep_setup"], ref["ep_setup"])
    assert_close("ep_hold", g["ep_hold"], ref["ep_hold"])
    np.testing.assert_array_equal(g["viol_setup"][:, 0], (ref["ep_setup"][:, 0] < 0).astype(np.uint8))
    ctx.close()
