"""GPU tests of the persistent dataflow schedule.

The dataflow kernels run the same per-item arithmetic as the level kernels
(item.cuh), so the two schedules must agree bit for bit; both are also held to
the FP64 oracle.  The failure-detection test makes a result that nothing
sets (a test hook withholds one cell's results), lets the bounded waits run out,
and checks that the host gets STA_ETIMEOUT and that the context still works."""
import numpy as np
import pytest

import oracle
from paper_2511_11660_b300 import sta, synth
from tests._parity import assert_close, tune_period
from tests.test_gpu_parity import check_all

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    sta.load()


ARRAYS = (("at", sta.AT), ("slew", sta.SLEW), ("rat", sta.RAT), ("slack", sta.SLACK))


def run(d, schedule, param=0):
    ctx = sta.Context(d)
    ctx.set_schedule(schedule, param)
    ctx.update_timing()
    out = {k: ctx.get_pin_state(w) for k, w in ARRAYS}
    out["ep_setup"], out["ep_hold"], out["viol_setup"], out["viol_hold"] = ctx.get_endpoint_slack()
    out["report"] = ctx.report_slack()
    ctx.close()
    return out


def same(a, b):
    for k, _ in ARRAYS:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    np.testing.assert_array_equal(a["ep_setup"], b["ep_setup"])
    np.testing.assert_array_equal(a["viol_setup"], b["viol_setup"])
    assert a["report"] == b["report"]


def _case(case):
    if case == "tiny":
        d = synth.workload("tiny", seed=1)
        d["period_ns"], _ = tune_period(d)
    elif case == "corners":
        ls, rs = synth.lut_corners()
        d = synth.make_design(3000, 20, seed=4, n_corners=4, lut_scale=ls, rc_scale=rs, period_ns=1.7)
    elif case == "star":
        d = synth.make_design(3000, 15, seed=5, placed=True)
        d["period_ns"], _ = tune_period(d)
    elif case == "smooth":
        d = synth.make_design(3000, 15, seed=6, gamma_ns=0.01)
        d["period_ns"], _ = tune_period(d)
    elif case == "fixed":
        d = synth.make_design(800, 40, seed=3, lib=synth.make_library(2, fixed_delay=True))
    else:
        d = synth.make_design(400, 6, seed=9, rc_nodes=(2000, 3000))
        d["rc_R"] = (d["rc_R"] * 0.1).astype(np.float32)
        d["rc_C"] = (d["rc_C"] * 0.01).astype(np.float32)
    return d


CASES = ["tiny", "corners", "star", "smooth", "fixed", "big_rc"]


PERSISTENT = [sta.SCHED_DATAFLOW, sta.SCHED_COOP, sta.SCHED_TILE]
PERSISTENT_IDS = ["dataflow", "coop", "tile"]


@pytest.mark.parametrize("schedule", PERSISTENT, ids=PERSISTENT_IDS)
@pytest.mark.parametrize("case", CASES)
def test_persistent_schedules_match_level_and_oracle(case, schedule):
    d = _case(case)
    g = run(d, schedule)
    same(g, run(d, sta.SCHED_LEVEL))
    ref = oracle.sta(d)
    check_all(d, g, ref)


@pytest.mark.parametrize("schedule", PERSISTENT, ids=PERSISTENT_IDS)
@pytest.mark.parametrize("blocks", [1, 3, 148])
def test_small_persistent_grids_make_progress(blocks, schedule):
    """One resident block (8 warps) must still finish: dataflow chunks are
    taken in order and only wait for earlier chunks; the cooperative grid
    strides over every level whatever its size; a tile schedule of one
    tile runs every level in one block (many waves per level, most ring
    slots overwritten before use, so most reads go through the mailbox)."""
    d = synth.make_design(5000, 40, seed=11, period_ns=2.5)
    same(run(d, schedule, blocks), run(d, sta.SCHED_LEVEL))


@pytest.mark.parametrize("schedule", PERSISTENT, ids=PERSISTENT_IDS)
def test_degenerate_designs_persistent(schedule):
    lib = synth.make_library(1)
    b = synth.Builder(lib)
    b.po(b.pi())
    d = b.design(period_ns=0.3)
    same(run(d, schedule), run(d, sta.SCHED_LEVEL))
    b = synth.Builder(lib)
    x = b.pi()
    q = b.cell("DFF", [x])
    z = b.cell("INV", [q])
    q2 = b.cell("DFF", [z])
    b.cell("BUF", [q2])
    b.po(q2)
    d = b.design(period_ns=0.2)
    g = run(d, schedule)
    same(g, run(d, sta.SCHED_LEVEL))
    check_all(d, g, oracle.sta(d), exact_viol=False)
    d = synth.make_design(1, 1, seed=3)
    same(run(d, schedule), run(d, sta.SCHED_LEVEL))


@pytest.mark.parametrize("schedule", [sta.SCHED_DATAFLOW, sta.SCHED_TILE], ids=["dataflow", "tile"])
def test_repeated_dataflow_updates_are_identical(schedule):
    d = synth.workload("tiny", seed=2)
    ctx = sta.Context(d)
    ctx.set_schedule(schedule)
    ctx.update_timing()
    first = {k: ctx.get_pin_state(w).copy() for k, w in ARRAYS}
    for _ in range(3):
        ctx.update_timing()
    for k, w in ARRAYS:
        np.testing.assert_array_equal(ctx.get_pin_state(w), first[k])
    ctx.close()


@pytest.mark.parametrize("schedule", [sta.SCHED_DATAFLOW, sta.SCHED_TILE], ids=["dataflow", "tile"])
def test_wait_limit_reports_timeout_and_context_recovers(schedule):
    d = synth.workload("tiny", seed=0)
    ref = oracle.sta(d)
    ctx = sta.Context(d)
    ctx.set_schedule(schedule)
    ctx.update_timing()
    ctx.sync()
    # a gate of level 1: its output flag is withheld, its fan-out waits run out
    levels = sta.sta_plan_levels(d)
    cell = int(np.nonzero(levels == 1)[0][0])
    ctx.set_wait_limit(20000)
    ctx.debug_hold_cell(cell)
    ctx.update_timing()
    with pytest.raises(sta.StaError) as ei:
        ctx.sync()
    assert ei.value.status == sta.ETIMEOUT
    # the same context, hook removed: a normal, correct pass
    ctx.debug_hold_cell(-1)
    ctx.set_wait_limit(1 << 23)
    ctx.update_timing()
    ctx.sync()
    assert_close("at", ctx.get_pin_state(sta.AT), ref["at"])
    assert_close("slack", ctx.get_pin_state(sta.SLACK), ref["slack"])
    ctx.close()


def test_coop_barrier_wait_limit_reports_timeout_and_context_recovers():
    """A one-poll limit on the grid barrier: blocks that reach a barrier
    before the last one arrives give up at once, the update reports
    STA_ETIMEOUT, and the same context then runs a normal, correct pass."""
    d = synth.make_design(20000, 60, seed=5, period_ns=2.5)
    ref = oracle.sta(d)
    ctx = sta.Context(d)
    ctx.set_schedule(sta.SCHED_COOP)
    ctx.update_timing()
    ctx.sync()
    ctx.set_wait_limit(1)
    ctx.update_timing()
    with pytest.raises(sta.StaError) as ei:
        ctx.sync()
    assert ei.value.status == sta.ETIMEOUT
    ctx.set_wait_limit(1 << 23)
    ctx.update_timing()
    ctx.sync()
    assert_close("at", ctx.get_pin_state(sta.AT), ref["at"])
    assert_close("slack", ctx.get_pin_state(sta.SLACK), ref["slack"])
    ctx.close()


def test_scale_design_persistent_full_size():
    """The 1M-cell workload under the dataflow, cooperative and tile
    schedules, against the oracle and bit-identical to the level schedule."""
    d = synth.workload("scale", seed=0)
    d["period_ns"], _ = tune_period(d)
    lv = run(d, sta.SCHED_LEVEL)
    ref = oracle.sta(d)
    for schedule in (sta.SCHED_DATAFLOW, sta.SCHED_COOP, sta.SCHED_TILE):
        g = run(d, schedule)
        same(g, lv)
        check_all(d, g, ref)


def test_tile_schedule_rejects_more_tiles_than_resident_blocks():
    d = synth.make_design(2000, 20, seed=3)
    ctx = sta.Context(d)
    with pytest.raises(sta.StaError) as ei:
        ctx.set_schedule(sta.SCHED_TILE, 60000)
    assert ei.value.status == sta.EINVAL
    # the context still works on another schedule
    ctx.set_schedule(sta.SCHED_TILE, 0)
    ctx.update_timing()
    ctx.sync()
    info = ctx.tile_info()
    assert info["n_tiles"] > 0 and info["crit_local"] <= info["crit_edges"]
    ctx.close()


def test_autotune_selects_a_schedule_and_keeps_results():
    import time
    d = synth.make_design(20000, 40, seed=13, period_ns=3.0)
    ref = oracle.sta(d)
    ctx = sta.Context(d)
    sch, par, ms = ctx.autotune(trials=3)
    assert sch in (sta.SCHED_LEVEL, sta.SCHED_DATAFLOW, sta.SCHED_COOP, sta.SCHED_TILE) and ms > 0
    assert_close("at", ctx.get_pin_state(sta.AT), ref["at"])
    assert_close("slack", ctx.get_pin_state(sta.SLACK), ref["slack"])
    t0 = time.perf_counter()
    again = ctx.autotune(trials=3)            # cached choice for this shape
    assert again[:2] == (sch, par) and time.perf_counter() - t0 < 1.0
    ctx.close()
