"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerance (per element, every AT, slew, RAT and slack): |gpu - oracle| <=
1e-4 ns, or <= 1e-5 relative; infinities equal.  Endpoint violation sets
bit-exact (the clock period sits in a gap wider than twice the tolerance).
WNS/TNS: the FP64 device reduction equals the FP64 sum of the device's own
endpoint slacks, and lies within the summed per-endpoint tolerance of the
oracle's."""
import numpy as np
import pytest

import oracle
from paper_2511_11660_b300 import sta, synth
from tests._parity import assert_close, assert_viol_defined, tune_period

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    sta.load()


def run_both(d, schedule=None, param=0):
    ref = oracle.sta(d)
    ctx = sta.Context(d)
    if schedule is not None:
        ctx.set_schedule(schedule, param)
    ctx.update_timing()
    out = {k: ctx.get_pin_state(w) for k, w in (("at", sta.AT), ("slew", sta.SLEW), ("rat", sta.RAT),
                                                  ("slack", sta.SLACK))}
    out["ep_setup"], out["ep_hold"], out["viol_setup"], out["viol_hold"] = ctx.get_endpoint_slack()
    out["report"] = ctx.report_slack()
    ctx.close()
    return out, ref


def check_all(d, g, ref, exact_viol=True, require_margin=True):
    """Every per-pin array and endpoint slack within tolerance, the FP64
    reductions, and (exact_viol) the setup and hold violation flags and
    counts bit for bit -- after asserting that the oracle's endpoint slacks
    keep clear of zero (require_margin), so that the sets are well
    defined."""
    errs = {}
    for k in ("at", "slew", "rat", "slack"):
        errs[k] = assert_close(k, g[k], ref[k])
    assert_close("ep_setup", g["ep_setup"], ref["ep_setup"])
    assert_close("ep_hold", g["ep_hold"], ref["ep_hold"])
    K = int(d.get("n_corners", 1))
    for k in range(K):
        rep = g["report"][k]
        es = g["ep_setup"][:, k].astype(np.float64)
        eh = g["ep_hold"][:, k].astype(np.float64)
        # the device FP64 reduction of the device's own endpoint slacks
        assert rep["tns_setup"] == pytest.approx(np.minimum(es, 0).sum(), rel=1e-12, abs=1e-12)
        assert rep["tns_hold"] == pytest.approx(np.minimum(eh, 0).sum(), rel=1e-12, abs=1e-12)
        assert rep["wns_setup"] == min(0.0, float(es.min())) if len(es) else True
        # against the oracle: within the summed elementwise tolerance
        nv = max(int(ref["n_viol_setup"][k]), 1)
        assert abs(rep["tns_setup"] - ref["tns_setup"][k]) <= nv * 1e-4 + 1e-5 * abs(ref["tns_setup"][k])
        assert abs(rep["wns_setup"] - ref["wns_setup"][k]) <= 1e-4 + 1e-5 * abs(ref["wns_setup"][k])
        if exact_viol:
            if require_margin:
                assert_viol_defined(ref)
            np.testing.assert_array_equal(g["viol_setup"][:, k], (ref["ep_setup"][:, k] < 0).astype(np.uint8))
            np.testing.assert_array_equal(g["viol_hold"][:, k], (ref["ep_hold"][:, k] < 0).astype(np.uint8))
            assert rep["n_viol_setup"] == ref["n_viol_setup"][k]
            assert rep["n_viol_hold"] == ref["n_viol_hold"][k]
    return errs


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tiny_design_parity(seed):
    d = synth.workload("tiny", seed=seed)
    d["period_ns"], half = tune_period(d)
    g, ref = run_both(d)
    assert 0.05 < ref["n_viol_setup"][0] / len(ref["endpoints"]) < 0.2
    check_all(d, g, ref)


@pytest.mark.parametrize("threads", [32, 64, 256])
def test_block_sizes_and_ragged_levels(threads):
    """Level widths of several blocks with a ragged tail, for three block sizes."""
    d = synth.make_design(6001, 9, seed=7)
    d["period_ns"], _ = tune_period(d)
    g, ref = run_both(d, sta.SCHED_LEVEL, threads)
    check_all(d, g, ref)


def test_multi_corner_parity():
    ls, rs = synth.lut_corners()
    d = synth.make_design(3000, 20, seed=4, n_corners=4, lut_scale=ls, rc_scale=rs, period_ns=1.7)
    g, ref = run_both(d)
    check_all(d, g, ref)


def test_star_rc_from_positions_parity():
    d = synth.make_design(3000, 15, seed=5, placed=True)
    d["period_ns"], _ = tune_period(d)
    g, ref = run_both(d)
    check_all(d, g, ref)


def test_smoothed_merges_parity():
    d = synth.make_design(3000, 15, seed=6, gamma_ns=0.01)
    d["period_ns"], _ = tune_period(d)
    g, ref = run_both(d)
    check_all(d, g, ref)


def test_large_rc_trees_use_global_sweeps():
    """Nets above the shared-memory tile (2048 RC nodes) take the global path.
    R and C are scaled down so that loads stay inside the tables (2,500 nodes
    of the default values would put 7 pF on 0.5 pF tables, where extrapolated
    slews double per stage and the comparison measures conditioning, not the
    kernel)."""
    d = synth.make_design(400, 6, seed=9, rc_nodes=(2000, 3000))
    d["rc_R"] = (d["rc_R"] * 0.1).astype(np.float32)
    d["rc_C"] = (d["rc_C"] * 0.01).astype(np.float32)
    g, ref = run_both(d)
    check_all(d, g, ref)


def test_degenerate_designs():
    lib = synth.make_library(1)
    # PI straight to PO: its hold slack is the bare net delay, near zero, so
    # the flags are compared without the margin precondition
    b = synth.Builder(lib)
    b.po(b.pi())
    d = b.design(period_ns=0.3)
    g, ref = run_both(d)
    check_all(d, g, ref, require_margin=False)
    # flip-flop ring with one gate: Q -> INV -> D of itself, plus an unused output
    b = synth.Builder(lib)
    x = b.pi()
    q = b.cell("DFF", [x])
    z = b.cell("INV", [q])
    q2 = b.cell("DFF", [z])
    b.cell("BUF", [q2])         # output drives nothing: RAT +inf, slack +inf
    b.po(q2)
    d = b.design(period_ns=0.2)
    g, ref = run_both(d)
    check_all(d, g, ref, exact_viol=False)
    assert np.isinf(g["rat"]).any()


def test_single_cell_and_fixed_delay():
    lib = synth.make_library(2, fixed_delay=True)
    d = synth.make_design(1, 1, seed=3, lib=lib)
    g, ref = run_both(d)
    check_all(d, g, ref)
    d = synth.make_design(800, 40, seed=3, lib=lib)
    g, ref = run_both(d)
    check_all(d, g, ref)


def test_repeated_updates_are_identical():
    d = synth.workload("tiny", seed=3)
    ctx = sta.Context(d)
    ctx.update_timing()
    a1 = ctx.get_pin_state(sta.AT).copy()
    r1 = ctx.get_pin_state(sta.RAT).copy()
    ctx.update_timing()
    ctx.update_timing()
    np.testing.assert_array_equal(ctx.get_pin_state(sta.AT), a1)
    np.testing.assert_array_equal(ctx.get_pin_state(sta.RAT), r1)
    ctx.close()


def test_device_outputs_and_views():
    import torch
    d = synth.workload("tiny", seed=4)
    ctx = sta.Context(d)
    ctx.update_timing()
    out = torch.empty((d["n_pins"], 1, 4), dtype=torch.float32, device="cuda")
    ctx.get_pin_state(sta.SLACK, out=out)
    host = ctx.get_pin_state(sta.SLACK)
    np.testing.assert_array_equal(out.cpu().numpy(), host)
    s, h, vs, vh = ctx.get_endpoint_slack(device=True)
    s2, h2, vs2, vh2 = ctx.get_endpoint_slack()
    np.testing.assert_array_equal(s.cpu().numpy(), s2)
    np.testing.assert_array_equal(vs.cpu().numpy(), vs2)
    v = ctx.views()
    assert v["at"] and v["gpu_pin_of"]
    ctx.close()


def test_set_rc_and_set_cell_types_match_fresh_contexts():
    d = synth.make_design(2000, 12, seed=12, lib=synth.make_library(12, strengths=2), period_ns=1.2)
    ctx = sta.Context(d)
    rng = np.random.default_rng(0)
    d2 = dict(d)
    d2["rc_R"] = (d["rc_R"] * rng.uniform(0.5, 1.5, len(d["rc_R"]))).astype(np.float32)
    d2["rc_C"] = (d["rc_C"] * rng.uniform(0.5, 1.5, len(d["rc_C"]))).astype(np.float32)
    ct = d["cell_type"].copy()
    pick = rng.choice(len(ct), 40, replace=False)
    ct[pick] = (ct[pick] + 8) % 16
    d2["cell_type"] = ct
    ctx.set_rc(d2["rc_R"], d2["rc_C"])
    ctx.set_cell_types(ct)
    ctx.update_timing()
    ref = oracle.sta(d2)
    assert_close("at", ctx.get_pin_state(sta.AT), ref["at"])
    assert_close("slack", ctx.get_pin_state(sta.SLACK), ref["slack"])
    ctx.close()


def test_scale_design_sampled_full_size():
    """The 1M-cell workload (depth 150, 2-10 RC nodes) on the default (level)
    schedule: full comparison with the oracle, violation sets bit for bit.
    The schedule the benchmark times is checked at this size in
    test_gpu_dataflow.py."""
    d = synth.workload("scale", seed=0)
    d["period_ns"], half = tune_period(d)
    g, ref = run_both(d)
    errs = check_all(d, g, ref)
    frac = ref["n_viol_setup"][0] / len(ref["endpoints"])
    assert 0.05 < frac < 0.15
    print("1M parity max abs err", {k: v[0] for k, v in errs.items()})


@pytest.mark.parametrize("schedule", [sta.SCHED_LEVEL, sta.SCHED_DATAFLOW, sta.SCHED_COOP, sta.SCHED_TILE])
def test_high_fanout_net(schedule):
    """One primary input drives 1,500 gates (more sinks than a shared-memory
    RC tile holds, so its net is swept in global scratch) and a long fan-out
    list in the backward pass."""
    lib = synth.make_library(4)
    b = synth.Builder(lib)
    a = b.pi()
    outs = [b.cell("INV", [a]) for _ in range(1500)]
    z = b.cell("NAND2", [outs[0], outs[1]])
    b.po(z)
    for o in outs[2:40]:
        b.po(o)
    d = b.design(period_ns=0.4, default_R=2.0, default_C=0.05)
    ref = oracle.sta(d)
    ctx = sta.Context(d)
    ctx.set_schedule(schedule)
    ctx.update_timing()
    for k, w in (("at", sta.AT), ("slew", sta.SLEW), ("rat", sta.RAT), ("slack", sta.SLACK)):
        assert_close(k, ctx.get_pin_state(w), ref[k])
    ctx.close()


@pytest.mark.parametrize("case", ["small", "big", "corners", "order1", "order2"])
def test_arnoldi_net_model_parity(case):
    """STA_NET_ARNOLDI: sink delays from the order-q reduced model, every
    arrival, slew, required time and slack against the FP64 oracle running
    the same model; small trees sweep in shared memory, 20-60 node trees in
    global scratch; every schedule gives the same bits."""
    if case == "big":
        d = synth.make_design(600, 8, seed=9, rc_nodes=(20, 60))
    elif case == "corners":
        ls, rs = synth.lut_corners()
        d = synth.make_design(3000, 20, seed=4, n_corners=4, lut_scale=ls, rc_scale=rs)
    else:
        d = synth.make_design(4000, 25, seed=2, rc_nodes=(2, 16))
    d.update(net_model=sta.NET_ARNOLDI, arnoldi_order={"order1": 1, "order2": 2}.get(case, 3))
    d["period_ns"], _ = tune_period(d)
    ref = oracle.sta(d)
    outs = []
    for sch in (sta.SCHED_LEVEL, sta.SCHED_DATAFLOW, sta.SCHED_COOP, sta.SCHED_TILE):
        ctx = sta.Context(d)
        ctx.set_schedule(sch)
        ctx.update_timing()
        outs.append({k: ctx.get_pin_state(w) for k, w in (("at", sta.AT), ("slew", sta.SLEW), ("rat", sta.RAT),
                                                           ("slack", sta.SLACK))})
        ctx.close()
    for k in ("at", "slew", "rat", "slack"):
        for o in outs[1:]:
            np.testing.assert_array_equal(o[k], outs[0][k], err_msg=k)
        assert_close(k, outs[0][k], ref[k])


def test_set_rc_async_matches_set_rc():
    """sta_set_rc_async: values staged on a copy stream are applied by the
    next update (equal to sta_set_rc's); a later staging before the update
    replaces an earlier one; a synchronous sta_set_rc replaces staged
    values; updates without new staging keep the applied values."""
    import torch
    d = synth.make_design(2000, 12, seed=21, period_ns=1.2)
    rng = np.random.default_rng(3)
    sets = []
    for _ in range(3):
        R = (d["rc_R"] * rng.uniform(0.5, 1.5, len(d["rc_R"]))).astype(np.float32)
        Cc = (d["rc_C"] * rng.uniform(0.5, 1.5, len(d["rc_C"]))).astype(np.float32)
        sets.append((torch.from_numpy(R).pin_memory(), torch.from_numpy(Cc).pin_memory()))
    ref = sta.Context(d)
    ctx = sta.Context(d)
    cs = torch.cuda.Stream()

    def want(i):
        ref.set_rc(sets[i][0].numpy(), sets[i][1].numpy())
        ref.update_timing()
        return ref.get_pin_state(sta.SLACK)

    ctx.set_rc_async(*sets[0], stream=cs)
    ctx.update_timing()
    np.testing.assert_array_equal(ctx.get_pin_state(sta.SLACK), want(0))
    ctx.update_timing()   # nothing staged: the same values
    np.testing.assert_array_equal(ctx.get_pin_state(sta.SLACK), want(0))
    ctx.set_rc_async(*sets[1], stream=cs)
    ctx.set_rc_async(*sets[2], stream=cs)   # replaces the staged set 1
    ctx.update_timing()
    np.testing.assert_array_equal(ctx.get_pin_state(sta.SLACK), want(2))
    ctx.set_rc_async(*sets[1], stream=cs)
    cs.synchronize()
    ctx.set_rc(sets[0][0].numpy(), sets[0][1].numpy())   # the synchronous call wins
    ctx.update_timing()
    np.testing.assert_array_equal(ctx.get_pin_state(sta.SLACK), want(0))
    # alternate two staged sets while updates run, as a placement loop would
    for i in range(6):
        ctx.set_rc_async(*sets[i % 2], stream=cs)
        ctx.update_timing()
        np.testing.assert_array_equal(ctx.get_pin_state(sta.SLACK), want(i % 2))
    ctx.close()
    ref.close()
