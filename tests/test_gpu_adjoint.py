"""GPU differentiable timing: the smoothed objective and its adjoint
(sta_backward) against the FP64 oracle (orc_objective_grad), whose adjoint is
itself pinned to central finite differences (tests/test_oracle_pins.py).

Tolerances (the adjoint runs in FP32, its sums in FP64): J within 1e-5
relative; every gradient component within 1e-3 * max|g*| + 1e-3 * |g*|."""
import numpy as np
import pytest

import oracle
from paper_2511_11660_b300 import sta, synth
from tests._parity import tune_period

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    sta.load()


def gpu_grad(d, w=(1.0, 1.0), schedule=sta.SCHED_DATAFLOW):
    ctx = sta.Context(d)
    ctx.set_schedule(schedule)
    ctx.update_timing()
    J, terms, g = ctx.backward(*w)
    ctx.close()
    return J, terms, g


def check_grad(g, ref, tol=1e-3):
    scale = np.abs(ref).max()
    err = np.abs(g - ref)
    bad = err > tol * scale + tol * np.abs(ref)
    assert not bad.any(), "max err %.3g (scale %.3g) at %s" % (err.max(), scale, np.argwhere(bad)[:3].tolist())
    return float(err.max() / scale)


def placed(n, depth, seed, **kw):
    d = synth.make_design(n, depth, seed=seed, placed=True, gamma_ns=0.01, **kw)
    d["period_ns"], _ = tune_period(d, min_half_gap=0.0)
    return d


@pytest.mark.parametrize("w", [(1.0, 1.0), (1.0, 0.0), (0.0, 1.0)])
def test_objective_and_gradient_small(w):
    d = placed(3000, 20, 3)
    J, terms, g = gpu_grad(d, w)
    J0, terms0, g0 = oracle.objective_grad(d, *w)
    assert J == pytest.approx(J0, rel=1e-5)
    np.testing.assert_allclose(terms, terms0, rtol=1e-5)
    check_grad(g, g0)


@pytest.mark.parametrize("schedule", [sta.SCHED_DATAFLOW, sta.SCHED_COOP, sta.SCHED_TILE],
                         ids=["dataflow", "coop", "tile"])
def test_every_forward_schedule_gives_the_same_gradient(schedule):
    d = placed(2000, 15, 4)
    a = gpu_grad(d, schedule=schedule)
    b = gpu_grad(d, schedule=sta.SCHED_LEVEL)
    assert a[0] == b[0]
    np.testing.assert_allclose(a[2], b[2], rtol=1e-9, atol=1e-12 * np.abs(b[2]).max())


def test_adjoint_schedules_give_the_same_gradient():
    """The reverse sweep as one persistent kernel or one launch per level:
    the same objective, and gradients equal up to the order of the FP64
    atomic sums."""
    d = placed(2000, 15, 5)
    out = []
    for sch in (sta.SCHED_DATAFLOW, sta.SCHED_LEVEL):
        ctx = sta.Context(d)
        ctx.set_adjoint_schedule(sch)
        ctx.update_timing()
        out.append(ctx.backward(1.0, 1.0))
        ctx.close()
    assert out[0][0] == out[1][0]
    np.testing.assert_allclose(out[0][2], out[1][2], rtol=1e-9, atol=1e-12 * np.abs(out[1][2]).max())


def test_four_corner_objective_and_gradient():
    ls, rs = synth.lut_corners()
    d = placed(2000, 15, 5, n_corners=4, lut_scale=ls, rc_scale=rs)
    J, terms, g = gpu_grad(d)
    J0, terms0, g0 = oracle.objective_grad(d)
    assert J == pytest.approx(J0, rel=1e-5)
    np.testing.assert_allclose(terms, terms0, rtol=1e-5)
    check_grad(g, g0)


def test_device_outputs_and_autograd():
    import torch
    from paper_2511_11660_b300.autograd import smoothed_objective
    d = placed(1500, 12, 6)
    ctx = sta.Context(d)
    ctx.set_schedule(sta.SCHED_DATAFLOW)
    xy = torch.tensor(d["cell_xy"], dtype=torch.float32, device="cuda", requires_grad=True)
    J = smoothed_objective(xy, ctx)
    J.backward()
    J0, _, g0 = oracle.objective_grad(d)
    assert float(J.detach()) == pytest.approx(J0, rel=1e-5)
    check_grad(xy.grad.double().cpu().numpy().reshape(-1, 2), g0)
    ctx.close()


def _steiner_design(case):
    if case == "fanout":
        # nets of 80 pins (minimum spanning tree) and 20-63 pins: trees of more
        # than 16 nodes, whose adjoint works in global scratch
        bld = synth.Builder(synth.make_library(0))
        rng = np.random.default_rng(2)
        pi = bld.pi(xy=(10.0, 10.0))
        for _ in range(80):
            bld.po(pi, xy=tuple(float(v) for v in rng.uniform(0, 300, 2)))
        for k in (20, 40, 63):
            x = bld.cell("BUF", [pi], xy=tuple(float(v) for v in rng.uniform(0, 300, 2)))
            for _ in range(k):
                bld.po(x, xy=tuple(float(v) for v in rng.uniform(0, 300, 2)))
        d = bld.design(placed=True, period_ns=2.0)
        d["gamma_ns"] = 0.01
    else:
        kw = {}
        if case == "corners":
            ls, rs = synth.lut_corners()
            kw = dict(n_corners=4, lut_scale=ls, rc_scale=rs)
        d = synth.make_design(3000, 20, seed=7, placed=True, placement="local", gamma_ns=0.01, **kw)
    d["wire_model"] = 1
    d["r_per_um"] = 0.5
    if case == "xy":
        d["r_per_um_y"], d["c_per_um_y"] = 0.3, 0.35
    d["period_ns"], _ = tune_period(d, min_half_gap=0.0)
    return d


@pytest.mark.parametrize("case", ["local", "xy", "corners", "fanout"])
@pytest.mark.parametrize("adj_schedule", [sta.SCHED_DATAFLOW, sta.SCHED_LEVEL], ids=["adj_dataflow", "adj_level"])
def test_steiner_gradient(case, adj_schedule):
    """Steiner-tree RC (STA_WIRE_STEINER) with the trees of the update held
    fixed: J, the per-corner terms and every gradient component against the
    oracle, whose Steiner adjoint is pinned to central differences."""
    d = _steiner_design(case)
    ctx = sta.Context(d)
    ctx.set_adjoint_schedule(adj_schedule)
    ctx.update_timing()
    J, terms, g = ctx.backward()
    ctx.close()
    J0, terms0, g0 = oracle.objective_grad(d)
    assert J == pytest.approx(J0, rel=1e-5)
    np.testing.assert_allclose(terms, terms0, rtol=1e-5)
    check_grad(g, g0)
    assert np.abs(g0).max() > 0


def test_backward_state_errors():
    d = synth.make_design(300, 5, seed=1)              # RC trees: not differentiable
    ctx = sta.Context(d)
    with pytest.raises(sta.StaError) as ei:
        ctx.backward()
    assert ei.value.status == sta.ESTATE
    ctx.close()
    d = placed(300, 5, 1)
    ctx = sta.Context(d)
    with pytest.raises(sta.StaError) as ei:
        ctx.backward()                                  # before any update
    assert ei.value.status == sta.ESTATE
    ctx.close()
    d = dict(placed(300, 5, 1), wire_model=1, net_model=1)   # Steiner with Arnoldi delays
    ctx = sta.Context(d)
    ctx.update_timing()
    with pytest.raises(sta.StaError) as ei:
        ctx.backward()
    assert ei.value.status == sta.ESTATE
    ctx.close()


def test_diff_workload_200k_against_oracle_and_differences():
    """The 200k-cell placed workload (star RC, gamma 0.01 ns): J and every
    gradient component against the FP64 oracle, then central differences
    (h = 1e-3 um) of the oracle's objective on 100 uniformly random cells
    and 20 of the 200 with the largest gradients (both axes) against the GPU
    gradient, with the per-component bound
    |g - fd| <= 1e-3 max|g*| + 1e-3 |fd|.  A component whose one-sided
    differences within +-h disagree by more than that bound has crossed a
    kink (a Manhattan |dx| = 0) or a table breakpoint, where the derivative
    is not defined at this resolution: it is counted as excluded, and at
    most 5% may be."""
    import multiprocessing as mp
    import os

    from tests import _fd
    d = synth.workload("diff", seed=0)
    d["period_ns"], _ = tune_period(d, min_half_gap=0.0)
    J, terms, g = gpu_grad(d)
    J0, terms0, g0 = oracle.objective_grad(d)
    assert J == pytest.approx(J0, rel=1e-5)
    rel = check_grad(g, g0)
    rng = np.random.default_rng(0)
    cells = rng.choice(d["n_cells"], 100, replace=False)
    # most random cells barely touch the critical endpoints (their gradient
    # is exponentially small under the smoothing): 20 more from the 200
    # largest gradients exercise large components too
    big = np.argsort(-np.abs(g0).max(1))[:200]
    cells = np.concatenate([cells, rng.choice(np.setdiff1d(big, cells), 20, replace=False)])
    h = 1e-3
    tasks = [(0, 0, 0.0)] + [(int(c), ax, sg * h) for c in cells for ax in (0, 1) for sg in (1.0, -1.0)]
    workers = max(1, min(16, (os.cpu_count() or 1)))
    with mp.get_context("spawn").Pool(workers, initializer=_fd.init, initargs=("diff", 0, d["period_ns"])) as pool:
        res = pool.map(_fd.objective_at, tasks, chunksize=4)
    Jc = res[0][0]
    assert Jc == pytest.approx(J0, rel=1e-12)
    scale = np.abs(g0).max()
    excluded, checked, worst, nonzero = 0, 0, 0.0, 0
    for i, c in enumerate(cells):
        for ax in (0, 1):
            (jp, xp), (jm, xm) = res[1 + 4 * i + 2 * ax], res[2 + 4 * i + 2 * ax]
            x0 = float(d["cell_xy"][2 * c + ax])
            fd = (jp - jm) / (xp - xm)
            fwd, bwd = (jp - Jc) / (xp - x0), (Jc - jm) / (x0 - xm)
            bound = 1e-3 * scale + 1e-3 * abs(fd)
            if abs(fwd - bwd) > bound:
                excluded += 1
                continue
            checked += 1
            nonzero += abs(fd) > 1e-6 * scale
            err = abs(fd - g[c, ax])
            worst = max(worst, err / bound)
            assert err <= bound, (int(c), ax, fd, float(g[c, ax]), err, bound)
    assert excluded <= 12, excluded
    assert nonzero >= 30, nonzero
    print("200k gradient: max error / max|g| = %.2e; central differences on %d components (%d above 1e-6 max|g|, "
          "%d excluded), worst error / bound = %.3f" % (rel, checked, nonzero, excluded, worst))


def test_large_library_uses_level_sweeps():
    """A 64-type library does not fit the dataflow kernels' shared-memory copy:
    the dataflow schedule is refused and the adjoint falls back to one launch
    per level; results still match the oracle."""
    lib = synth.make_library(9, strengths=8)
    d = synth.make_design(1500, 12, seed=9, lib=lib, placed=True, gamma_ns=0.01)
    rng = np.random.default_rng(1)
    ct = d["cell_type"].copy()
    ct += 8 * rng.integers(0, 8, size=len(ct))        # spread cells over the drive strengths
    d["cell_type"] = ct.astype(np.int32)
    d["period_ns"], _ = tune_period(d, min_half_gap=0.0)
    ctx = sta.Context(d)
    with pytest.raises(sta.StaError) as ei:
        ctx.set_schedule(sta.SCHED_DATAFLOW)
    assert ei.value.status == sta.EINVAL
    ctx.update_timing()
    J, terms, g = ctx.backward()
    J0, terms0, g0 = oracle.objective_grad(d)
    assert J == pytest.approx(J0, rel=1e-5)
    check_grad(g, g0)
    ctx.close()
