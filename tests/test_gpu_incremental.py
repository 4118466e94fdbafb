"""Incremental differentiable timing (the large-workload loop at reduced
size): each iteration moves 1% of the cells by U(-5, 5) um and resizes 1% of
the cells to the other drive strength (tables x 0.7), then runs the timing
pass and the smoothed-objective gradient on the same context.  After every
iteration the context must agree with a fresh FP64 oracle run on the edited
design."""
import numpy as np
import pytest

import oracle
from paper_2511_11660_b300 import sta, synth
from tests._parity import assert_close
from tests.test_gpu_adjoint import check_grad

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    sta.load()


def test_moves_and_resizes_track_the_oracle():
    import torch
    ls, rs = synth.lut_corners()
    d = synth.make_design(20000, 40, seed=17, placed=True, gamma_ns=0.01, n_corners=4, lut_scale=ls, rc_scale=rs,
                          lib=synth.make_library(17, strengths=2), period_ns=30.0)
    ctx = sta.Context(d)
    ctx.set_schedule(sta.SCHED_DATAFLOW)
    rng = np.random.default_rng(0)
    C = d["n_cells"]
    xy = d["cell_xy"].astype(np.float32).copy()
    types = d["cell_type"].copy()
    for it in range(3):
        mv = rng.choice(C, C // 100, replace=False)
        xy.reshape(-1, 2)[mv] += rng.uniform(-5, 5, size=(len(mv), 2)).astype(np.float32)
        rz = rng.choice(C, C // 100, replace=False)
        types[rz] = np.where(types[rz] < 8, types[rz] + 8, types[rz] - 8)
        ctx.set_positions(torch.tensor(xy, device="cuda"))
        ctx.set_cell_types(types)
        ctx.update_timing()
        J, terms, g = ctx.backward()
        de = dict(d)
        de["cell_xy"] = xy.copy()
        de["cell_type"] = types.copy()
        ref = oracle.sta(de)
        assert_close("at", ctx.get_pin_state(sta.AT), ref["at"])
        assert_close("rat", ctx.get_pin_state(sta.RAT), ref["rat"])
        J0, terms0, g0 = oracle.objective_grad(de)
        assert J == pytest.approx(J0, rel=1e-5), it
        check_grad(g, g0)
    ctx.close()


def test_device_resize_equals_full_type_update():
    import torch
    lib = synth.make_library(5, strengths=2)
    d = synth.make_design(5000, 20, seed=5, lib=lib, period_ns=2.0)
    rng = np.random.default_rng(1)
    cells = rng.choice(d["n_cells"], 300, replace=False).astype(np.int32)
    types = d["cell_type"][cells]
    types = np.where(types < 8, types + 8, types - 8).astype(np.int32)
    a = sta.Context(d)
    a.resize_cells(torch.tensor(cells, device="cuda"), torch.tensor(types, device="cuda"))
    a.update_timing()
    full = d["cell_type"].copy()
    full[cells] = types
    b = sta.Context(d)
    b.set_cell_types(full)
    b.update_timing()
    for w in (sta.AT, sta.SLEW, sta.RAT, sta.SLACK):
        np.testing.assert_array_equal(a.get_pin_state(w), b.get_pin_state(w))
    # a type that changes the input count is refused on the device
    bad = np.array([int(np.nonzero(d["cell_type"] == 0)[0][0])], np.int32)   # an INV
    a.resize_cells(bad, np.array([2], np.int32))                             # NAND2 has two inputs
    with pytest.raises(sta.StaError) as ei:
        a.sync()
    assert ei.value.status == sta.EINVAL
    a.close()
    b.close()
