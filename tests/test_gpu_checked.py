"""The bounds-checking debug build (libsta_checked.so, compiled with
-DSTA_CHECKS): every index a kernel derives from plan data is range-checked
on the device, and a violation sets the bounds bit of the device error word,
which the next synchronising call reports.  This runs representative cases
through that build -- every schedule, several corners, a batch, large RC
trees swept in global scratch, star RC, Steiner trees (all three Steiner
kernels) with the Arnoldi model, exceptions with -through sets, the adjoint
on stars and on Steiner trees, and the path report -- in a child process
(the binding holds one library per process), checks them against the FP64
oracle and requires that no check fired."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
sys.path.insert(0, ROOT)
import numpy as np
import oracle
from paper_2511_11660_b300 import build, sta, synth
from tests._parity import assert_close

sta.load(build.build(checked=True))
ls, rs = synth.lut_corners()
cases = {
    "tiny": synth.workload("tiny", seed=1),
    "corners": synth.make_design(3000, 20, seed=4, n_corners=4, lut_scale=ls, rc_scale=rs, period_ns=1.7),
    "big_rc": synth.make_design(400, 6, seed=9, rc_nodes=(20, 60)),
    "star_smooth": synth.make_design(3000, 15, seed=6, placed=True, gamma_ns=0.01, period_ns=1.5),
    "steiner_arnoldi": dict(synth.make_design(3000, 15, seed=7, placed=True, period_ns=1.5), wire_model=1,
                            net_model=1, arnoldi_order=3),
}
# exceptions with -through sets on 4 corners
exc = synth.make_design(3000, 20, seed=8, n_corners=4, lut_scale=ls, rc_scale=rs, period_ns=1.7)
exc.update(synth.exception_groups(exc, np.random.default_rng(8), 3, max_thru=2))
cases["exceptions_through"] = exc
# a net of 80 pins (minimum spanning tree only) and nets of 20-63 pins (warp kernel)
bld = synth.Builder(synth.make_library(0))
rng = np.random.default_rng(2)
pi = bld.pi(xy=(10.0, 10.0))
for _ in range(80):
    bld.po(pi, xy=tuple(float(v) for v in rng.uniform(0, 500, 2)))
for k in (20, 40, 63):
    x = bld.cell("BUF", [pi], xy=tuple(float(v) for v in rng.uniform(0, 500, 2)))
    for _ in range(k):
        bld.po(x, xy=tuple(float(v) for v in rng.uniform(0, 500, 2)))
fan = bld.design(placed=True, period_ns=2.0)
fan["wire_model"] = 1
cases["steiner_fanout"] = fan
# the Steiner adjoint: trees in shared-memory columns and (the large nets) in global scratch
cases["steiner_grad"] = dict(synth.make_design(3000, 15, seed=5, placed=True, placement="local", gamma_ns=0.01,
                                               period_ns=1.0), wire_model=1)
cases["steiner_fanout_grad"] = dict(fan, gamma_ns=0.01)
for name, d in cases.items():
    ref = oracle.sta(d)
    for sch in (sta.SCHED_LEVEL, sta.SCHED_DATAFLOW, sta.SCHED_COOP, sta.SCHED_TILE):
        ctx = sta.Context(d)
        ctx.set_schedule(sch)
        ctx.update_timing()
        if d.get("gamma_ns", 0) > 0:
            ctx.backward(1.0, 1.0)
        ctx.report_paths(64)
        ctx.sync()
        assert_close("at", ctx.get_pin_state(sta.AT), ref["at"])
        assert_close("slack", ctx.get_pin_state(sta.SLACK), ref["slack"])
        ctx.close()
batch = synth.batch_workload(seed=0, n_designs=3, lo=500, hi=3000, depth=12)
b = sta.Context(None, batch=batch)
for sch in (sta.SCHED_LEVEL, sta.SCHED_DATAFLOW, sta.SCHED_COOP, sta.SCHED_TILE):
    b.set_schedule(sch)
    b.update_timing()
    b.sync()
b.close()
print("CHECKED-OK")
'''


def test_checked_build_runs_clean():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], cwd=ROOT, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0 and "CHECKED-OK" in r.stdout, (r.stdout[-2000:], r.stderr[-4000:])
