"""The bounds-checking debug build (libsta_checked.so, compiled with
-DSTA_CHECKS): every index a kernel derives from plan data is range-checked
on the device, and a violation sets the bounds bit of the device error word,
which the next synchronising call reports.  This runs representative cases
through that build -- every schedule, several corners, a batch, large RC
trees swept in global scratch, star RC, the adjoint and the path report -- in
a child process
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
}
for name, d in cases.items():
    ref = oracle.sta(d)
    for sch in (sta.SCHED_LEVEL, sta.SCHED_DATAFLOW, sta.SCHED_COOP):
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
for sch in (sta.SCHED_LEVEL, sta.SCHED_DATAFLOW, sta.SCHED_COOP):
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
