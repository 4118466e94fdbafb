"""The allocation-free WNS/TNS entry point (sta_reduce_slack_noalloc).

Callers that cannot call cudaMalloc -- their device memory is already owned
by another allocator, or they cannot afford its implicit synchronisation --
use this variant of the FP64 endpoint-slack reduction; its partial sums sit
in a fixed device array inside the library.  This test feeds it the endpoint
slacks of a timing pass and checks it twice in a row against what the
regular entry point (sta_report_slack) reports for the same pass.  The file
is named to be collected last."""
import numpy as np
import pytest

from paper_2511_11660_b300 import sta, synth

pytestmark = pytest.mark.gpu

FIELDS = ("wns_setup", "tns_setup", "wns_hold", "tns_hold", "worst_setup", "worst_hold", "n_viol_setup",
          "n_viol_hold")


@pytest.mark.parametrize("n_cells,corners", [(2000, 1), (60000, 4)])
def test_noalloc_reduction_matches_report(n_cells, corners):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    kw = {}
    if corners > 1:
        ls, rs = synth.lut_corners()
        kw = dict(n_corners=corners, lut_scale=ls, rc_scale=rs)
    d = synth.make_design(n_cells, 30, seed=5, period_ns=2.0, **kw)
    ctx = sta.Context(d)
    ctx.update_timing()
    want = ctx.report_slack()
    setup, hold, _, _ = ctx.get_endpoint_slack(device=True)
    for _ in range(2):
        out = torch.full((corners, 8), float("nan"), dtype=torch.float64, device="cuda")
        sta.reduce_slack_noalloc(setup, hold, out)
        got = out.cpu().numpy()
        for k in range(corners):
            for i, f in enumerate(FIELDS):
                assert got[k, i] == pytest.approx(want[k][f], rel=1e-12, abs=1e-12), (k, f)
    ctx.close()


def test_noalloc_rejects_oversize():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    lib = sta.load()
    n = 8193 * 4096   # 8193 chunks of 4096 endpoints: one past the fixed scratch
    # buffers of the claimed size, so that a regression of the host-side check
    # reads only memory it owns (a wrong status, never an out-of-range read)
    x = torch.zeros(n, dtype=torch.float32, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = lib.sta_reduce_slack_noalloc(x.data_ptr(), x.data_ptr(), n, 1, out.data_ptr(), None)
    assert st == sta.EINVAL
    del x


def test_noalloc_binding_checks_inputs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    s = torch.zeros((10, 2), dtype=torch.float32, device="cuda")
    out = torch.zeros((2, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        sta.reduce_slack_noalloc(s.double(), s, out)          # wrong dtype
    with pytest.raises(ValueError):
        sta.reduce_slack_noalloc(s, s[:5], out)               # shapes differ
    with pytest.raises(ValueError):
        sta.reduce_slack_noalloc(s, s, out[:1])               # out too short
    with pytest.raises(ValueError):
        sta.reduce_slack_noalloc(s.t(), s.t(), out)           # not contiguous
    with pytest.raises(ValueError):
        sta.reduce_slack_noalloc(s.cpu(), s, out)             # host tensor
