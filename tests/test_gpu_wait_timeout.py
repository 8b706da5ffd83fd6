"""Failure detection without a GPU fault: the bounded mbarrier wait every
kernel uses gives up after its limit when nothing completes the phase, latches
SVLF_DEV_WAIT_TIMEOUT in the device status (cleared on read) and returns; the
context stays usable afterwards."""
import numpy as np
import pytest
import torch

from tests.gpu_common import gpu_inputs, net_for, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


def test_wait_gives_up_reports_and_context_survives(tiny):
    from paper_2205_07058_b300 import svlf
    svlf.svlf_get_device_status()  # start from a clear status
    limit = 2_000_000  # SM clocks, about a millisecond
    ok, clocks = svlf.svlf_selftest_wait(limit, arrive=False)
    assert not ok and clocks >= limit
    assert svlf.svlf_get_device_status() == svlf.SVLF_DEV_WAIT_TIMEOUT
    assert svlf.svlf_get_device_status() == 0  # cleared on read
    # the control: the phase completes, the wait returns at once and nothing is latched
    ok, clocks = svlf.svlf_selftest_wait(limit, arrive=True)
    assert ok and clocks < limit
    assert svlf.svlf_get_device_status() == 0
    # the context still renders
    tree, f, p, r = gpu_inputs(tiny)
    rgb, depth, _, _, _ = svlf.svlf_render_rays(tree, f, p, net_for(tiny, svlf.FP32), r, 4)
    torch.cuda.synchronize()
    assert torch.isfinite(rgb).all() and torch.isfinite(depth).all()
    assert svlf.svlf_get_device_status() == 0


def test_wait_arguments_checked():
    from paper_2205_07058_b300 import svlf
    with pytest.raises(svlf.SvlfError):
        svlf.svlf_selftest_wait(0)


def test_step_limit_latches_truncates_and_context_survives(tiny):
    """The traversal's step bound (svlf_set_step_limit) set far below what the
    tiny view's rays need: every ray stops after two walk steps with the hits
    it found so far (a prefix of its full hit list), SVLF_DEV_STEP_LIMIT is
    latched and read back through the stream-ordered status call, the kernel
    returns, and with the default bound restored the next render is
    bit-identical to the one before."""
    from paper_2205_07058_b300 import svlf
    svlf.svlf_get_device_status()
    tree, f, p, r = gpu_inputs(tiny)
    net = net_for(tiny, svlf.FP32)
    K = tiny.K
    ref_rgb, ref_depth, ref_hits, _, _ = svlf.svlf_render_rays(tree, f, p, net, r, K, want_hits=True)
    assert svlf.svlf_get_device_status() == 0
    saved = svlf.svlf_get_tuning()
    try:
        svlf.svlf_set_tuning(**dict(saved, trace_budget=1))
        svlf.svlf_set_step_limit(1)
        _, _, hits, _, _ = svlf.svlf_render_rays(tree, f, p, net, r, K, want_hits=True)
        assert svlf.svlf_get_device_status(torch.cuda.current_stream()) & svlf.SVLF_DEV_STEP_LIMIT
    finally:
        svlf.svlf_set_step_limit(0)
        svlf.svlf_set_tuning(**saved)
    h, rh = hits.cpu().numpy(), ref_hits.cpu().numpy()
    n, rn = (h >= 0).sum(axis=1), (rh >= 0).sum(axis=1)
    assert np.all(n <= rn) and np.any(n < rn)
    for i in np.nonzero(n)[0]:
        assert np.array_equal(h[i, :n[i]], rh[i, :n[i]])
    assert np.all(h[np.arange(K)[None, :] >= n[:, None]] == -1)
    rgb, depth, hits2, _, _ = svlf.svlf_render_rays(tree, f, p, net, r, K, want_hits=True)
    assert svlf.svlf_get_device_status() == 0
    assert torch.equal(hits2, ref_hits) and torch.equal(rgb, ref_rgb) and torch.equal(depth, ref_depth)


def test_step_limit_arguments_checked():
    from paper_2205_07058_b300 import svlf
    with pytest.raises(svlf.SvlfError):
        svlf.svlf_set_step_limit(-1)
