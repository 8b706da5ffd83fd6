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
