"""svlf_render_rays_static: rendering for callers that cannot allocate device
memory (fixed-budget hosts, frame loops that must not call cudaMalloc). It
must give the same image as svlf_render_rays with a caller workspace, on two
calls in a row (the shared scratch array keeps the previous call's contents),
and must refuse a call larger than its fixed scratch."""
import numpy as np
import pytest
import torch

from paper_2205_07058_b300 import inputs as I
from tests.gpu_common import gpu_inputs, net_for, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]

COLOUR_TOL = 1e-5  # the FP32 colour tolerance of the render parity tests


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_static_scratch_render_matches_workspace_render(prec):
    from paper_2205_07058_b300 import svlf
    w = I.tiny_workload()
    tree, f, p, r = gpu_inputs(w)
    net = net_for(w, svlf.PRECISIONS[prec])
    bg = (0.2, 0.4, 0.6)
    ref_rgb, ref_depth, _, _, _ = svlf.svlf_render_rays(tree, f, p, net, r, w.K, bg=bg)
    # a different workload in between, so the second call starts from stale scratch
    r2 = r.flip(0).contiguous()
    for call in range(2):
        rgb, depth = svlf.svlf_render_rays_static(tree, f, p, net, r, w.K, bg=bg)
        torch.cuda.synchronize()
        assert torch.max(torch.abs(rgb - ref_rgb)).item() <= COLOUR_TOL, call
        assert torch.max(torch.abs(depth - ref_depth) / (1 + ref_depth)).item() <= COLOUR_TOL, call
        svlf.svlf_render_rays_static(tree, f, p, net, r2, w.K, bg=bg)
    assert svlf.svlf_get_device_status() == 0


def test_static_scratch_rejects_oversized_call():
    from paper_2205_07058_b300 import svlf
    w = I.tiny_workload()
    tree, f, p, r = gpu_inputs(w)
    net = net_for(w, svlf.FP32)
    big = r.repeat(64, 1)  # 262144 rays x K=4 needs more than the fixed scratch
    with pytest.raises(svlf.SvlfError) as e:
        svlf.svlf_render_rays_static(tree, f, p, net, big, w.K)
    assert e.value.code == svlf.SVLF_ERR_WORKSPACE
