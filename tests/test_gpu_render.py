"""GPU parity of the render path against the FP64 oracle (tiny workload in
full; random rays including ones that start inside the cube)."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2205_07058_b300 import inputs as I
from tests.gpu_common import compare_hits, gpu_inputs, net_for, random_rays, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]

COLOUR_TOL_FP32 = 1e-5


def _oracle(w, rays=None, K=None, bg=(0, 0, 0), params=None, bf16=False):
    tree = O.build_octree(w.scene.leaf_ijk, w.scene.depth)
    dims = O.layer_dims(w.mlp.feat_dim, w.mlp.hidden, w.mlp.n_hidden)
    return tree, O.render(tree, w.features, w.params if params is None else params, dims,
                          w.rays if rays is None else rays, K or w.K, bg=bg, bf16=bf16)


def test_octree_leaves_in_rank_order(tiny):
    from paper_2205_07058_b300 import svlf
    tree, *_ = gpu_inputs(tiny)
    oracle_tree = O.build_octree(tiny.scene.leaf_ijk, tiny.scene.depth)
    assert tree.n_leaves == oracle_tree.n_leaves
    assert np.array_equal(tree.leaf_ijk().cpu().numpy(), oracle_tree.leaf_ijk())
    info = tree.info()
    assert info["n_leaves"] == tree.n_leaves and info["n_bricks"] > 0


def test_duplicate_and_out_of_range_leaves():
    from paper_2205_07058_b300 import svlf
    ijk = torch.tensor([[1, 2, 3], [1, 2, 3], [0, 0, 0]], dtype=torch.int32)
    t = svlf.Octree(ijk, 3)
    assert t.n_leaves == 2
    with pytest.raises(svlf.SvlfError) as e:
        svlf.Octree(torch.tensor([[8, 0, 0]], dtype=torch.int32), 3)
    assert e.value.code == svlf.SVLF_ERR_ARG


@pytest.mark.parametrize("K", [1, 3, 4, 32])
def test_hit_lists_bit_exact_tiny(tiny, K):
    from paper_2205_07058_b300 import svlf
    rng = np.random.default_rng(3)
    rays = np.concatenate([tiny.rays, random_rays(rng, 20000)])
    tree, f, p, r = gpu_inputs(tiny, rays=rays)
    net = net_for(tiny, svlf.FP32)
    _, _, hits, tio, _ = svlf.svlf_render_rays(tree, f, p, net, r, K, want_hits=True)
    torch.cuda.synchronize()
    oh = O.trace(O.build_octree(tiny.scene.leaf_ijk, tiny.scene.depth), rays, K)
    n_ok, n_deg, mism = compare_hits(oh, hits.cpu().numpy(), tio.cpu().numpy())
    assert n_ok > 19000
    assert (oh.n > 0).sum() > 2000
    assert mism <= n_deg
    assert svlf.svlf_get_device_status() == 0


@pytest.mark.parametrize("refill", [1, 16])
def test_hit_lists_independent_of_lane_refill(tiny, refill):
    """Lanes refilled across chunk boundaries give the same hit lists."""
    from paper_2205_07058_b300 import svlf
    rng = np.random.default_rng(4)
    rays = np.concatenate([tiny.rays, random_rays(rng, 20000)])
    tree, f, p, r = gpu_inputs(tiny, rays=rays)
    net = net_for(tiny, svlf.FP32)
    try:
        svlf.svlf_set_tuning(trace_refill=32)
        _, _, h0, t0, _ = svlf.svlf_render_rays(tree, f, p, net, r, 8, want_hits=True)
        svlf.svlf_set_tuning(trace_refill=refill, trace_budget=2)
        _, _, h1, t1, _ = svlf.svlf_render_rays(tree, f, p, net, r, 8, want_hits=True)
        torch.cuda.synchronize()
    finally:
        svlf.svlf_set_tuning()
    assert torch.equal(h0, h1) and torch.equal(t0, t1)
    assert svlf.svlf_get_device_status() == 0


def test_render_fp32_matches_oracle_tiny(tiny):
    from paper_2205_07058_b300 import svlf
    rng = np.random.default_rng(4)
    params = I.make_mlp(rng, tiny.mlp, bias_std=0.5)
    bg = (0.25, 0.5, 0.75)
    tree, f, p, r = gpu_inputs(tiny, params=params)
    net = net_for(tiny, svlf.FP32)
    rgb, depth, hits, _, _ = svlf.svlf_render_rays(tree, f, p, net, r, tiny.K, bg=bg, want_hits=True)
    torch.cuda.synchronize()
    _, ref = _oracle(tiny, params=params, bg=bg)
    ok = ~ref.hits.degenerate
    rgb, depth = rgb.cpu().numpy(), depth.cpu().numpy()
    err = np.abs(rgb[ok] - ref.rgb[ok]).max()
    assert err <= COLOUR_TOL_FP32, err
    derr = np.abs(depth[ok] - ref.depth[ok]) / (1 + ref.depth[ok])
    assert derr.max() <= 1e-5, derr.max()
    # invariants: empty rays return exactly bg, depth 0
    empty = ref.hits.n == 0
    assert empty.sum() > 100
    assert np.array_equal(rgb[empty], np.broadcast_to(np.float32(bg), (empty.sum(), 3)))
    assert np.all(depth[empty] == 0)


def test_render_fp32_constant_network_closed_form(tiny):
    """Zero weights, b_out = (bc, bc, bc, bt): C = sigmoid(bc)(1 - e^{-n tau}) + e^{-n tau} bg."""
    from paper_2205_07058_b300 import svlf
    params = np.zeros_like(tiny.params)
    params[-4:] = [0.3, 0.3, 0.3, 0.7]
    bg = (0.1, 0.2, 0.3)
    tree, f, p, r = gpu_inputs(tiny, params=params)
    rgb, depth, hits, _, _ = svlf.svlf_render_rays(tree, f, p, net_for(tiny, svlf.FP32), r, tiny.K,
                                                   bg=bg, want_hits=True)
    n = (hits.cpu().numpy() >= 0).sum(axis=1).astype(np.float64)
    sig = 1 / (1 + math.exp(-0.3))
    expect = sig * (1 - np.exp(-0.7 * n))[:, None] + np.exp(-0.7 * n)[:, None] * np.array(bg)
    np.testing.assert_allclose(rgb.cpu().numpy(), expect, atol=2e-6)


def test_empty_octree_and_zero_rays(tiny):
    from paper_2205_07058_b300 import svlf
    tree = svlf.Octree(torch.zeros((0, 3), dtype=torch.int32), 6)
    assert tree.n_leaves == 0
    r = torch.from_numpy(tiny.rays).cuda()
    p = torch.from_numpy(tiny.params).cuda()
    f = torch.zeros((1, 16), device="cuda")
    rgb, depth, hits, _, _ = svlf.svlf_render_rays(tree, f, p, net_for(tiny, svlf.FP32), r, 4,
                                                   bg=(0.5, 0.5, 0.5), want_hits=True)
    assert torch.all(rgb == 0.5) and torch.all(depth == 0) and torch.all(hits == -1)
    t2, f2, p2, r2 = gpu_inputs(tiny)
    rgb, depth, _, _, _ = svlf.svlf_render_rays(t2, f2, p2, net_for(tiny, svlf.FP32), r2[:0], 4)
    assert rgb.shape == (0, 3)


def test_bad_arguments_are_reported(tiny):
    from paper_2205_07058_b300 import svlf
    tree, f, p, r = gpu_inputs(tiny)
    ws32 = svlf.alloc_workspace(net_for(tiny, svlf.FP32), r.shape[0], 32)
    with pytest.raises(svlf.SvlfError) as e:
        svlf.svlf_render_rays(tree, f, p, net_for(tiny, svlf.FP32), r, 33, workspace=ws32)
    assert e.value.code == svlf.SVLF_ERR_UNSUPPORTED
    ws = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(svlf.SvlfError) as e:  # workspace too small
        svlf.svlf_render_rays(tree, f, p, net_for(tiny, svlf.FP32), r, 4, workspace=ws)
    assert e.value.code == svlf.SVLF_ERR_WORKSPACE
    with pytest.raises(ValueError):  # feature table narrower than the descriptor's feat_dim
        svlf.svlf_render_rays(tree, f[:, :8].contiguous(), p, net_for(tiny, svlf.FP32), r, 4)
