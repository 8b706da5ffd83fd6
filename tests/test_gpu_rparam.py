"""The network input under the other reading of Sec. 4.1's "voxel origin"
(svlf_render_opts.rparam_mode = SVLF_RPARAM_AABB: the ray's entry and exit
points of the voxel box in voxel-local coordinates) against the oracle's
aabb reading: colours and depth (FP32 and the 16-bit tensor-core paths),
gradients (FP32), origins inside the cube (entry clipped at t = 0), and the
two readings giving different images."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2205_07058_b300 import inputs as I
from tests.gpu_common import gpu_inputs, net_for, random_rays, requires_gpu
from tests.test_gpu_train import _targets

pytestmark = [pytest.mark.gpu, requires_gpu]


def _rays(tiny):
    extra = random_rays(np.random.default_rng(21), 4096, inside_frac=0.3)
    return np.concatenate([tiny.rays, extra])


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_aabb_reading_render_matches_oracle(tiny, prec):
    from paper_2205_07058_b300 import svlf
    rays = _rays(tiny)
    rng = np.random.default_rng(4)
    params = I.make_mlp(rng, tiny.mlp, bias_std=0.3)
    tree, f, p, r = gpu_inputs(tiny, params=params, rays=rays)
    net = net_for(tiny, svlf.PRECISIONS[prec])
    bg = (0.2, 0.3, 0.4)
    rgb, depth, _, _, _ = svlf.svlf_render_rays(tree, f, p, net, r, tiny.K, bg=bg, rparam=svlf.RPARAM_AABB)
    rgb_s, _, _, _, _ = svlf.svlf_render_rays(tree, f, p, net, r, tiny.K, bg=bg)
    torch.cuda.synchronize()
    assert svlf.svlf_get_device_status() == 0
    tree_o = O.build_octree(tiny.scene.leaf_ijk, tiny.scene.depth)
    dims = O.layer_dims(16, 64, 2)
    ref = O.render(tree_o, tiny.features, params, dims, rays, tiny.K, bg=bg, rparam="aabb",
                   bf16=False if prec == "fp32" else prec)
    ok = ~ref.hits.degenerate
    g, gd = rgb.cpu().numpy(), depth.cpu().numpy()
    tol = 1e-5 if prec == "fp32" else 2e-3
    assert np.abs(g[ok] - ref.rgb[ok]).max() <= tol
    assert np.all(np.abs(gd[ok] - ref.depth[ok]) <= tol * (1 + ref.depth[ok]))
    # rays starting inside occupied voxels were covered, and the readings differ
    assert np.any(ref.hits.t_in[ok][:, 0] == 0.0)
    assert np.abs(g - rgb_s.cpu().numpy()).max() > 1e-3


def test_aabb_reading_gradients_match_oracle_adjoint(tiny):
    """FP32 gradients under the aabb reading against the oracle's adjoint
    (normwise 1e-4, the FP32 bar); the depth term is masked on rays where
    |D - D*| is within rounding noise of the L1 kink, on both sides."""
    from paper_2205_07058_b300 import svlf
    rng = np.random.default_rng(5)
    params = I.make_mlp(rng, tiny.mlp, bias_std=0.3)
    bg = (0.3, 0.2, 0.1)
    rgb_t, depth_t, mask = _targets(tiny)
    tree_o = O.build_octree(tiny.scene.leaf_ijk, tiny.scene.depth)
    dims = O.layer_dims(16, 64, 2)
    ref = O.render(tree_o, tiny.features, params, dims, tiny.rays, tiny.K, bg=bg, rparam="aabb")
    mask = np.where(np.abs(ref.depth - depth_t) > 1e-4, mask, 0.0).astype(np.float32)
    dfr, dpr, _, _ = O.backward(tree_o, ref, params, dims, rgb_t.astype(np.float64), depth_t.astype(np.float64),
                                mask.astype(np.float64), bg, tree_o.n_leaves, 16)
    tree, f, p, r = gpu_inputs(tiny, params=params)
    net = net_for(tiny, svlf.FP32)
    A = svlf.RPARAM_AABB
    rgb, depth, _, _, ws = svlf.svlf_render_rays(tree, f, p, net, r, tiny.K, bg=bg, rparam=A)
    d_rgb, d_depth = torch.empty_like(rgb), torch.empty_like(depth)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    svlf.svlf_loss(rgb, depth, torch.from_numpy(rgb_t).cuda(), torch.from_numpy(depth_t).cuda(),
                   torch.from_numpy(mask).cuda(), 0.1, d_rgb, d_depth, loss)
    df, dp = torch.zeros_like(f), torch.zeros_like(p)
    svlf.svlf_render_rays_backward(tree, f, p, net, r, tiny.K, bg, d_rgb, d_depth, df, dp, ws, rparam=A)
    torch.cuda.synchronize()
    assert svlf.svlf_get_device_status() == 0
    g = np.concatenate([df.cpu().numpy().reshape(-1), dp.cpu().numpy()])
    gr = np.concatenate([dfr.reshape(-1), dpr])
    assert np.linalg.norm(g - gr) / np.linalg.norm(gr) <= 1e-4


def test_aabb_reading_batched_and_static_match_single_call(tiny):
    from paper_2205_07058_b300 import svlf
    tree, f, p, r = gpu_inputs(tiny)
    net = net_for(tiny, svlf.BF16)
    A = svlf.RPARAM_AABB
    rgb, depth, _, _, _ = svlf.svlf_render_rays(tree, f, p, net, r, tiny.K, rparam=A)
    b = svlf.BatchScene(tree, f, p, r)
    svlf.svlf_render_rays_batched([b], net, tiny.K, rparam=A)
    rs, ds = svlf.svlf_render_rays_static(tree, f, p, net, r, tiny.K, rparam=A)
    torch.cuda.synchronize()
    assert torch.equal(b.rgb, rgb) and torch.equal(b.depth, depth)
    assert torch.equal(rs, rgb) and torch.equal(ds, depth)


def test_rparam_mode_checked(tiny):
    from paper_2205_07058_b300 import svlf
    tree, f, p, r = gpu_inputs(tiny)
    with pytest.raises(svlf.SvlfError) as e:
        svlf.svlf_render_rays(tree, f, p, net_for(tiny, svlf.FP32), r, tiny.K, rparam=7)
    assert e.value.code == svlf.SVLF_ERR_ARG
