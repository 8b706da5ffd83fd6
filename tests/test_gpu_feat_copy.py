"""The BF16 tensor-core network rounds every feature to bf16 (nearest even) as
it forms its input row (Sec. 4.5's network on tensor cores), so reading a bf16
copy of the float32 feature table, the one svlf_adam_step writes through its
bf16_shadow argument, gives the same network inputs: render outputs are
bit-identical, and gradients agree up to the order of the float32 atomic
additions. The training step uses this to halve its gather bytes."""
import numpy as np
import pytest
import torch

from paper_2205_07058_b300 import inputs as I
from tests.gpu_common import gpu_inputs, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


def _bf16_copy_from_adam(f):
    """The copy as the training step makes it: one Adam step with lr = 0
    leaves the float32 table unchanged and writes its bf16 rounding."""
    from paper_2205_07058_b300 import svlf
    master = f.clone()
    copy = torch.empty(f.shape, dtype=torch.bfloat16, device=f.device)
    z = torch.zeros_like(master)
    svlf.svlf_adam_step(master, torch.randn_like(master), z.clone(), z.clone(), 1, lr=0.0, bf16_shadow=copy)
    torch.cuda.synchronize()
    assert torch.equal(master, f)
    assert torch.equal(copy, f.to(torch.bfloat16))
    return copy


def _render_and_grads(tree, feats, params, net, rays, K, targets):
    from paper_2205_07058_b300 import svlf
    rgb, depth, hits, _, ws = svlf.svlf_render_rays(tree, feats, params, net, rays, K, want_hits=True)
    d_rgb, d_depth = torch.empty_like(rgb), torch.empty_like(depth)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    svlf.svlf_loss(rgb, depth, *targets, 0.1, d_rgb, d_depth, loss)
    df = torch.zeros(feats.shape, dtype=torch.float32, device="cuda")
    dp = torch.zeros_like(params)
    svlf.svlf_render_rays_backward(tree, feats, params, net, rays, K, (0.0, 0.0, 0.0), d_rgb, d_depth, df, dp, ws)
    torch.cuda.synchronize()
    assert svlf.svlf_get_device_status() == 0
    return rgb, depth, hits, loss, df, dp


def _check(tree, f, p, rays, K, shape, targets):
    from paper_2205_07058_b300 import svlf
    net32 = svlf.Network(shape.feat_dim, shape.hidden, shape.n_hidden, svlf.BF16, svlf.FEAT_F32)
    net16 = svlf.Network(shape.feat_dim, shape.hidden, shape.n_hidden, svlf.BF16, svlf.FEAT_BF16)
    a = _render_and_grads(tree, f, p, net32, rays, K, targets)
    b = _render_and_grads(tree, _bf16_copy_from_adam(f), p, net16, rays, K, targets)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])
    assert abs(a[3].item() - b[3].item()) <= 1e-12 * abs(a[3].item())  # FP64 sums, any order
    for ga, gb in zip(a[4:], b[4:]):
        e = (torch.linalg.norm(ga - gb) / torch.linalg.norm(ga)).item()
        assert e <= 1e-6, e
    return int((a[2] >= 0).sum())


def test_bf16_copy_bit_identical_tiny(tiny):
    rng = np.random.default_rng(5)
    params = I.make_mlp(rng, tiny.mlp, bias_std=0.3)
    tree, f, p, r = gpu_inputs(tiny, params=params)
    rgb_t = torch.from_numpy(rng.uniform(0, 1, size=(r.shape[0], 3)).astype(np.float32)).cuda()
    depth_t, mask = I.analytic_depth(tiny.rays, tiny.scene)
    targets = (rgb_t, torch.from_numpy(depth_t).cuda(), torch.from_numpy(mask).cuda())
    assert _check(tree, f, p, r, tiny.K, tiny.mlp, targets) > 0


def test_bf16_copy_bit_identical_depth9_many_tiles():
    """The headline network (41 -> 3x128 -> 4, K = 8) on the depth-9 scene:
    65536 training rays, hundreds of 128-sample tiles with a ragged tail."""
    from paper_2205_07058_b300 import svlf
    rng = np.random.default_rng(1002)
    scene = I.make_scene(rng, 9, 64, 32)
    shape = I.MLPShape(32, 128, 3)
    feats = I.make_features(rng, scene.n_leaves, 32)
    params = I.make_mlp(rng, shape, bias_std=0.1)
    az, el = I.random_view_angles(np.random.default_rng(7), 100)
    rays = I.training_rays(np.random.default_rng(8), 100, 800, 65536, az, el)
    tree = svlf.Octree(torch.from_numpy(scene.leaf_ijk), 9)
    f = torch.from_numpy(feats).cuda()
    p = torch.from_numpy(params).cuda()
    r = torch.from_numpy(rays).cuda()
    rgb_t = torch.from_numpy(np.random.default_rng(9).uniform(0, 1, size=(rays.shape[0], 3)).astype(np.float32))
    depth_t, mask = I.analytic_depth(rays, scene)
    targets = (rgb_t.cuda(), torch.from_numpy(depth_t).cuda(), torch.from_numpy(mask).cuda())
    n_samples = _check(tree, f, p, r, 8, shape, targets)
    assert n_samples > 100 * 128 and n_samples % 128 != 0
