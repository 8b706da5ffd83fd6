"""The FP32 plain form (SIMT kernels) over network shapes: hidden widths 32,
64 and 128 (two, four and eight output rows per thread in the register-tiled
GEMM), one to six hidden layers (the weights-resident forward and, for 4 and 5
layers of 128, the per-layer staged one), float32 and bf16 feature rows. Colours and
depth against the FP64 oracle at the FP32 bar (1e-5), gradients against the
oracle's adjoint (1e-4 normwise)."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2205_07058_b300 import inputs as I
from tests.gpu_common import requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


@pytest.fixture(scope="module")
def scene():
    rng = np.random.default_rng(881)
    sc = I.make_scene(rng, 6, 10, 3)
    rays = np.concatenate([I.pinhole_rays(math.radians(a), math.radians(e), 48, 48)
                           for a, e in ((35, 20), (200, -15))])
    # rays the oracle flags as near-degenerate are dropped: their hit lists may differ
    keep = ~O.trace(O.build_octree(sc.leaf_ijk, sc.depth), rays, 4).degenerate
    return sc, rays[keep]


@pytest.mark.parametrize("fb", [False, True])
# 4 x 128 and 5 x 128: the network does not fit in shared memory beside its tile,
# so the forward stages each layer's W^T instead of holding the whole network;
# the FP32 backward keeps every layer's activations (68-float rows) in shared
# memory, without staged weights for 4 x 128, and refuses 5 x 128
@pytest.mark.parametrize("F,H,nh", [(8, 32, 1), (16, 32, 2), (16, 64, 2), (32, 128, 3), (24, 64, 3), (16, 64, 6),
                                    (32, 128, 4), (32, 128, 5), (16, 256, 1)])
def test_fp32_shapes_render_and_gradients(scene, F, H, nh, fb):
    from paper_2205_07058_b300 import svlf
    sc, rays = scene
    rng = np.random.default_rng(F * 100 + H + nh)
    feats = I.make_features(rng, sc.n_leaves, F)
    if fb:  # bf16 storage: the oracle takes the stored values
        feats = torch.from_numpy(feats).to(torch.bfloat16).float().numpy()
    params = I.make_mlp(rng, I.MLPShape(F, H, nh), bias_std=0.3)
    params[-1] += 1.0  # the optical-thickness output's bias: tau > 0, so every shape has a gradient
    bg = (0.2, 0.1, 0.3)
    K = 4
    tree = svlf.Octree(torch.from_numpy(sc.leaf_ijk), sc.depth)
    f = torch.from_numpy(feats).cuda()
    if fb:
        f = f.to(torch.bfloat16)
    p, r = torch.from_numpy(params).cuda(), torch.from_numpy(rays).cuda()
    net = svlf.Network(F, H, nh, svlf.FP32, svlf.FEAT_BF16 if fb else svlf.FEAT_F32)
    rgb, depth, _, _, ws = svlf.svlf_render_rays(tree, f, p, net, r, K, bg=bg)
    rgb_t = rng.uniform(0, 1, size=(rays.shape[0], 3)).astype(np.float32)
    depth_t, mask = I.analytic_depth(rays, sc)
    d_rgb, d_depth = torch.empty_like(rgb), torch.empty_like(depth)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    svlf.svlf_loss(rgb, depth, torch.from_numpy(rgb_t).cuda(), torch.from_numpy(depth_t).cuda(),
                   torch.from_numpy(mask).cuda(), 0.1, d_rgb, d_depth, loss)
    df = torch.zeros((sc.n_leaves, F), device="cuda")
    dp = torch.zeros_like(p)
    in0p = (F + 9 + 3) // 4 * 4
    backward = H <= 128 and 4 * 68 * (in0p + nh * H + 2 * max(in0p, H)) <= 220 * 1024
    if backward:
        svlf.svlf_render_rays_backward(tree, f, p, net, r, K, bg, d_rgb, d_depth, df, dp, ws)
    else:
        with pytest.raises(svlf.SvlfError) as e:
            svlf.svlf_render_rays_backward(tree, f, p, net, r, K, bg, d_rgb, d_depth, df, dp, ws)
        assert e.value.code == svlf.SVLF_ERR_UNSUPPORTED
    torch.cuda.synchronize()
    assert svlf.svlf_get_device_status() == 0

    otree = O.build_octree(sc.leaf_ijk, sc.depth)
    dims = O.layer_dims(F, H, nh)
    ref = O.render(otree, feats, params, dims, rays, K, bg=bg)
    assert not ref.hits.degenerate.any() and (ref.hits.n > 0).sum() > 200
    err = np.abs(rgb.cpu().numpy() - ref.rgb).max()
    derr = (np.abs(depth.cpu().numpy() - ref.depth) / (1 + ref.depth)).max()
    assert err <= 1e-5 and derr <= 1e-5, (err, derr)
    if not backward:
        return
    dfr, dpr, _, _ = O.backward(otree, ref, params, dims, rgb_t, depth_t.astype(np.float64),
                                mask.astype(np.float64), bg, otree.n_leaves, F)
    g = np.concatenate([df.cpu().numpy().reshape(-1), dp.cpu().numpy()])
    gr = np.concatenate([dfr.reshape(-1), dpr])
    e = np.linalg.norm(g - gr) / np.linalg.norm(gr)
    assert e <= 1e-4, e


def test_fp32_forward_refuses_what_does_not_fit(scene):
    """Two hidden layers of 256: neither the whole network nor two activation
    tiles fit in shared memory; the call is refused before any launch."""
    from paper_2205_07058_b300 import svlf
    sc, rays = scene
    rng = np.random.default_rng(3)
    params = I.make_mlp(rng, I.MLPShape(16, 256, 2), bias_std=0.3)
    tree = svlf.Octree(torch.from_numpy(sc.leaf_ijk), sc.depth)
    f = torch.from_numpy(I.make_features(rng, sc.n_leaves, 16)).cuda()
    net = svlf.Network(16, 256, 2, svlf.FP32)
    with pytest.raises(svlf.SvlfError) as e:
        svlf.svlf_render_rays(tree, f, torch.from_numpy(params).cuda(), net, torch.from_numpy(rays).cuda(), 4)
    assert e.value.code == svlf.SVLF_ERR_UNSUPPORTED
    torch.cuda.synchronize()
    assert svlf.svlf_get_device_status() == 0
