"""tcgen05 backward (recomputed activations, TMEM-resident dW/db, warp-aggregated
feature-gradient scatter) against the oracle's adjoint."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2205_07058_b300 import inputs as I
from tests.gpu_common import gpu_inputs, net_for, requires_gpu
from tests.test_gpu_train import _gpu_grads, _oracle_grads, _targets

pytestmark = [pytest.mark.gpu, requires_gpu]


def _rel(g, r):
    return float(np.linalg.norm(g - r) / np.linalg.norm(r))


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_tc_gradients_tiny(tiny, prec):
    from paper_2205_07058_b300 import svlf
    rng = np.random.default_rng(5)
    params = I.make_mlp(rng, tiny.mlp, bias_std=0.3)
    bg = (0.3, 0.2, 0.1)
    rgb_t, depth_t, mask = _targets(tiny)
    precision = svlf.BF16 if prec == "bf16" else svlf.FP16
    L, rgb, depth, d_rgb, d_depth, df, dp = _gpu_grads(tiny, precision, params, bg, rgb_t, depth_t, mask)
    # against the oracle that rounds activations and weights the same way
    Lr, r, dfr, dpr, _, _ = _oracle_grads(tiny, params, bg, rgb_t, depth_t, mask, bf16=prec)
    _, _, df64, dp64, _, _ = _oracle_grads(tiny, params, bg, rgb_t, depth_t, mask)
    e_feat, e_par = _rel(df, dfr), _rel(dp, dpr)
    print(f"{prec}: normwise relative error vs {prec}-emulating oracle: features {e_feat:.2e}, "
          f"network {e_par:.2e}; vs FP64 oracle: features {_rel(df, df64):.2e}, network {_rel(dp, dp64):.2e}")
    tol = 1e-2
    assert e_feat <= tol and e_par <= tol, (e_feat, e_par)
    # every layer's weights and biases individually
    dims = O.layer_dims(16, 64, 2)
    off = 0
    for o, i in dims:
        for n in (o * i, o):
            assert _rel(dp[off:off + n], dpr[off:off + n]) <= 3 * tol
            off += n


def test_tc_gradients_full_scene_subset():
    """Depth-9 scene, 41 -> 3x128 -> 4, K = 8, on 8192 training rays. Rays the
    oracle flags as near-degenerate are dropped (their hit lists may
    legitimately differ), and the depth term is masked where |D - D*| is
    within float32 noise (the L1 kink)."""
    from paper_2205_07058_b300 import svlf
    rng = np.random.default_rng(1002)
    scene = I.make_scene(rng, 9, 64, 32)
    shape = I.MLPShape(32, 128, 3)
    feats = I.make_features(rng, scene.n_leaves, 32)
    params = I.make_mlp(rng, shape, bias_std=0.1)
    az, el = I.random_view_angles(np.random.default_rng(7), 100)
    rays = I.training_rays(np.random.default_rng(8), 100, 800, 8192, az, el)
    tree = O.build_octree(scene.leaf_ijk, 9)
    keep = ~O.trace(tree, rays, 8).degenerate
    rays = rays[keep]
    w = I.Workload("sub", scene, shape, 8, feats, params, rays)
    rgb_t = np.random.default_rng(9).uniform(0, 1, size=(rays.shape[0], 3)).astype(np.float32)
    depth_t, mask = I.analytic_depth(rays, scene)
    ref = O.render(tree, feats, params, O.layer_dims(32, 128, 3), rays, 8)
    mask = np.where(np.abs(ref.depth - depth_t) < 1e-4, 0.0, mask).astype(np.float32)
    res = {}
    for prec in (svlf.FP32, svlf.FP16, svlf.BF16):
        res[prec] = _gpu_grads(w, prec, params, (0, 0, 0), rgb_t, depth_t, mask)
    Lr, r, dfr, dpr, _, _ = _oracle_grads(w, params, (0, 0, 0), rgb_t, depth_t, mask)
    _, _, dfe, dpe, _, _ = _oracle_grads(w, params, (0, 0, 0), rgb_t, depth_t, mask, bf16="bf16")
    _, _, dfh, dph, _, _ = _oracle_grads(w, params, (0, 0, 0), rgb_t, depth_t, mask, bf16="fp16")
    for name, prec, f_ref, p_ref in (("fp32", svlf.FP32, dfr, dpr), ("fp16", svlf.FP16, dfh, dph),
                                     ("bf16", svlf.BF16, dfe, dpe)):
        print(name, "features", _rel(res[prec][5], f_ref), "network", _rel(res[prec][6], p_ref),
              "| vs FP64:", _rel(res[prec][5], dfr), _rel(res[prec][6], dpr))
    assert _rel(res[svlf.FP32][5], dfr) <= 1e-4 and _rel(res[svlf.FP32][6], dpr) <= 1e-4
    # FP32 per parameter: 64 random network parameters and 64 random feature entries with gradient,
    # relative error floored at 1e-3 of the largest of each set (the tiny workload's bar)
    pick = np.random.default_rng(0)
    for g, gr in ((res[svlf.FP32][6], dpr), (res[svlf.FP32][5].reshape(-1), dfr.reshape(-1))):
        nz = np.nonzero(gr != 0)[0]
        sel = pick.choice(nz, 64, replace=False)
        scale = np.maximum(np.abs(gr[sel]), 1e-3 * np.abs(gr[sel]).max())
        rel = np.abs(g[sel] - gr[sel]) / scale
        assert rel.max() <= 1e-4, rel.max()
    assert _rel(res[svlf.FP16][5], dfh) <= 1e-2 and _rel(res[svlf.FP16][6], dph) <= 1e-2
    assert _rel(res[svlf.BF16][5], dfe) <= 1e-2 and _rel(res[svlf.BF16][6], dpe) <= 1e-2


@pytest.mark.parametrize("prec,fb", [("bf16", False), ("bf16", True), ("fp16", False)])
def test_backward_two_warpgroups_equal_one(prec, fb):
    """The tensor-core backward with a second warpgroup per tile (tuning
    mlp_bwd_warpgroups 2: each warpgroup half of every epilogue, of the input
    row and of the feature-gradient columns) against the one-warpgroup form:
    the same MMAs and roundings, so the gradients agree up to the order of
    the float32 atomic additions. Depth-9 scene, 41 -> 3x128 -> 4, 16384
    training rays (hundreds of tiles, a ragged tail)."""
    from paper_2205_07058_b300 import svlf
    rng = np.random.default_rng(1002)
    scene = I.make_scene(rng, 9, 64, 32)
    shape = I.MLPShape(32, 128, 3)
    feats = I.make_features(rng, scene.n_leaves, 32)
    params = I.make_mlp(rng, shape, bias_std=0.1)
    az, el = I.random_view_angles(np.random.default_rng(7), 100)
    rays = I.training_rays(np.random.default_rng(8), 100, 800, 16384, az, el)
    tree = svlf.Octree(torch.from_numpy(scene.leaf_ijk), 9)
    f = torch.from_numpy(feats).cuda()
    if fb:
        f = f.to(torch.bfloat16)
    p, r = torch.from_numpy(params).cuda(), torch.from_numpy(rays).cuda()
    net = svlf.Network(32, 128, 3, svlf.PRECISIONS[prec], svlf.FEAT_BF16 if fb else svlf.FEAT_F32)
    rgb_t = torch.from_numpy(np.random.default_rng(9).uniform(0, 1, size=(rays.shape[0], 3)).astype(np.float32))
    depth_t, mask = I.analytic_depth(rays, scene)
    out = {}
    try:
        for wgs in (1, 2):
            svlf.svlf_set_tuning(mlp_bwd_warpgroups=wgs)
            rgb, depth, _, _, ws = svlf.svlf_render_rays(tree, f, p, net, r, 8)
            d_rgb, d_depth = torch.empty_like(rgb), torch.empty_like(depth)
            loss = torch.zeros(1, dtype=torch.float64, device="cuda")
            svlf.svlf_loss(rgb, depth, rgb_t.cuda(), torch.from_numpy(depth_t).cuda(), torch.from_numpy(mask).cuda(),
                           0.1, d_rgb, d_depth, loss)
            df = torch.zeros((scene.n_leaves, 32), device="cuda")
            dp = torch.zeros_like(p)
            svlf.svlf_render_rays_backward(tree, f, p, net, r, 8, (0.0, 0.0, 0.0), d_rgb, d_depth, df, dp, ws)
            torch.cuda.synchronize()
            assert svlf.svlf_get_device_status() == 0
            out[wgs] = (df, dp)
    finally:
        svlf.svlf_set_tuning()
    for a, b in zip(out[1], out[2]):
        assert torch.linalg.norm(a) > 0
        e = (torch.linalg.norm(a - b) / torch.linalg.norm(a)).item()
        assert e <= 1e-6, e
    # every parameter block individually (weights and biases of each layer)
    dims = O.layer_dims(32, 128, 3)
    off = 0
    for o, i in dims:
        for n in (o * i, o):
            a, b = out[1][1][off:off + n], out[2][1][off:off + n]
            assert (torch.linalg.norm(a - b) / max(torch.linalg.norm(a).item(), 1e-30)).item() <= 1e-5
            off += n
