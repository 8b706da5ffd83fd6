"""GPU parity of the training path (loss, compositing backward, network
backward with recomputation, feature-gradient scatter, Adam) against the FP64
oracle's adjoint, which the CPU tests pin to central finite differences."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2205_07058_b300 import inputs as I
from tests.gpu_common import gpu_inputs, net_for, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


def _targets(w, seed=9):
    rng = np.random.default_rng(seed)
    rgb_t = rng.uniform(0, 1, size=(w.rays.shape[0], 3)).astype(np.float32)
    depth_t, mask = I.analytic_depth(w.rays, w.scene)
    return rgb_t, depth_t, mask


def _gpu_grads(w, precision, params, bg, rgb_t, depth_t, mask):
    from paper_2205_07058_b300 import svlf
    tree, f, p, r = gpu_inputs(w, params=params)
    net = net_for(w, precision)
    rgb, depth, _, _, ws = svlf.svlf_render_rays(tree, f, p, net, r, w.K, bg=bg)
    d_rgb = torch.empty_like(rgb)
    d_depth = torch.empty_like(depth)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    svlf.svlf_loss(rgb, depth, torch.from_numpy(rgb_t).cuda(), torch.from_numpy(depth_t).cuda(),
                   torch.from_numpy(mask).cuda(), 0.1, d_rgb, d_depth, loss)
    df = torch.zeros_like(f)
    dp = torch.zeros_like(p)
    svlf.svlf_render_rays_backward(tree, f, p, net, r, w.K, bg, d_rgb, d_depth, df, dp, ws)
    torch.cuda.synchronize()
    assert svlf.svlf_get_device_status() == 0
    return (loss.item(), rgb.cpu().numpy(), depth.cpu().numpy(), d_rgb.cpu().numpy(),
            d_depth.cpu().numpy(), df.cpu().numpy(), dp.cpu().numpy())


def _oracle_grads(w, params, bg, rgb_t, depth_t, mask, bf16=False):
    tree = O.build_octree(w.scene.leaf_ijk, w.scene.depth)
    dims = O.layer_dims(w.mlp.feat_dim, w.mlp.hidden, w.mlp.n_hidden)
    r = O.render(tree, w.features, params, dims, w.rays, w.K, bg=bg, bf16=bf16)
    L = O.loss(r.rgb, r.depth, rgb_t, depth_t, mask)
    df, dp, dC, dD = O.backward(tree, r, params, dims, rgb_t, depth_t, mask, bg, tree.n_leaves,
                                w.mlp.feat_dim, bf16=bf16)
    return L, r, df, dp, dC, dD


def test_fp32_gradients_match_oracle_adjoint(tiny):
    from paper_2205_07058_b300 import svlf
    rng = np.random.default_rng(5)
    params = I.make_mlp(rng, tiny.mlp, bias_std=0.3)
    bg = (0.3, 0.2, 0.1)
    rgb_t, depth_t, mask = _targets(tiny)
    L, rgb, depth, d_rgb, d_depth, df, dp = _gpu_grads(tiny, svlf.FP32, params, bg, rgb_t, depth_t, mask)
    Lr, r, dfr, dpr, dC, dD = _oracle_grads(tiny, params, bg, rgb_t, depth_t, mask)
    assert r.hits.degenerate.sum() == 0  # the tiny view has no near-degenerate ray
    assert abs(L - Lr) <= 1e-6 * max(1.0, abs(Lr))
    np.testing.assert_allclose(d_rgb, dC, atol=1e-9)
    # the L1 term's sign: equal wherever |D - D*| is not within float32 noise
    far = np.abs(r.depth - depth_t) > 1e-4
    np.testing.assert_allclose(d_depth[far], dD[far], atol=1e-12)
    g = np.concatenate([df.reshape(-1), dp])
    gr = np.concatenate([dfr.reshape(-1), dpr])
    normwise = np.linalg.norm(g - gr) / np.linalg.norm(gr)
    assert normwise <= 1e-4, normwise
    # per-parameter relative error on 64 random parameters that have gradient
    nz = np.nonzero(gr != 0)[0]
    pick = np.random.default_rng(0).choice(nz, 64, replace=False)
    scale = np.maximum(np.abs(gr[pick]), 1e-3 * np.abs(gr[pick]).max())
    rel = np.abs(g[pick] - gr[pick]) / scale
    assert rel.max() <= 1e-4, rel.max()


def test_adam_matches_oracle():
    from paper_2205_07058_b300 import svlf
    rng = np.random.default_rng(2)
    n = 100003
    p = rng.standard_normal(n).astype(np.float32)
    m = np.zeros(n, np.float32)
    v = np.zeros(n, np.float32)
    tp, tm, tv = (torch.from_numpy(x.copy()).cuda() for x in (p, m, v))
    shadow = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    pr, mr, vr = p.astype(np.float64), m.astype(np.float64), v.astype(np.float64)
    for step in range(1, 4):
        g = rng.standard_normal(n).astype(np.float32)
        svlf.svlf_adam_step(tp, torch.from_numpy(g).cuda(), tm, tv, step, lr=1e-3, bf16_shadow=shadow)
        pr, mr, vr = O.adam(pr, g, mr, vr, step)
    torch.cuda.synchronize()
    np.testing.assert_allclose(tp.cpu().numpy(), pr, atol=2e-6, rtol=0)
    np.testing.assert_allclose(tm.cpu().numpy(), mr, atol=1e-6, rtol=1e-5)
    np.testing.assert_allclose(tv.cpu().numpy(), vr, atol=1e-7, rtol=1e-5)
    np.testing.assert_array_equal(shadow.float().cpu().numpy(),
                                  tp.cpu().to(torch.bfloat16).float().numpy())


def test_autograd_function_matches_direct_calls(tiny):
    from paper_2205_07058_b300 import svlf
    tree, f, p, r = gpu_inputs(tiny)
    f.requires_grad_(True)
    p.requires_grad_(True)
    net = net_for(tiny, svlf.FP32)
    rgb, depth = svlf.render(f, p, tree, net, r, tiny.K)
    (rgb.sum() + 0.5 * depth.sum()).backward()
    d_rgb = torch.ones_like(rgb)
    d_depth = torch.full_like(depth, 0.5)
    _, _, _, _, ws = svlf.svlf_render_rays(tree, f.detach(), p.detach(), net, r, tiny.K)
    df = torch.zeros_like(f)
    dp = torch.zeros_like(p)
    svlf.svlf_render_rays_backward(tree, f.detach(), p.detach(), net, r, tiny.K, (0, 0, 0), d_rgb,
                                   d_depth, df, dp, ws)
    torch.cuda.synchronize()
    # both calls accumulate per-sample contributions with float atomics, in
    # an order that differs from call to call: agreement to rounding of the
    # sums, scaled by the gradient's magnitude
    torch.testing.assert_close(f.grad, df, rtol=1e-5, atol=1e-6 * float(df.abs().max()))
    torch.testing.assert_close(p.grad, dp, rtol=1e-5, atol=1e-6 * float(dp.abs().max()))
