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


def test_adam_with_device_step_matches_host_step_and_replays_in_a_graph():
    """svlf_adam_step_device reads the step from device memory: eager calls
    after svlf_step_advance equal the host-step calls bit for bit, and a CUDA
    graph of [advance, Adam] replayed three times equals three eager steps."""
    from paper_2205_07058_b300 import svlf
    rng = np.random.default_rng(3)
    n = 50001  # vector body + scalar tail
    p0 = torch.from_numpy(rng.standard_normal(n).astype(np.float32)).cuda()
    grads = [torch.from_numpy(rng.standard_normal(n).astype(np.float32)).cuda() for _ in range(3)]
    ref = [p0.clone(), torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")]
    for t, g in enumerate(grads, 1):
        svlf.svlf_adam_step(ref[0], g, ref[1], ref[2], t, lr=1e-3)
    dev = [p0.clone(), torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")]
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    for g in grads:
        svlf.svlf_step_advance(step)
        svlf.svlf_adam_step_device(dev[0], g, dev[1], dev[2], step, lr=1e-3)
    torch.cuda.synchronize()
    assert step.item() == 3
    for a, b in zip(dev, ref):
        assert torch.equal(a, b)
    # the same three steps replayed from one captured graph
    gp = [p0.clone(), torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")]
    gstep = torch.zeros(1, dtype=torch.int64, device="cuda")
    gin = torch.empty(n, device="cuda")
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            svlf.svlf_step_advance(gstep)
            svlf.svlf_adam_step_device(gp[0], gin, gp[1], gp[2], gstep, lr=1e-3)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    assert gstep.item() == 0  # capture runs nothing
    for g in grads:
        gin.copy_(g)
        graph.replay()
    torch.cuda.synchronize()
    assert gstep.item() == 3
    for a, b in zip(gp, ref):
        assert torch.equal(a, b)


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


def test_shard_losses_and_gradients_sum_to_the_batch(tiny):
    """Data-parallel training's arithmetic on one GPU: the tiny view's rays
    split into three uneven shards, each shard's loss divided by the whole
    batch's ray count (svlf_loss_shard) and its backward accumulated into the
    same gradient buffers, give the batch's loss and gradients (up to the
    order of float32 atomic additions)."""
    from paper_2205_07058_b300 import svlf
    from paper_2205_07058_b300 import dp
    rng = np.random.default_rng(5)
    params = I.make_mlp(rng, tiny.mlp, bias_std=0.3)
    rgb_t, depth_t, mask = _targets(tiny)
    tree, f, p, r = gpu_inputs(tiny, params=params)
    net = net_for(tiny, svlf.FP32)
    N, K = r.shape[0], tiny.K
    tg = [torch.from_numpy(x).cuda() for x in (rgb_t, depth_t, mask)]

    def run(sl, gbuf, loss):
        rr = r[sl].contiguous()
        rgb, depth, _, _, ws = svlf.svlf_render_rays(tree, f, p, net, rr, K)
        d_rgb, d_depth = torch.empty_like(rgb), torch.empty_like(depth)
        svlf.svlf_loss(rgb, depth, *(t[sl].contiguous() for t in tg), 0.1, d_rgb, d_depth, loss, n_total=N)
        svlf.svlf_render_rays_backward(tree, f, p, net, rr, K, (0, 0, 0), d_rgb, d_depth, gbuf.views[0],
                                       gbuf.views[1], ws)

    full, parts = (dp.GradientBuffer([tuple(f.shape), tuple(p.shape)], device="cuda") for _ in range(2))
    L_full = torch.zeros(1, dtype=torch.float64, device="cuda")
    L_parts = torch.zeros(1, dtype=torch.float64, device="cuda")
    run(slice(0, N), full, L_full)
    for k in range(3):
        run(dp.shard(N, k, 3), parts, L_parts)
    torch.cuda.synchronize()
    assert svlf.svlf_get_device_status() == 0
    assert abs(L_parts.item() - L_full.item()) <= 1e-12 * abs(L_full.item())
    e = (torch.linalg.norm(parts.flat - full.flat) / torch.linalg.norm(full.flat)).item()
    assert e <= 1e-6, e
