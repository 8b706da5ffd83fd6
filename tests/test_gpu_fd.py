"""Central finite differences on the GPU (the adjoint of Eq. 3 through the
network and the loss): the FP32 CUDA render and loss are evaluated at
theta +- h on 64 random parameters (32 feature entries of hit leaves, 32
network parameters) of the tiny workload, and the difference quotient is
compared with the GPU's own backward at theta. FP64 is used on the GPU only
in the loss reduction (svlf_loss's accumulator); the quotient is formed on
the host in float64.

Parameters whose perturbation would flip a kink (a hidden ReLU, the optical
thickness ReLU, or the sign of D - D* on a masked ray) are skipped, decided by
the oracle at theta +- h as in the oracle's own central-difference pin.

Tolerance per parameter: 1e-4 relative (floored at 1e-3 of the largest
gradient among the 64, as in the oracle's pin) plus the error that float32
rounding of the rendered outputs can put into the quotient: each of L(theta
+- h) is off by at most (1/N) sum over the rays the parameter reaches of
[sum_ch (2 |C - C*| + e_C) e_C + 0.1 m e_D], where e_C and e_D bound the
float32 render's colour and depth error (twice the largest error against
the FP64 oracle over those rays at theta); the quotient's error is then at
most twice that over the actual step (the float32 values of theta +- h
differ by slightly more or less than 2h)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2205_07058_b300 import inputs as I
from tests.gpu_common import net_for, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


def test_central_differences_on_the_gpu_match_the_gpu_adjoint(tiny):
    from paper_2205_07058_b300 import svlf
    rng = np.random.default_rng(5)
    params = I.make_mlp(rng, tiny.mlp, bias_std=0.3)
    feats = tiny.features
    rays = tiny.rays
    N, K, F = rays.shape[0], tiny.K, 16
    rgb_t = rng.uniform(0, 1, size=(N, 3)).astype(np.float32)
    depth_t, mask = I.analytic_depth(rays, tiny.scene)
    bg = (0.3, 0.2, 0.1)
    dims = O.layer_dims(16, 64, 2)
    tree_o = O.build_octree(tiny.scene.leaf_ijk, tiny.scene.depth)
    hits = O.trace(tree_o, rays, K)
    assert not hits.degenerate.any()
    r0 = O.render(tree_o, feats, params, dims, rays, K, bg=bg, hits=hits)
    pat0 = O.kink_pattern(r0, depth_t.astype(np.float64), mask.astype(np.float64))

    net = net_for(tiny, svlf.FP32)
    tree = svlf.Octree(torch.from_numpy(tiny.scene.leaf_ijk), tiny.scene.depth)
    r = torch.from_numpy(rays).cuda()
    tg = (torch.from_numpy(rgb_t).cuda(), torch.from_numpy(depth_t).cuda(), torch.from_numpy(mask).cuda())
    ws = svlf.alloc_workspace(net, N, K)

    def gpu_loss(f, p, grads=None):
        rgb, depth, _, _, _ = svlf.svlf_render_rays(tree, f, p, net, r, K, bg=bg, workspace=ws)
        d_rgb, d_depth = torch.empty_like(rgb), torch.empty_like(depth)
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        svlf.svlf_loss(rgb, depth, *tg, 0.1, d_rgb, d_depth, loss)
        if grads is not None:
            svlf.svlf_render_rays_backward(tree, f, p, net, r, K, bg, d_rgb, d_depth, grads[0], grads[1], ws)
        return loss.item(), rgb.cpu().numpy().astype(np.float64), depth.cpu().numpy().astype(np.float64)

    f0 = torch.from_numpy(feats).cuda()
    p0 = torch.from_numpy(params).cuda()
    g_f, g_p = torch.zeros_like(f0), torch.zeros_like(p0)
    _, rgb0, depth0 = gpu_loss(f0, p0, (g_f, g_p))
    assert svlf.svlf_get_device_status() == 0
    g_f, g_p = g_f.cpu().numpy().astype(np.float64), g_p.cpu().numpy().astype(np.float64)
    err_c = np.abs(rgb0 - r0.rgb).max(axis=1)        # per ray, float32 render vs FP64
    err_d = np.abs(depth0 - r0.depth)

    pick = np.random.default_rng(11)
    hit_leaves = np.unique(hits.rank[hits.rank >= 0])
    any_hit = hits.n > 0
    h = 1e-3
    fd, ad, bound, flips = [], [], [], 0
    while len(fd) < 64:
        if len(fd) % 2 == 0:
            which, idx = "f", (int(pick.choice(hit_leaves)), int(pick.integers(F)))
            reach = np.any(hits.rank == idx[0], axis=1)
        else:
            which, idx = "p", int(pick.integers(params.size))
            reach = any_hit
        # the float32 values at theta +- h, and the oracle's kink check there
        base = feats[idx] if which == "f" else params[idx]
        vp, vm = np.float32(base + np.float32(h)), np.float32(base - np.float32(h))
        ok = True
        for v in (vp, vm):
            f2, p2 = feats.copy(), params.copy()
            if which == "f":
                f2[idx] = v
            else:
                p2[idx] = v
            rs = O.render(tree_o, f2, p2, dims, rays, K, bg=bg, hits=hits)
            ok &= O.same_pattern(O.kink_pattern(rs, depth_t.astype(np.float64), mask.astype(np.float64)), pat0)
        if not ok:
            flips += 1
            continue
        Ls = []
        for v in (vp, vm):
            f2, p2 = f0.clone(), p0.clone()
            if which == "f":
                f2[idx] = float(v)
            else:
                p2[idx] = float(v)
            Ls.append(gpu_loss(f2, p2)[0])
        step = float(vp) - float(vm)
        fd.append((Ls[0] - Ls[1]) / step)
        ad.append(g_f[idx] if which == "f" else g_p[idx])
        eC, eD = 2.0 * err_c[reach].max(), 2.0 * err_d[reach].max()
        dl = (np.sum((2.0 * np.abs(rgb0[reach] - rgb_t[reach]) + eC) * eC) +
              0.1 * np.sum(mask[reach]) * eD) / N
        bound.append(2.0 * dl / step)
    assert svlf.svlf_get_device_status() == 0
    fd, ad, bound = np.array(fd), np.array(ad), np.array(bound)
    scale = np.maximum(np.abs(ad), 1e-3 * np.abs(ad).max())
    err = np.abs(fd - ad)
    rel = err / scale
    normwise = np.linalg.norm(fd - ad) / np.linalg.norm(ad)
    print(f"GPU central differences vs GPU adjoint over 64 parameters: max relative {rel.max():.2e}, "
          f"normwise {normwise:.2e}, largest rounding allowance / scale {(bound / scale).max():.2e}, "
          f"kink flips skipped {flips}")
    assert np.all(err <= 1e-4 * scale + bound), (rel.max(), (err - bound).max())
    assert normwise <= 1e-3, normwise
