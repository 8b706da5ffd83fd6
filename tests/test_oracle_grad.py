"""Pins for the oracle's adjoint (hand-derived from Eq. 3 and the loss) and
for Adam (Kingma & Ba, as cited in Sec. 4.5)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2205_07058_b300 import inputs as I


def _setup(tiny, seed=5):
    tree = O.build_octree(tiny.scene.leaf_ijk, tiny.scene.depth)
    dims = O.layer_dims(16, 64, 2)
    rng = np.random.default_rng(seed)
    params = I.make_mlp(rng, I.MLPShape(16, 64, 2), bias_std=0.3).astype(np.float64)
    feats = tiny.features.astype(np.float64)
    rays = tiny.rays
    rgb_t = rng.uniform(0, 1, size=(rays.shape[0], 3))
    depth_t, mask = I.analytic_depth(rays, tiny.scene)
    bg = np.array([0.3, 0.2, 0.1])
    hits = O.trace(tree, rays, tiny.K)
    return tree, dims, params, feats, rays, rgb_t, depth_t.astype(np.float64), mask.astype(np.float64), bg, hits


def _loss(tree, dims, params, feats, rays, rgb_t, depth_t, mask, bg, hits, K):
    r = O.render(tree, feats, params, dims, rays, K, bg=bg, hits=hits)
    return O.loss(r.rgb, r.depth, rgb_t, depth_t, mask), r


def test_adjoint_matches_central_differences(tiny):
    tree, dims, params, feats, rays, rgb_t, depth_t, mask, bg, hits = _setup(tiny)
    K = tiny.K
    L0, r0 = _loss(tree, dims, params, feats, rays, rgb_t, depth_t, mask, bg, hits, K)
    dfeat, dparams, _, _ = O.backward(tree, r0, params, dims, rgb_t, depth_t, mask, bg,
                                      tree.n_leaves, 16)
    pat0 = O.kink_pattern(r0, depth_t, mask)
    rng = np.random.default_rng(11)
    hit_leaves = np.unique(hits.rank[hits.rank >= 0])
    h = 1e-3
    fd, ad, flips = [], [], 0
    while len(fd) < 64:
        if len(fd) % 2 == 0:
            leaf = rng.choice(hit_leaves)
            col = rng.integers(16)
            which, idx = "f", (leaf, col)
        else:
            which, idx = "p", rng.integers(params.size)
        vals = []
        ok = True
        for s in (+1, -1):
            p2, f2 = params.copy(), feats.copy()
            if which == "f":
                f2[idx] += s * h
            else:
                p2[idx] += s * h
            Ls, rs = _loss(tree, dims, p2, f2, rays, rgb_t, depth_t, mask, bg, hits, K)
            if not O.same_pattern(O.kink_pattern(rs, depth_t, mask), pat0):
                ok = False
            vals.append(Ls)
        if not ok:
            flips += 1
            continue
        fd.append((vals[0] - vals[1]) / (2 * h))
        ad.append(dfeat[idx] if which == "f" else dparams[idx])
    fd, ad = np.array(fd), np.array(ad)
    scale = np.maximum(np.abs(fd), 1e-3 * np.abs(fd).max())
    rel = np.abs(ad - fd) / scale
    assert rel.max() <= 1e-4, (rel.max(), flips)
    assert np.linalg.norm(ad - fd) / np.linalg.norm(fd) <= 1e-5


def test_gradient_of_depth_term_only_reaches_masked_rays(tiny):
    tree, dims, params, feats, rays, rgb_t, depth_t, mask, bg, hits = _setup(tiny)
    L0, r0 = _loss(tree, dims, params, feats, rays, rgb_t, depth_t, mask, bg, hits, tiny.K)
    _, _, dC, dD = O.backward(tree, r0, params, dims, rgb_t, depth_t, mask, bg, tree.n_leaves, 16)
    assert np.all(dD[mask == 0] == 0)
    np.testing.assert_allclose(np.abs(dD[mask > 0]), 0.1 / rays.shape[0])
    np.testing.assert_allclose(dC, 2 * (r0.rgb - rgb_t) / rays.shape[0])


def test_adam_closed_form_first_step():
    """With bias correction, the first step moves each parameter by
    -lr * g / (|g| + eps): -lr * sign(g) up to eps."""
    rng = np.random.default_rng(0)
    p = rng.standard_normal(1000)
    g = rng.standard_normal(1000)
    p1, m1, v1 = O.adam(p, g, np.zeros(1000), np.zeros(1000), 1, lr=1e-3)
    np.testing.assert_allclose(p1 - p, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m1, 0.1 * g)
    np.testing.assert_allclose(v1, 0.001 * g * g)


def test_adam_matches_torch_optimizer():
    rng = np.random.default_rng(1)
    p = rng.standard_normal(500)
    tp = torch.tensor(p.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    m = np.zeros(500)
    v = np.zeros(500)
    for step in range(1, 6):
        g = rng.standard_normal(500)
        tp.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        p, m, v = O.adam(p, g, m, v, step)
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=0, atol=1e-12)
