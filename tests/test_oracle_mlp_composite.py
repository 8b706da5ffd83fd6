"""Pins for the per-sample network (ReLU hidden layers, sigmoid colour, ReLU
optical thickness: Sec. 4.5) and for compositing (Eq. 3)."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2205_07058_b300 import inputs as I


def test_bf16_rounding_matches_torch_and_ties_to_even():
    assert O.bf16_round(np.array([1.0 + 2.0 ** -8]))[0] == 1.0           # tie -> even (down)
    assert O.bf16_round(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6  # tie -> even (up)
    assert O.bf16_round(np.array([1.0 + 2.0 ** -8 + 2.0 ** -20]))[0] == 1.0 + 2.0 ** -7
    x = np.random.default_rng(0).standard_normal(100000) * 10.0
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(O.bf16_round(x), ref)


def test_network_closed_form():
    """Identity first layer and an all-ones second layer: out = sum relu(x) + b."""
    rng = np.random.default_rng(1)
    n_in = 5
    x = rng.standard_normal((50, n_in))
    layers = [(np.eye(n_in), np.zeros(n_in)), (np.ones((4, n_in)), np.array([0.5, -1.0, 2.0, 0.0]))]
    xs, pres = O.mlp_forward(x, layers)
    expect = np.maximum(x, 0).sum(axis=1)[:, None] + np.array([0.5, -1.0, 2.0, 0.0])
    np.testing.assert_allclose(pres[-1], expect, atol=1e-13)
    np.testing.assert_allclose(pres[0], x, atol=0)


def test_network_matches_elementwise_sums():
    """Compare against a scalar triple loop on a small case."""
    rng = np.random.default_rng(2)
    dims = O.layer_dims(3, 6, 2)
    params = rng.standard_normal(sum(o * i + o for o, i in dims))
    layers = O.split_params(params, dims)
    x = rng.standard_normal((7, 12))
    _, pres = O.mlp_forward(x, layers)
    for s in range(7):
        a = list(x[s])
        for li, (W, b) in enumerate(layers):
            nxt = []
            for j in range(W.shape[0]):
                acc = b[j]
                for k in range(W.shape[1]):
                    acc += W[j, k] * a[k]
                nxt.append(acc)
            a = [max(v, 0.0) for v in nxt] if li + 1 < len(layers) else nxt
        np.testing.assert_allclose(pres[-1][s], a, atol=1e-12)


@pytest.mark.parametrize("beta_c,beta_tau", [(0.3, 0.7), (-1.0, 0.05), (2.0, -0.4)])
def test_constant_network_closed_form(tiny, beta_c, beta_tau):
    """All weights zero, b_out = (bc, bc, bc, bt): a ray with n hits returns
    sigmoid(bc) (1 - e^{-n tau}) + e^{-n tau} bg, tau = max(bt, 0)."""
    tree = O.build_octree(tiny.scene.leaf_ijk, tiny.scene.depth)
    dims = O.layer_dims(16, 64, 2)
    params = np.zeros(sum(o * i + o for o, i in dims))
    params[-4:] = [beta_c, beta_c, beta_c, beta_tau]
    bg = np.array([0.2, 0.5, 0.9])
    r = O.render(tree, tiny.features, params, dims, tiny.rays, tiny.K, bg=bg)
    tau = max(beta_tau, 0.0)
    n = r.hits.n.astype(np.float64)
    sig = 1.0 / (1.0 + math.exp(-beta_c))
    expect = sig * (1.0 - np.exp(-n * tau))[:, None] + np.exp(-n * tau)[:, None] * bg[None, :]
    np.testing.assert_allclose(r.rgb, expect, atol=1e-14)
    # depth: weights e^{-(i) tau}(1 - e^{-tau}) on the segment midpoints
    D = np.zeros(len(n))
    for i in range(tiny.K):
        D += np.where(i < n, math.exp(-i * tau) * (1 - math.exp(-tau)) * 0.5
                      * (r.hits.t_in[:, i] + r.hits.t_out[:, i]), 0.0)
    np.testing.assert_allclose(r.depth, D, atol=1e-13)


def test_composite_invariants(tiny):
    tree = O.build_octree(tiny.scene.leaf_ijk, tiny.scene.depth)
    dims = O.layer_dims(16, 64, 2)
    rng = np.random.default_rng(3)
    params = I.make_mlp(rng, I.MLPShape(16, 64, 2), bias_std=0.5)
    bg = np.array([0.1, 0.7, 0.3])
    r = O.render(tree, tiny.features, params, dims, tiny.rays, tiny.K, bg=bg)
    wsum = r.w.sum(axis=1)
    np.testing.assert_allclose(wsum, 1.0 - r.T[:, -1], atol=1e-14)
    assert np.all(wsum <= 1.0 + 1e-15) and np.all(wsum >= 0)
    empty = r.hits.n == 0
    assert empty.sum() > 100
    assert np.array_equal(r.rgb[empty], np.broadcast_to(bg, (empty.sum(), 3)))
    assert np.all(r.depth[empty] == 0)
    assert np.all((r.rgb >= 0) & (r.rgb <= 1))


def test_fp16_rounding_matches_torch():
    assert O.fp16_round(np.array([1.0 + 2.0 ** -11]))[0] == 1.0          # tie -> even (down)
    assert O.fp16_round(np.array([1.0 + 3 * 2.0 ** -11]))[0] == 1.0 + 2.0 ** -9
    # float32 values (what the GPU rounds), so torch converts with one rounding too
    x = (np.random.default_rng(1).standard_normal(100000) * 10.0).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.float16).to(torch.float64).numpy()
    np.testing.assert_array_equal(O.fp16_round(x.astype(np.float64)), ref)
