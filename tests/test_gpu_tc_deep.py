"""Tensor-core backward of the four-hidden-layer network (41 -> 4x128 -> 4,
K = 16, bf16-representable features): its weights and activations do not fit in
shared memory together, so the hidden layers' weights are streamed through
two slots. Gradients against the oracle that rounds operands the same way."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2205_07058_b300 import inputs as I
from tests.gpu_common import requires_gpu
from tests.test_gpu_train import _gpu_grads, _oracle_grads

pytestmark = [pytest.mark.gpu, requires_gpu]


def _rel(g, r):
    return float(np.linalg.norm(g - r) / np.linalg.norm(r))


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_tc_gradients_four_hidden_layers(prec):
    from paper_2205_07058_b300 import svlf
    rng = np.random.default_rng(1005)
    scene = I.make_scene(rng, 8, 24, 12)
    shape = I.MLPShape(32, 128, 4)
    feats = torch.from_numpy(I.make_features(rng, scene.n_leaves, 32)).to(torch.bfloat16).float().numpy()
    params = I.make_mlp(rng, shape, bias_std=0.1)
    az, el = I.random_view_angles(np.random.default_rng(7), 100)
    rays = I.training_rays(np.random.default_rng(8), 100, 400, 8192, az, el)
    tree = O.build_octree(scene.leaf_ijk, 8)
    rays = rays[~O.trace(tree, rays, 16).degenerate]
    w = I.Workload("deep", scene, shape, 16, feats, params, rays)
    rgb_t = np.random.default_rng(9).uniform(0, 1, size=(rays.shape[0], 3)).astype(np.float32)
    depth_t, mask = I.analytic_depth(rays, scene)
    ref = O.render(tree, feats, params, O.layer_dims(32, 128, 4), rays, 16)
    mask = np.where(np.abs(ref.depth - depth_t) < 1e-4, 0.0, mask).astype(np.float32)
    assert (ref.hits.n > 0).sum() > 1000
    precision = svlf.PRECISIONS[prec]
    L, rgb, depth, d_rgb, d_depth, df, dp = _gpu_grads(w, precision, params, (0, 0, 0), rgb_t, depth_t, mask)
    _, _, dfe, dpe, _, _ = _oracle_grads(w, params, (0, 0, 0), rgb_t, depth_t, mask, bf16=prec)
    _, _, df64, dp64, _, _ = _oracle_grads(w, params, (0, 0, 0), rgb_t, depth_t, mask)
    e_f, e_p = _rel(df, dfe), _rel(dp, dpe)
    print(f"{prec} 4x128: vs emulating oracle features {e_f:.2e} network {e_p:.2e}; "
          f"vs FP64 features {_rel(df, df64):.2e} network {_rel(dp, dp64):.2e}")
    assert e_f <= 1e-2 and e_p <= 1e-2
    off = 0
    for o, i in O.layer_dims(32, 128, 4):
        for n in (o * i, o):
            assert _rel(dp[off:off + n], dpe[off:off + n]) <= 3e-2
            off += n
