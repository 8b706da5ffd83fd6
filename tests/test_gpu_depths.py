"""Hit lists bit-exact against the oracle's finest-grid walk at every
supported octree depth (2 .. 10), on scenes that mix dense surface shells with
isolated leaves in large empty regions (so empty blocks of every size are
skipped), for rays in general position and rays parallel to one or two axes."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2205_07058_b300 import inputs as I
from tests.gpu_common import compare_hits, random_rays, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


def _scene_leaves(rng, depth):
    n = 1 << depth
    if depth <= 4:
        occ = rng.uniform(size=(n, n, n)) < 0.15
        ijk = np.argwhere(occ)
    else:
        ijk = I.make_scene(rng, depth, 6, 3).leaf_ijk
    # isolated leaves anywhere, including the cube's faces and corners
    iso = rng.integers(0, n, size=(64, 3))
    corners = np.array([[0, 0, 0], [n - 1, n - 1, n - 1], [0, n - 1, 0], [n - 1, 0, n - 1]])
    return np.unique(np.concatenate([ijk, iso, corners]).astype(np.int32), axis=0)


def _axis_rays(rng, n):
    r = random_rays(rng, n, inside_frac=0.5)
    d = r[:, 3:].astype(np.float64)
    for q in range(n):
        k = q % 3
        zero = rng.choice(3, size=1 + (q % 2), replace=False) if k else []
        d[q, list(zero)] = 0.0
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    # rays with zeroed components start inside the cube so they can hit something
    o = r[:, :3].astype(np.float64)
    flat = (d == 0).any(axis=1)
    o[flat] = rng.uniform(0.0, 1.0, size=(flat.sum(), 3))
    return np.concatenate([o, d], axis=1).astype(np.float32)


@pytest.mark.parametrize("depth", [2, 3, 4, 5, 6, 8, 10])
def test_hit_lists_bit_exact_across_depths(depth):
    from paper_2205_07058_b300 import svlf
    rng = np.random.default_rng(700 + depth)
    ijk = _scene_leaves(rng, depth)
    rays = np.concatenate([random_rays(rng, 6000), _axis_rays(rng, 3000)])
    K = 8
    tree = svlf.Octree(torch.from_numpy(ijk), depth)
    feats = torch.zeros(tree.n_leaves, 8, device="cuda")
    net = svlf.Network(8, 32, 1, svlf.FP32)
    params = torch.zeros(I.MLPShape(8, 32, 1).n_params, device="cuda")
    _, _, hits, tio, _ = svlf.svlf_render_rays(tree, feats, params, net, torch.from_numpy(rays).cuda(), K,
                                               want_hits=True)
    torch.cuda.synchronize()
    assert svlf.svlf_get_device_status() == 0
    oh = O.trace(O.build_octree(ijk, depth), rays, K)
    n_ok, n_deg, mism = compare_hits(oh, hits.cpu().numpy(), tio.cpu().numpy())
    assert n_ok > 8500
    assert (oh.n > 0).sum() > 500
    assert mism <= n_deg
