"""Traversal order for image rays (svlf_render_opts.image_width): the rays of
whole images walked in tiles of 8 x 4 pixels instead of in their own order.
The order is a schedule only, so colours, depth, hit lists and segments are
bit-identical to the given-order walk, and agree with the FP64 oracle; the
backward after a tiled render differs only in the summation order of the
parameter gradients. Covers the single-scene call (FP32 and BF16; hit slots
in shared memory, K = 4, and in global scratch, K = 32), a batched
call mixing an image scene with a scene of scattered rays and one whose ray
count is not whole bands of four rows (both kept in their order), widths that
fall back to the given order, and the argument check."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2205_07058_b300 import inputs as I
from tests.gpu_common import compare_hits, random_rays, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]

W = 48  # image width and height: six tiles of 8 pixels per row, twelve bands of four rows


@pytest.fixture(scope="module")
def scene():
    rng = np.random.default_rng(4242)
    sc = I.make_scene(rng, 6, 10, 3)
    rays = np.concatenate([I.pinhole_rays(math.radians(a), math.radians(e), W, W)
                           for a, e in ((30, 25), (150, -10), (260, 40))])
    feats = I.make_features(rng, sc.n_leaves, 16)
    params = I.make_mlp(rng, I.MLPShape(16, 64, 2), bias_std=0.3)
    params[-1] += 1.0  # positive optical thickness: every ray with hits has a gradient
    return sc, rays, feats, params


def _render(svlf, tree, f, p, net, r, K, width):
    rgb, depth, hits, t_io, ws = svlf.svlf_render_rays(tree, f, p, net, r, K, bg=(0.2, 0.1, 0.3), want_hits=True,
                                                       image_width=width)
    torch.cuda.synchronize()
    assert svlf.svlf_get_device_status() == 0
    return rgb, depth, hits, t_io, ws


# K = 4: hit slots in shared memory; K = 32: in the global scratch area
@pytest.mark.parametrize("precision,K", [("fp32", 4), ("bf16", 4), ("bf16", 32)])
def test_tiled_walk_is_bit_identical_and_matches_the_oracle(scene, precision, K):
    from paper_2205_07058_b300 import svlf
    sc, rays, feats, params = scene
    prec = svlf.FP32 if precision == "fp32" else svlf.BF16
    net = svlf.Network(16, 64, 2, prec)
    tree = svlf.Octree(torch.from_numpy(sc.leaf_ijk), sc.depth)
    f, p, r = (torch.from_numpy(x).cuda() for x in (feats, params, rays))
    ref = _render(svlf, tree, f, p, net, r, K, 0)
    til = _render(svlf, tree, f, p, net, r, K, W)
    for a, b in zip(ref[:4], til[:4]):
        assert torch.equal(a, b)
    # widths that do not divide the rays into whole 8 x 4 tiles keep the given order
    for width in (12, 40, 3 * W * W):
        other = _render(svlf, tree, f, p, net, r, K, width)
        for a, b in zip(ref[:4], other[:4]):
            assert torch.equal(a, b)
    # the hit lists of the tiled walk against the oracle's traversal
    hits = O.trace(O.build_octree(sc.leaf_ijk, sc.depth), rays, K)
    n_ok, _, _ = compare_hits(hits, til[2].cpu().numpy(), til[3].cpu().numpy())
    assert n_ok > 0.9 * rays.shape[0] and (hits.n > 0).sum() > 500


def test_backward_after_a_tiled_render(scene):
    """The backward reads the samples in the order the walk wrote them: the
    gradients equal those after a given-order render up to summation order."""
    from paper_2205_07058_b300 import svlf
    sc, rays, feats, params = scene
    K = 4
    net = svlf.Network(16, 64, 2, svlf.BF16)
    tree = svlf.Octree(torch.from_numpy(sc.leaf_ijk), sc.depth)
    f, p, r = (torch.from_numpy(x).cuda() for x in (feats, params, rays))
    rng = np.random.default_rng(7)
    g_rgb = torch.from_numpy(rng.standard_normal((rays.shape[0], 3)).astype(np.float32)).cuda()
    g_depth = torch.from_numpy(rng.standard_normal(rays.shape[0]).astype(np.float32)).cuda()
    grads = []
    for width in (0, W):
        _, _, _, _, ws = _render(svlf, tree, f, p, net, r, K, width)
        df = torch.zeros_like(f)
        dp = torch.zeros_like(p)
        svlf.svlf_render_rays_backward(tree, f, p, net, r, K, (0.2, 0.1, 0.3), g_rgb, g_depth, df, dp, ws)
        torch.cuda.synchronize()
        assert svlf.svlf_get_device_status() == 0
        grads.append(torch.cat([df.reshape(-1), dp]).double())
    a, b = grads
    assert a.norm() > 0
    assert ((a - b).norm() / a.norm()).item() <= 1e-5


def test_batched_call_tiles_only_the_image_scenes(scene):
    from paper_2205_07058_b300 import svlf
    sc, rays, feats, params = scene
    K = 4
    net = svlf.Network(16, 64, 2, svlf.BF16)
    tree = svlf.Octree(torch.from_numpy(sc.leaf_ijk), sc.depth)
    f, p = torch.from_numpy(feats).cuda(), torch.from_numpy(params).cuda()
    rng = np.random.default_rng(11)
    sets = [rays, random_rays(rng, 3001), rays[: 2 * W * W + 5 * W]]  # image, scattered, ragged band
    outs = []
    for width in (0, W):
        scenes = [svlf.BatchScene(tree, f, p, torch.from_numpy(x).cuda()) for x in sets]
        svlf.svlf_render_rays_batched(scenes, net, K, image_width=width)
        torch.cuda.synchronize()
        assert svlf.svlf_get_device_status() == 0
        outs.append([(s.rgb, s.depth) for s in scenes])
    for (a_rgb, a_d), (b_rgb, b_d) in zip(*outs):
        assert torch.equal(a_rgb, b_rgb) and torch.equal(a_d, b_d)


def test_negative_width_is_refused(scene):
    from paper_2205_07058_b300 import svlf
    sc, rays, feats, params = scene
    net = svlf.Network(16, 64, 2, svlf.BF16)
    tree = svlf.Octree(torch.from_numpy(sc.leaf_ijk), sc.depth)
    f, p, r = (torch.from_numpy(x).cuda() for x in (feats, params, rays))
    with pytest.raises(svlf.SvlfError) as e:
        svlf.svlf_render_rays(tree, f, p, net, r, 4, image_width=-8)
    assert e.value.code == svlf.SVLF_ERR_ARG
