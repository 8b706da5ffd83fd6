"""Pins for the oracle's traversal (slab test per voxel, Sec. 4.2; hits in
order of intersection along the ray, Sec. 4.3)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2205_07058_b300 import inputs as I


def test_morton_bit_order():
    L = O.lib()
    assert [L.oracle_morton(*c, 3) for c in [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 1)]] \
        == [0, 1, 2, 4, 7]
    assert L.oracle_morton(2, 0, 0, 3) == 8 and L.oracle_morton(0, 0, 4, 3) == 256
    assert L.oracle_morton(7, 7, 7, 3) == 511


def test_leaf_set_dedups_sorts_and_rejects_out_of_range():
    ijk = np.array([[1, 0, 0], [0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=np.int32)
    t = O.build_octree(ijk, 2)
    assert t.n_leaves == 3
    assert t.codes.tolist() == [0, 1, 2]
    assert t.leaf_ijk().tolist() == [[0, 0, 0], [1, 0, 0], [0, 1, 0]]
    with pytest.raises(ValueError):
        O.build_octree(np.array([[4, 0, 0]], dtype=np.int32), 2)


def _column_tree(depth, i, j, ks):
    ijk = np.array([[i, j, k] for k in ks], dtype=np.int32)
    return O.build_octree(ijk, depth)


@pytest.mark.parametrize("direction", [+1, -1])
def test_axis_aligned_column_closed_form(direction):
    """A ray along +-z through the centre of column (i, j) meets the leaves of
    that column in z order, at t = |k h - o_z| exactly."""
    depth, i, j = 3, 5, 2
    h = 2.0 ** -depth
    ks = [0, 2, 3, 7]
    tree = _column_tree(depth, i, j, ks)
    oz = -0.5 if direction > 0 else 1.5
    ray = np.array([[(i + 0.5) * h, (j + 0.5) * h, oz, 0, 0, direction]], dtype=np.float32)
    for mode in ("dda", "brute"):
        hits = O.trace(tree, ray, 8, mode)
        order = ks if direction > 0 else ks[::-1]
        assert hits.n[0] == 4
        # ranks: leaves sorted by Morton code = by k for a single column
        assert hits.rank[0, :4].tolist() == [ks.index(k) for k in order]
        t_expect = [(k * h - oz) if direction > 0 else (oz - (k + 1) * h) for k in order]
        np.testing.assert_array_equal(hits.t_in[0, :4], np.array(t_expect))
        np.testing.assert_array_equal(hits.t_out[0, :4], np.array(t_expect) + h)
        assert hits.rank[0, 4:].tolist() == [-1] * 4


def test_single_leaf_and_eight_leaves():
    tree = O.build_octree(np.array([[1, 1, 1]], dtype=np.int32), 2)
    # diagonal ray through the cube centre region hits voxel (1,1,1) of a 4^3 grid
    d = np.array([1.0, 1.0, 1.0]) / math.sqrt(3.0)
    o = np.array([0.3, 0.3, 0.3]) - 2 * d
    ray = np.concatenate([o, d]).astype(np.float32)[None, :]
    for mode in ("dda", "brute"):
        h = O.trace(tree, ray, 4, mode)
        assert h.n[0] == 1 and h.rank[0, 0] == 0
    # all 8 voxels of a 2^3 grid: an x-aligned ray through y,z in cell 0 meets cells 0 and 1
    all8 = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], dtype=np.int32)
    tree = O.build_octree(all8, 1)
    ray = np.array([[-1.0, 0.25, 0.75, 1.0, 0.0, 0.0]], dtype=np.float32)
    for mode in ("dda", "brute"):
        h = O.trace(tree, ray, 4, mode)
        assert h.n[0] == 2 and h.rank[0, :2].tolist() == [4, 5]
        np.testing.assert_array_equal(h.t_in[0, :2], [1.0, 1.5])


def _random_rays(rng, n, inside_frac=0.3):
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = rng.uniform(-1.5, 2.5, size=(n, 3))
    m = rng.uniform(size=n) < inside_frac
    o[m] = rng.uniform(0.0, 1.0, size=(m.sum(), 3))  # origins inside the cube (t clipped at 0)
    return np.concatenate([o, d], axis=1).astype(np.float32)


@pytest.mark.parametrize("K", [1, 4, 32])
def test_dda_equals_brute_force(tiny, K):
    tree = O.build_octree(tiny.scene.leaf_ijk, tiny.scene.depth)
    rng = np.random.default_rng(7)
    rays = np.concatenate([tiny.rays, _random_rays(rng, 3000)])
    a = O.trace(tree, rays, K, "dda")
    b = O.trace(tree, rays, K, "brute")
    np.testing.assert_array_equal(a.rank, b.rank)
    np.testing.assert_array_equal(a.n, b.n)
    np.testing.assert_array_equal(a.t_in, b.t_in)
    np.testing.assert_array_equal(a.t_out, b.t_out)
    assert (a.n > 0).sum() > 300
    # segments are positive, ordered and disjoint
    for r in np.nonzero(a.n > 1)[0][:200]:
        n = a.n[r]
        assert np.all(a.t_out[r, :n] > a.t_in[r, :n])
        assert np.all(a.t_in[r, 1:n] >= a.t_out[r, :n - 1])


def test_single_sphere_hit_bounds():
    """One sphere: the first hit starts no later than the analytic surface hit
    and lies within (1 + sqrt(3)/2) 2^-L of the surface; rays that pass the
    sphere by more than that meet no leaf."""
    depth = 6
    hL = 2.0 ** -depth
    c = np.array([0.5, 0.45, 0.55])
    rad = 0.2
    leaves = I.voxelize(np.array([[*c, rad]]), np.zeros((0, 6)), depth)
    tree = O.build_octree(leaves, depth)
    rays = I.pinhole_rays(0.7, 0.3, 48, 48, fov_deg=15.0)
    hits = O.trace(tree, rays, 4)
    o = rays[:, :3].astype(np.float64)
    d = rays[:, 3:].astype(np.float64)
    oc = o - c
    b = np.sum(oc * d, axis=1)
    q = oc - b[:, None] * d
    miss_dist = np.linalg.norm(q, axis=1) - rad
    bound = (1.0 + math.sqrt(3.0) / 2.0) * hL
    far = miss_dist > bound
    assert far.sum() > 100 and np.all(hits.n[far] == 0)
    through = miss_dist < -bound
    assert through.sum() > 100 and np.all(hits.n[through] > 0)
    t_star = -b - np.sqrt(np.maximum(rad * rad - np.sum(q * q, axis=1), 0))
    sel = np.nonzero(through)[0]
    assert np.all(hits.t_in[sel, 0] <= t_star[sel] + 1e-12)
    x1 = o[sel] + hits.t_in[sel, 0:1] * d[sel]
    assert np.all(np.abs(np.linalg.norm(x1 - c, axis=1) - rad) <= bound + 1e-12)


def test_box_shell_hit_bounds():
    depth = 6
    hL = 2.0 ** -depth
    box = np.array([[0.5, 0.5, 0.5, 0.2, 0.15, 0.1]])
    leaves = I.voxelize(np.zeros((0, 4)), box, depth)
    tree = O.build_octree(leaves, depth)
    rays = I.pinhole_rays(1.1, 0.4, 48, 48, fov_deg=15.0)
    hits = O.trace(tree, rays, 4)
    D, mask = I.analytic_depth(rays, I.Scene(depth, np.zeros((0, 4)), box, leaves))
    hit = mask > 0
    assert hit.sum() > 100
    bound = (1.0 + math.sqrt(3.0) / 2.0) * hL
    sel = np.nonzero(hit & (hits.n > 0))[0]
    assert len(sel) > 0.9 * hit.sum()
    assert np.all(hits.t_in[sel, 0] <= D[sel] + 1e-6)
    assert np.all(D[sel] - hits.t_in[sel, 0] <= 2 * bound + 1e-6)


def test_near_degenerate_flag():
    """A ray through a voxel edge next to a leaf is flagged; the same ray moved
    off the edge is not; rays far from every leaf are never flagged."""
    depth = 3
    h = 2.0 ** -depth
    d = np.array([1.0, 1.0, 0.3])
    d /= np.linalg.norm(d)
    # edge x = y = 2h at z ~ 0.41 (cell k = 3): leaf (2, 1, 3) borders it
    tree = O.build_octree(np.array([[2, 1, 3]], dtype=np.int32), depth)
    o = np.array([2 * h, 2 * h, 0.41]) - 3 * d
    rays = np.array([np.concatenate([o, d]),
                     np.concatenate([o + np.array([0.013, 0.0, 0.0]), d])], dtype=np.float32)
    hits = O.trace(tree, rays, 4)
    assert hits.degenerate.tolist() == [True, False]
    far = O.build_octree(np.array([[7, 0, 0]], dtype=np.int32), depth)
    assert not O.trace(far, rays[:1], 4).degenerate[0]


def test_degenerate_fraction_is_small(tiny):
    tree = O.build_octree(tiny.scene.leaf_ijk, tiny.scene.depth)
    hits = O.trace(tree, tiny.rays, tiny.K)
    assert hits.degenerate.sum() <= 0.01 * (hits.n > 0).sum() + 2
