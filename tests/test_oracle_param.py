"""Pins for the ray parameterisation r = [p~1 | p~2] (Sec. 4.1): the ray's
entry and exit points on the voxel's minimum bounding sphere, relative to
the voxel centre, scaled to unit norm."""
import math

import pytest

import numpy as np

from oracle import oracle as O


def _rand(rng, n, L=9):
    c = rng.uniform(0.2, 0.8, size=(n, 3))
    R = 0.5 * math.sqrt(3.0) * 2.0 ** -L
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    # aim at a random point inside the sphere from about 2.5 away
    tgt = c + rng.uniform(-0.55, 0.55, size=(n, 3)) * R
    o = tgt - 2.5 * d
    return o, d, c, R


def test_unit_norm_and_on_sphere():
    rng = np.random.default_rng(0)
    o, d, c, R = _rand(rng, 2000)
    p1, p2 = O.sphere_params(o, d, c, R)
    np.testing.assert_allclose(np.linalg.norm(p1, axis=1), 1.0, atol=1e-14)
    np.testing.assert_allclose(np.linalg.norm(p2, axis=1), 1.0, atol=1e-14)
    # entry before exit: (p2 - p1) points along d
    assert np.all(np.sum((p2 - p1) * d, axis=1) > 0)


def test_through_centre_gives_minus_d_plus_d():
    rng = np.random.default_rng(1)
    c = rng.uniform(0.2, 0.8, size=(100, 3))
    d = rng.standard_normal((100, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = c - 2.5 * d
    p1, p2 = O.sphere_params(o, d, c, 0.01)
    np.testing.assert_allclose(p1, -d, atol=1e-12)
    np.testing.assert_allclose(p2, d, atol=1e-12)


def test_tangent_ray_entry_equals_exit():
    c = np.array([[0.5, 0.5, 0.5]])
    R = 0.01
    d = np.array([[0.0, 1.0, 0.0]])
    o = np.array([[0.5 + R, -2.0, 0.5]])
    p1, p2 = O.sphere_params(o, d, c, R)
    np.testing.assert_allclose(p1, [[1.0, 0.0, 0.0]], atol=1e-12)
    np.testing.assert_allclose(p2, [[1.0, 0.0, 0.0]], atol=1e-12)


def test_reversed_ray_swaps_entry_and_exit():
    rng = np.random.default_rng(2)
    o, d, c, R = _rand(rng, 500)
    p1, p2 = O.sphere_params(o, d, c, R)
    q1, q2 = O.sphere_params(o + 5.0 * d, -d, c, R)
    np.testing.assert_allclose(q1, p2, atol=1e-10)
    np.testing.assert_allclose(q2, p1, atol=1e-10)


@pytest.mark.parametrize("L", [2, 4, 6, 9, 10])
def test_matches_textbook_quadratic_in_extended_precision(L):
    """Solve a t^2 + 2 b t + cc = 0 directly in long double and compare.

    In float64 the foot of the perpendicular carries a rounding error of a
    few ulp of |o - c| (~2.5), which the normalisation divides by R, so the
    attainable agreement is about eps64 |o - c| / R: 1e-13 holds for voxels
    down to depth 4 and the bound 16 eps64 |o - c| / R (1.4e-12 at depth 10)
    holds at every depth."""
    rng = np.random.default_rng(3)
    o, d, c, R = _rand(rng, 2000, L)
    p1, p2 = O.sphere_params(o, d, c, R)
    ld = np.longdouble
    oL, dL, cL = o.astype(ld), d.astype(ld), c.astype(ld)
    oc = oL - cL
    a = np.sum(dL * dL, axis=1)
    b = np.sum(dL * oc, axis=1)
    cc = np.sum(oc * oc, axis=1) - ld(R) * ld(R)
    disc = np.sqrt(b * b - a * cc)
    bound = 16.0 * np.finfo(np.float64).eps * np.linalg.norm(o - c, axis=1) / R
    if L <= 4:
        bound = np.minimum(bound, 1e-13)
    for t, p in (((-b - disc) / a, p1), ((-b + disc) / a, p2)):
        x = oL + t[:, None] * dL - cL
        x /= np.sqrt(np.sum(x * x, axis=1))[:, None]
        err = np.abs(p - x.astype(np.float64)).max(axis=1)
        assert np.all(err <= bound), float((err / bound).max())


# ----------------------------------------------------------------------------
# The voxel's minimum bounding sphere and the network input assembly
# (Sec. 4.1 "Ray parameterization"): the sphere of a cube voxel
# [ijk, ijk + 1] * 2^-L is the one through its eight corners, centred on the
# voxel centre with radius half the cube diagonal. These pins fail for the
# inscribed radius 2^-L / 2 and for a centre at the voxel's low corner.
# ----------------------------------------------------------------------------
def _corners(ijk, L):
    h = 2.0 ** -L
    offs = np.array([[a, b, c] for c in (0, 1) for b in (0, 1) for a in (0, 1)], dtype=np.float64)
    return (ijk[:, None, :].astype(np.float64) + offs[None]) * h


def test_bounding_sphere_passes_through_all_eight_corners():
    rng = np.random.default_rng(11)
    for L in range(2, 11):
        ijk = rng.integers(0, 2 ** L, size=(64, 3))
        c, R = O.voxel_centre_radius(ijk, L)
        dist = np.linalg.norm(_corners(ijk, L) - c[:, None, :], axis=2)
        # equidistant corners: c is the cube centre; the common distance is R
        np.testing.assert_allclose(dist, R, rtol=1e-15, atol=0)
        # half the cube diagonal, from the voxel's own corners
        diag = np.linalg.norm(_corners(ijk, L)[:, 7] - _corners(ijk, L)[:, 0], axis=1)
        np.testing.assert_allclose(R, 0.5 * diag, rtol=1e-15)


def _corner_ray(L, ijk, d):
    """A float32 ray whose line passes (to float32 rounding of the origin)
    through the low corner of voxel ijk, entering the voxel there."""
    h = 2.0 ** -L
    d32 = (np.asarray(d, dtype=np.float64) / np.linalg.norm(d)).astype(np.float32)
    corner = np.asarray(ijk, dtype=np.float64) * h
    o32 = (corner - 0.25 * d32.astype(np.float64)).astype(np.float32)
    return np.concatenate([o32, d32])[None, :].astype(np.float32)


@pytest.mark.parametrize("direction", [(1.0, 2.0, 3.0), (3.0, 1.0, 2.0), (1.0, 1.0, 1.0)])
def test_ray_entering_at_a_corner_enters_the_sphere_there(direction):
    """A ray that enters the voxel exactly at its low corner enters the
    bounding sphere at that corner too (the corner lies on the sphere and the
    voxel lies inside it), so through trace + sample_inputs p~1 =
    (corner - c) / R = -(1, 1, 1)/sqrt(3) for every such direction, not only
    the cube diagonal."""
    L = 3
    ijk = np.array([3, 4, 2])
    tree = O.build_octree(ijk[None, :].astype(np.int32), L)
    ray = _corner_ray(L, ijk, direction)
    hits = O.trace(tree, ray, 4)
    assert hits.n[0] == 1 and hits.rank[0, 0] == 0
    F = 4
    feats = np.arange(F, dtype=np.float32)[None, :] + 1.0
    ray_of, slot, rank, h0, tmid = O.sample_inputs(tree, ray, hits, feats)
    p1 = h0[0, F + 3:F + 6]
    np.testing.assert_allclose(p1, -np.ones(3) / math.sqrt(3.0), atol=2e-6)
    if np.allclose(direction, 1.0):
        # along the diagonal the exit is the opposite corner
        np.testing.assert_allclose(h0[0, F + 6:F + 9], np.ones(3) / math.sqrt(3.0), atol=2e-6)


def _scene_hits(seed, L, n_rays):
    from paper_2205_07058_b300 import inputs as I
    rng = np.random.default_rng(seed)
    scene = I.make_scene(rng, L, 6, 3)
    tree = O.build_octree(scene.leaf_ijk, L)
    az, el = I.random_view_angles(rng, 1)
    rays = I.pinhole_rays(az[0], el[0], 48, 48)[:n_rays]
    hits = O.trace(tree, rays, 6)
    return tree, rays, hits


@pytest.mark.parametrize("L", [4, 6, 9])
def test_sample_inputs_columns_and_sphere_points_on_the_ray(L):
    """h0 = [z | d | p~1 | p~2]: z is the hit leaf's feature row, d the ray
    direction; c + R p~i (c, R written out here from the voxel's corners) lie
    on the ray, p~1 before p~2 along d, and the hit segment's midpoint lies
    inside the voxel of the hit leaf's coordinates."""
    tree, rays, hits = _scene_hits(100 + L, L, 48 * 48)
    F = 5
    feats = np.random.default_rng(1).standard_normal((tree.n_leaves, F)).astype(np.float32)
    ray_of, slot, rank, h0, tmid = O.sample_inputs(tree, rays, hits, feats)
    assert h0.shape == (ray_of.shape[0], F + 9) and ray_of.shape[0] > 100
    np.testing.assert_array_equal(h0[:, :F], feats[hits.rank[ray_of, slot]].astype(np.float64))
    o = rays[ray_of, :3].astype(np.float64)
    d = rays[ray_of, 3:].astype(np.float64)
    np.testing.assert_array_equal(h0[:, F:F + 3], d)
    ijk = tree.leaf_ijk()[rank]
    cr = _corners(ijk, L)
    c = cr.mean(axis=1)
    R = 0.5 * np.linalg.norm(cr[:, 7] - cr[:, 0], axis=1)
    h = 2.0 ** -L
    for col in (F + 3, F + 6):
        pt = c + R[:, None] * h0[:, col:col + 3]
        off = np.cross(pt - o, d)  # distance from the ray's line
        assert np.abs(off).max() <= 1e-9 * max(1.0, 1.0 / (R.min() * 1e3)), np.abs(off).max()
    t1 = np.sum((c + R[:, None] * h0[:, F + 3:F + 6] - o) * d, axis=1)
    t2 = np.sum((c + R[:, None] * h0[:, F + 6:F + 9] - o) * d, axis=1)
    assert np.all(t2 > t1)
    # the sphere chord contains the voxel's slab segment
    t_in, t_out = hits.t_in[ray_of, slot], hits.t_out[ray_of, slot]
    assert np.all(t1 <= t_in + 1e-12) and np.all(t2 >= t_out - 1e-12)
    mid = o + tmid[:, None] * d
    assert np.all(mid >= ijk * h - 1e-12) and np.all(mid <= (ijk + 1) * h + 1e-12)


# ----------------------------------------------------------------------------
# The voxel-box reading (rparam "aabb"): r = [x~1 | x~2] = the slab segment's
# ends in voxel-local coordinates (x - c) / (h / 2).
# ----------------------------------------------------------------------------
def test_aabb_reading_axis_column_closed_form():
    """A ray along +z through the centre of a column enters every leaf at its
    low z face and leaves at its high face: x~1 = (0, 0, -1), x~2 = (0, 0, 1)
    exactly; for a ray off the column centre by (a, b) h / 2 the first two
    components are (a, b)."""
    L, i, j = 3, 5, 2
    h = 2.0 ** -L
    tree = O.build_octree(np.array([[i, j, k] for k in (0, 2, 3)], dtype=np.int32), L)
    for a, b in ((0.0, 0.0), (0.5, -0.25)):
        ray = np.array([[(i + 0.5 + 0.5 * a) * h, (j + 0.5 + 0.5 * b) * h, -0.5, 0, 0, 1]], dtype=np.float32)
        hits = O.trace(tree, ray, 4)
        F = 2
        _, _, _, h0, _ = O.sample_inputs(tree, ray, hits, np.zeros((3, F), np.float32), rparam="aabb")
        assert h0.shape[0] == 3
        np.testing.assert_array_equal(h0[:, F + 3:F + 6], np.tile([a, b, -1.0], (3, 1)))
        np.testing.assert_array_equal(h0[:, F + 6:F + 9], np.tile([a, b, 1.0], (3, 1)))


@pytest.mark.parametrize("L", [4, 9])
def test_aabb_reading_points_are_the_segment_ends_inside_the_box(L):
    """Every x~ lies in [-1, 1]^3; x~2 lies on a face (a component of
    magnitude 1); x~1 lies on a face unless the origin is inside the voxel
    (then x~1 is the origin); c + (h/2) x~i are the points o + t_in d and
    o + t_out d of the slab segment (checked by collinearity with the ray and
    their distance along it), and their midpoint is the sample's midpoint."""
    tree, rays, hits = _scene_hits(300 + L, L, 48 * 48)
    F = 3
    feats = np.zeros((tree.n_leaves, F), np.float32)
    ray_of, slot, rank, h0, tmid = O.sample_inputs(tree, rays, hits, feats, rparam="aabb")
    x1, x2 = h0[:, F + 3:F + 6], h0[:, F + 6:F + 9]
    assert np.all(np.abs(x1) <= 1 + 1e-9) and np.all(np.abs(x2) <= 1 + 1e-9)
    assert np.all(np.abs(np.abs(x2).max(axis=1) - 1.0) <= 1e-9)
    inside = hits.t_in[ray_of, slot] == 0.0
    assert np.all(np.abs(np.abs(x1[~inside]).max(axis=1) - 1.0) <= 1e-9)
    o = rays[ray_of, :3].astype(np.float64)
    d = rays[ray_of, 3:].astype(np.float64)
    h = 2.0 ** -L
    c = (tree.leaf_ijk()[rank] + 0.5) * h
    p1, p2 = c + 0.5 * h * x1, c + 0.5 * h * x2
    for p in (p1, p2):
        assert np.abs(np.cross(p - o, d)).max() <= 1e-12
    np.testing.assert_allclose(np.sum((p2 - p1) * d, axis=1),
                               hits.t_out[ray_of, slot] - hits.t_in[ray_of, slot], atol=1e-12)
    np.testing.assert_allclose(0.5 * (p1 + p2), o + tmid[:, None] * d, atol=1e-12)
