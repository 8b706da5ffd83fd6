"""Pins of the depth-map voxelisation: closed forms and properties that fix
it, independent of its own formula."""
import math

import numpy as np

from oracle import depth_octree as DO
from paper_2205_07058_b300 import inputs as I


def test_plane_at_known_height_closed_form():
    """A camera looking straight down at the plane z = 0.3: every point's z
    voxel is floor(0.3 * 2^L) and the x, y voxels cover the footprint."""
    L = 6
    n = 1 << L
    xs, ys = np.meshgrid(np.linspace(0.1, 0.9, 40), np.linspace(0.2, 0.8, 30))
    o = np.stack([xs.ravel(), ys.ravel(), np.full(xs.size, 0.95)], axis=1)
    d = np.tile([0.0, 0.0, -1.0], (xs.size, 1))
    rays = np.concatenate([o, d], axis=1).astype(np.float32)
    depth = np.full(xs.size, 0.95 - 0.3, dtype=np.float32)
    v = DO.depth_voxels(rays, depth, L)
    zc = np.floor(np.float32(np.float32(0.95) + np.float32(-0.65)) * n)
    assert np.all(v[:, 2] == zc)
    expect = {(int(math.floor(x * n)), int(math.floor(y * n))) for x, y in zip(o[:, 0].astype(np.float32),
                                                                                o[:, 1].astype(np.float32))}
    assert {(a, b) for a, b, _ in v} == expect


def test_invalid_depths_skipped_and_unique():
    rays = np.tile(np.array([[0.5, 0.5, 0.5, 1.0, 0.0, 0.0]], np.float32), (6, 1))
    depth = np.array([0.1, 0.1, np.nan, -1.0, 0.0, np.inf], np.float32)
    v = DO.depth_voxels(rays, depth, 4)
    assert v.shape == (1, 3) and tuple(v[0]) == (9, 8, 8)  # floor(0.6 * 16) = 9


def test_depth_points_of_an_analytic_scene_lie_in_surface_voxels():
    """Back-projected analytic depths are surface points, so every voxel found
    has its centre within sqrt(3)/2 voxel of a primitive's surface: inside the
    occupancy band |SDF(centre)| <= 2^-L of the voxelised scene."""
    rng = np.random.default_rng(1012)
    L = 7
    sc = I.make_scene(rng, L, 6, 3)
    az, el = I.random_view_angles(rng, 3)
    rays = np.concatenate([I.pinhole_rays(az[v], el[v], 64, 64) for v in range(3)])
    depth, mask = I.analytic_depth(rays, sc)
    depth = np.where(mask > 0, depth, np.nan).astype(np.float32)
    v = DO.depth_voxels(rays, depth, L)
    assert v.shape[0] > 500
    occupied = {tuple(x) for x in sc.leaf_ijk}
    missing = [tuple(x) for x in v if tuple(x) not in occupied]
    assert len(missing) == 0, missing[:5]
