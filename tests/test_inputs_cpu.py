"""The seeded input generators: the threaded C helper for the analytic depth
targets gives, bit for bit, what the array formulation gives (rays from the
pinhole views plus axis-parallel rays and origins inside primitives)."""
import numpy as np

from paper_2205_07058_b300 import inputs as I


def test_analytic_depth_helper_matches_array_formulation():
    rng = np.random.default_rng(1002)
    scene = I.make_scene(rng, 6, 24, 12)
    az, el = I.random_view_angles(rng, 2)
    rays = np.concatenate([I.pinhole_rays(az[v], el[v], 64, 64) for v in range(2)])
    extra = np.array([[0.5, 0.5, -1, 0, 0, 1], [0.3, 0.3, 0.3, 1, 0, 0], [0.5, 0.5, 0.5, 0, 1, 0],
                      [0.35, 0.36, 2, 0, 0, -1], [-1, 0.5, 0.5, 1, 0, 0]], dtype=np.float32)
    from_centres = np.concatenate([scene.spheres[:4, :3], np.tile([[0.0, 0.6, 0.8]], (4, 1))], axis=1)
    rays = np.concatenate([rays, extra, from_centres.astype(np.float32)])
    d1, m1 = I.analytic_depth(rays, scene)
    d2, m2 = I._analytic_depth_numpy(rays, scene)
    assert np.array_equal(m1, m2) and np.array_equal(d1, d2)
    assert 0.05 < m1.mean() < 0.95 and np.all(m1[-4:] == 1)  # rays from sphere centres leave them
