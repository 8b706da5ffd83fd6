"""Pins for the ray parameterisation r = [p~1 | p~2] (Sec. 4.1): the ray's
entry and exit points on the voxel's minimum bounding sphere, relative to
the voxel centre, scaled to unit norm."""
import math

import numpy as np

from oracle import oracle as O


def _rand(rng, n):
    c = rng.uniform(0.2, 0.8, size=(n, 3))
    R = 0.5 * math.sqrt(3.0) * 2.0 ** -9
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


def test_matches_textbook_quadratic_in_extended_precision():
    """Solve a t^2 + 2 b t + cc = 0 directly in long double and compare."""
    rng = np.random.default_rng(3)
    o, d, c, R = _rand(rng, 500)
    p1, p2 = O.sphere_params(o, d, c, R)
    ld = np.longdouble
    oL, dL, cL = o.astype(ld), d.astype(ld), c.astype(ld)
    oc = oL - cL
    a = np.sum(dL * dL, axis=1)
    b = np.sum(dL * oc, axis=1)
    cc = np.sum(oc * oc, axis=1) - ld(R) * ld(R)
    disc = np.sqrt(b * b - a * cc)
    for t, p in (((-b - disc) / a, p1), ((-b + disc) / a, p2)):
        x = oL + t[:, None] * dL - cL
        x /= np.sqrt(np.sum(x * x, axis=1))[:, None]
        np.testing.assert_allclose(p, x.astype(np.float64), atol=1e-8)
