"""Seeded synthetic inputs for the SVLF hot path.

Both the CUDA path and the CPU oracle take these arrays as given; this module
holds none of the rendering method's arithmetic (no traversal, no ray
parameterisation, no network, no compositing). It stands in for the paper's
RTMV scenes, which are not available here:

* scenes live in the unit cube (Sec. 3.1: every scene is normalised to a unit
  cube) and only voxels near a surface are occupied (Sec. 4.1);
* cameras sit on a sphere around the scene centre, like the paper's
  hemisphere placement (Sec. 3.1, camera placements), at radius 2.5 with a
  40 degree field of view;
* the paper's SVLF evaluates fewer than ten voxels per ray on average
  (Sec. 5, timing discussion), which the K = 4..16 hit budgets mirror.

Every generator is driven by ``numpy.random.default_rng(seed)`` with a fixed
draw order: sphere centres, sphere radii, box centres, box half-extents,
features, MLP weights, camera angles, training-ray samples.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libsvlf_inputs.so")


def build_voxelizer(force: bool = False) -> str:
    """Compile the voxeliser helper with gcc (input generation only)."""
    src = os.path.join(_HERE, "voxelize.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        os.makedirs(os.path.dirname(_SO), exist_ok=True)
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC", "-o", tmp, src,
                               "-lm"])
        os.replace(tmp, _SO)
    return _SO


_lib = None


def _voxlib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build_voxelizer())
        _lib.svlf_voxelize_union.restype = ctypes.c_int64
        _lib.svlf_voxelize_union.argtypes = [
            ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
            ctypes.c_int, ctypes.c_void_p, ctypes.c_int64]
        _lib.svlf_analytic_depth.restype = None
        _lib.svlf_analytic_depth.argtypes = [
            ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
            ctypes.c_void_p, ctypes.c_void_p]
    return _lib


# --------------------------------------------------------------------------
# Scenes
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Scene:
    depth: int
    spheres: np.ndarray  # (n, 4) float64: centre xyz, radius
    boxes: np.ndarray    # (m, 6) float64: centre xyz, half-extent xyz
    leaf_ijk: np.ndarray  # (n_leaves, 3) int32, Morton order

    @property
    def n_leaves(self) -> int:
        return int(self.leaf_ijk.shape[0])


def voxelize(spheres: np.ndarray, boxes: np.ndarray, depth: int) -> np.ndarray:
    """Leaves (int32 ijk, Morton order) of the union of solid spheres and box
    shells: voxels whose centre is within 2^-depth of the union surface."""
    lib = _voxlib()
    sph = np.ascontiguousarray(spheres, dtype=np.float64).reshape(-1, 4)
    box = np.ascontiguousarray(boxes, dtype=np.float64).reshape(-1, 6)
    cap = 1 << 16
    while True:
        out = np.zeros((cap, 3), dtype=np.int32)
        n = lib.svlf_voxelize_union(sph.ctypes.data, sph.shape[0], box.ctypes.data,
                                    box.shape[0], depth, out.ctypes.data, cap)
        if n <= cap:
            return out[:n].copy()
        cap = int(n)


def make_scene(rng: np.random.Generator, depth: int, n_spheres: int, n_boxes: int,
               radius_range=(0.05, 0.2), half_range=(0.03, 0.15)) -> Scene:
    """Union of seeded spheres (centres U[0.25,0.75]^3) and box shells."""
    sc = rng.uniform(0.25, 0.75, size=(n_spheres, 3))
    sr = rng.uniform(radius_range[0], radius_range[1], size=(n_spheres, 1))
    bc = rng.uniform(0.25, 0.75, size=(n_boxes, 3))
    bh = rng.uniform(half_range[0], half_range[1], size=(n_boxes, 3))
    spheres = np.concatenate([sc, sr], axis=1)
    boxes = np.concatenate([bc, bh], axis=1)
    return Scene(depth, spheres, boxes, voxelize(spheres, boxes, depth))


# --------------------------------------------------------------------------
# Parameters
# --------------------------------------------------------------------------
@dataclasses.dataclass
class MLPShape:
    feat_dim: int
    hidden: int
    n_hidden: int
    out_dim: int = 4

    @property
    def in_dim(self) -> int:
        return self.feat_dim + 9  # feature | ray dir (3) | p~1 (3) | p~2 (3)

    def layer_dims(self) -> List[tuple]:
        dims = [self.in_dim] + [self.hidden] * self.n_hidden + [self.out_dim]
        return [(dims[i + 1], dims[i]) for i in range(len(dims) - 1)]  # (out, in)

    @property
    def n_params(self) -> int:
        return sum(o * i + o for o, i in self.layer_dims())


def make_features(rng: np.random.Generator, n_leaves: int, feat_dim: int,
                  std: float = 0.1) -> np.ndarray:
    return (rng.standard_normal((n_leaves, feat_dim)) * std).astype(np.float32)


def make_mlp(rng: np.random.Generator, shape: MLPShape, bias_std: float = 0.0) -> np.ndarray:
    """Flat fp32 parameters: per layer W (out x in, row-major) then b (out).
    He initialisation W ~ N(0, 2/fan_in); biases N(0, bias_std^2) (0 = zero)."""
    parts = []
    for o, i in shape.layer_dims():
        parts.append((rng.standard_normal((o, i)) * math.sqrt(2.0 / i)).reshape(-1))
        parts.append(rng.standard_normal(o) * bias_std if bias_std > 0 else np.zeros(o))
    return np.concatenate(parts).astype(np.float32)


def make_mlp_dims(rng: np.random.Generator, dims, bias_std: float = 0.0) -> np.ndarray:
    """Flat fp32 parameters for layers given as (out, in) pairs, initialised as
    make_mlp does."""
    parts = []
    for o, i in dims:
        parts.append((rng.standard_normal((o, i)) * math.sqrt(2.0 / i)).reshape(-1))
        parts.append(rng.standard_normal(o) * bias_std if bias_std > 0 else np.zeros(o))
    return np.concatenate(parts).astype(np.float32)


def split_mlp(flat: np.ndarray, shape: MLPShape):
    """Views (W_l, b_l) into a flat parameter vector."""
    out, off = [], 0
    for o, i in shape.layer_dims():
        W = flat[off:off + o * i].reshape(o, i)
        off += o * i
        b = flat[off:off + o]
        off += o
        out.append((W, b))
    return out


# --------------------------------------------------------------------------
# Cameras and rays
# --------------------------------------------------------------------------
CENTRE = np.array([0.5, 0.5, 0.5])


def camera_basis(azimuth: float, elevation: float, radius: float = 2.5):
    """Camera on a sphere around the scene centre, looking at it, world up +z."""
    ce = math.cos(elevation)
    eye = CENTRE + radius * np.array([ce * math.cos(azimuth), ce * math.sin(azimuth),
                                      math.sin(elevation)])
    fwd = CENTRE - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.array([0.0, 0.0, 1.0]))
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    return eye, fwd, right, up


def pinhole_rays(azimuth: float, elevation: float, width: int, height: int,
                 fov_deg: float = 40.0, radius: float = 2.5,
                 pixels: Optional[np.ndarray] = None) -> np.ndarray:
    """(N, 6) float32 rays (origin, unit direction), row-major over pixel
    centres (+0.5), or over the given (row, col) pixel list."""
    eye, fwd, right, up = camera_basis(azimuth, elevation, radius)
    tan_half = math.tan(math.radians(fov_deg) / 2.0)
    if pixels is None:
        r, c = np.meshgrid(np.arange(height), np.arange(width), indexing="ij")
        r, c = r.reshape(-1), c.reshape(-1)
    else:
        r, c = pixels[:, 0], pixels[:, 1]
    x = (2.0 * (c + 0.5) / width - 1.0) * tan_half
    y = (1.0 - 2.0 * (r + 0.5) / height) * tan_half
    d = fwd[None, :] + x[:, None] * right[None, :] + y[:, None] * up[None, :]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = np.empty((d.shape[0], 6), dtype=np.float32)
    rays[:, :3] = eye[None, :]
    rays[:, 3:] = d
    return rays


def random_view_angles(rng: np.random.Generator, n: int):
    """Directions uniform on the sphere (z ~ U[-1,1], azimuth ~ U[0,2pi)),
    resampled while |z| > 0.98."""
    az = np.empty(n)
    el = np.empty(n)
    for v in range(n):
        while True:
            z = rng.uniform(-1.0, 1.0)
            a = rng.uniform(0.0, 2.0 * math.pi)
            if abs(z) <= 0.98:
                break
        az[v], el[v] = a, math.asin(z)
    return az, el


def _morton2(r: np.ndarray, c: np.ndarray) -> np.ndarray:
    """Interleave the bits of two non-negative integers below 2^16 (Z order)."""
    def spread(x):
        x = x.astype(np.uint64) & np.uint64(0xFFFF)
        x = (x | (x << np.uint64(8))) & np.uint64(0x00FF00FF)
        x = (x | (x << np.uint64(4))) & np.uint64(0x0F0F0F0F)
        x = (x | (x << np.uint64(2))) & np.uint64(0x33333333)
        return (x | (x << np.uint64(1))) & np.uint64(0x55555555)
    return spread(c) | (spread(r) << np.uint64(1))


def training_rays(rng: np.random.Generator, n_views: int, res: int, batch: int,
                  az: np.ndarray, el: np.ndarray, coherent: bool = False) -> np.ndarray:
    """`batch` rays drawn uniformly over (view, pixel) of n_views res x res views.
    With `coherent` the same draws are returned ordered by view, then by the Z
    order of the pixel (neighbouring rows of the batch are neighbouring rays);
    the batch as a set, and every draw, are unchanged."""
    views = rng.integers(0, n_views, size=batch)
    pix = rng.integers(0, res, size=(batch, 2))
    if coherent:
        key = (views.astype(np.uint64) << np.uint64(32)) | _morton2(pix[:, 0], pix[:, 1])
        order = np.argsort(key, kind="stable")
        views, pix = views[order], pix[order]
    rays = np.empty((batch, 6), dtype=np.float32)
    for v in np.unique(views):
        sel = np.nonzero(views == v)[0]
        rays[sel] = pinhole_rays(az[v], el[v], res, res, pixels=pix[sel])
    return rays


# --------------------------------------------------------------------------
# Analytic depth targets (first boundary crossing of the primitives)
# --------------------------------------------------------------------------
def analytic_depth(rays: np.ndarray, scene: Scene):
    """D* = first t >= 0 where the ray meets a sphere or box surface; mask = 1
    where one exists. Computed in float64 from the float32 rays (C helper,
    threaded; the same arithmetic as _analytic_depth_numpy)."""
    r = np.ascontiguousarray(rays, dtype=np.float32).reshape(-1, 6)
    sph = np.ascontiguousarray(scene.spheres, dtype=np.float64).reshape(-1, 4)
    box = np.ascontiguousarray(scene.boxes, dtype=np.float64).reshape(-1, 6)
    depth = np.empty(r.shape[0], dtype=np.float32)
    mask = np.empty(r.shape[0], dtype=np.float32)
    _voxlib().svlf_analytic_depth(r.ctypes.data, r.shape[0], sph.ctypes.data, sph.shape[0], box.ctypes.data,
                                  box.shape[0], depth.ctypes.data, mask.ctypes.data)
    return depth, mask


def _analytic_depth_numpy(rays: np.ndarray, scene: Scene):
    """Array formulation of analytic_depth (slow; kept to check the C helper)."""
    o = rays[:, :3].astype(np.float64)
    d = rays[:, 3:].astype(np.float64)
    best = np.full(o.shape[0], np.inf)
    for cx, cy, cz, r in scene.spheres:
        oc = o - np.array([cx, cy, cz])
        a = np.sum(d * d, axis=1)
        b = np.sum(oc * d, axis=1)
        c = np.sum(oc * oc, axis=1) - r * r
        disc = b * b - a * c
        ok = disc >= 0
        sq = np.sqrt(np.where(ok, disc, 0.0))
        t0 = (-b - sq) / a
        t1 = (-b + sq) / a
        t = np.where(t0 >= 0, t0, t1)
        t = np.where(ok & (t >= 0), t, np.inf)
        best = np.minimum(best, t)
    for cx, cy, cz, hx, hy, hz in scene.boxes:
        lo = np.array([cx - hx, cy - hy, cz - hz])
        hi = np.array([cx + hx, cy + hy, cz + hz])
        with np.errstate(divide="ignore", invalid="ignore"):
            ta = (lo[None, :] - o) / d
            tb = (hi[None, :] - o) / d
        tmin = np.nanmax(np.minimum(ta, tb), axis=1)
        tmax = np.nanmin(np.maximum(ta, tb), axis=1)
        hit = tmax >= np.maximum(tmin, 0.0)
        t = np.where(tmin >= 0, tmin, tmax)  # shell: exit face if starting inside
        best = np.minimum(best, np.where(hit, t, np.inf))
    mask = np.isfinite(best)
    return np.where(mask, best, 0.0).astype(np.float32), mask.astype(np.float32)


# --------------------------------------------------------------------------
# The five benchmark workloads
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    scene: Scene
    mlp: MLPShape
    K: int
    features: np.ndarray
    params: np.ndarray
    rays: np.ndarray
    feat_bf16: bool = False


def tiny_workload(seed: int = 1001, bias_std: float = 0.0) -> Workload:
    """Depth 6, 8 spheres, F = 16 fp32, 25 -> 64 -> 64 -> 4, K = 4, one
    64 x 64 view at azimuth 30 deg, elevation 20 deg."""
    rng = np.random.default_rng(seed)
    scene = make_scene(rng, 6, 8, 0)
    shape = MLPShape(16, 64, 2)
    feats = make_features(rng, scene.n_leaves, 16)
    params = make_mlp(rng, shape, bias_std)
    rays = pinhole_rays(math.radians(30.0), math.radians(20.0), 64, 64)
    return Workload("tiny_d6_4096rays", scene, shape, 4, feats, params, rays)


def full_scene(seed: int = 1002) -> Scene:
    """Depth 9 union of 64 spheres and 32 box shells (~1.6 M leaves)."""
    rng = np.random.default_rng(seed)
    return make_scene(rng, 9, 64, 32)


def full_render_workload(seed: int = 1002, views: int = 4, res: int = 1600,
                         bias_std: float = 0.0) -> Workload:
    rng = np.random.default_rng(seed)
    scene = make_scene(rng, 9, 64, 32)
    shape = MLPShape(32, 128, 3)
    feats = make_features(rng, scene.n_leaves, 32)
    params = make_mlp(rng, shape, bias_std)
    az, el = random_view_angles(rng, views)
    rays = np.concatenate([pinhole_rays(az[v], el[v], res, res) for v in range(views)])
    return Workload(f"render_d9_{views}x{res}sq", scene, shape, 8, feats, params, rays)


def batched_scenes(seed: int = 1004, n: int = 64, min_leaves: float = 1e4, max_leaves: float = 2e6):
    """Scenes of uneven size: depth ~ U{7, 8, 9, 10}, a target leaf count
    log-uniform in [min_leaves, max_leaves], met by choosing how many spheres
    and box shells to draw (about 1.3e3 * 4^(L-6) leaves per primitive)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        depth = int(rng.integers(7, 11))
        target = math.exp(rng.uniform(math.log(min_leaves), math.log(max_leaves)))
        n_prim = int(np.clip(round(target / (1300.0 * 4.0 ** (depth - 6))), 1, 256))
        n_box = n_prim // 3
        out.append(make_scene(rng, depth, n_prim - n_box, n_box))
    return out
