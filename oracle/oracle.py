"""SVLF CPU oracle in float64. TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module. It shares no code with the CUDA path and
imports nothing from the package.

Every function computes a plain definition from the paper, widened from the
float32 inputs to float64:

* traversal: ``svlf_oracle.c`` (slab test per voxel, Sec. 4.2; hits in the
  order of intersection along the ray, Sec. 4.3);
* ray parameterisation r = [p~1 | p~2] from the ray's intersections with the
  voxel's minimum bounding sphere, taken relative to the voxel centre and
  scaled to unit norm (Sec. 4.1, "Ray parameterization"), or, under the
  other reading of its "voxel origin", the ray's entry and exit points of
  the voxel box in voxel-local coordinates (aabb_params);
* the per-sample network: ReLU hidden layers, colour through a sigmoid and
  optical thickness through a ReLU (Sec. 4.5, "Architecture"); the single
  network over [feature | ray direction | r] is the workload's form of the
  paper's decoders (Eq. 1-2);
* compositing c(r) = sum_i T_i (1 - exp(-tau_i)) c_i with
  T_i = prod_{j<i} exp(-tau_j) (Sec. 4.3, Eq. 3); alpha = 1 - exp(-tau) is the
  opacity (Sec. 4, footnote on optical thickness). The transmittance left
  after the K-th hit multiplies a background colour, and depth is the
  weight-averaged segment midpoint;
* the training loss (L2 colour + 0.1 L1 depth, mean over rays), its adjoint
  derived by hand from Eq. 3, and Adam (Sec. 4.5, "Training"; Kingma & Ba).

Pins that tie this oracle to something other than itself live in
``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libsvlf_oracle.so")

NEAR_DEGENERATE = 1e-6  # gap (in t) between crossings below which a ray may be flagged


# ----------------------------------------------------------------------------
# C traversal library
# ----------------------------------------------------------------------------
def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "svlf_oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        os.makedirs(os.path.dirname(_SO), exist_ok=True)
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        L.oracle_leaf_codes.restype = i64
        L.oracle_leaf_codes.argtypes = [vp, i64, i32, vp]
        L.oracle_morton.restype = ctypes.c_uint64
        L.oracle_morton.argtypes = [i64, i64, i64, i32]
        L.oracle_trace_brute.restype = None
        L.oracle_trace_brute.argtypes = [vp, i64, i32, vp, i64, i32, vp, vp, vp, vp]
        L.oracle_trace_dda.restype = None
        L.oracle_trace_dda.argtypes = [vp, i64, i32, vp, i64, i32, vp, vp, vp, vp, vp, vp, vp, vp]
        L.oracle_set_threads.restype = None
        L.oracle_set_threads.argtypes = [i32]
        L.oracle_max_threads.restype = i32
        L.oracle_max_threads.argtypes = []
        _lib = L
    return _lib


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


@dataclass
class Octree:
    """The oracle's octree: the sorted Morton codes of the occupied leaves."""
    depth: int
    codes: np.ndarray  # uint64, ascending; leaf rank = index

    @property
    def n_leaves(self) -> int:
        return int(self.codes.shape[0])

    def leaf_ijk(self) -> np.ndarray:
        c = self.codes
        out = np.zeros((c.shape[0], 3), dtype=np.int64)
        for b in range(self.depth):
            for a in range(3):
                out[:, a] |= ((c >> np.uint64(3 * b + a)) & np.uint64(1)).astype(np.int64) << b
        return out


def build_octree(leaf_ijk: np.ndarray, depth: int) -> Octree:
    ijk = np.ascontiguousarray(leaf_ijk, dtype=np.int32).reshape(-1, 3)
    codes = np.zeros(max(ijk.shape[0], 1), dtype=np.uint64)
    n = lib().oracle_leaf_codes(_p(ijk), ijk.shape[0], depth, _p(codes))
    if n < 0:
        raise ValueError("leaf coordinate outside [0, 2^depth)")
    return Octree(depth, codes[:n].copy())


@dataclass
class Hits:
    rank: np.ndarray     # (N, K) int32, -1 = empty
    t_in: np.ndarray     # (N, K) float64
    t_out: np.ndarray    # (N, K) float64
    n: np.ndarray        # (N,) int32
    t_start: Optional[np.ndarray] = None  # (N,) root entry (-1 = miss)
    t_end: Optional[np.ndarray] = None    # (N,) where inspection stopped
    walked: Optional[np.ndarray] = None   # (N,) voxels walked by the DDA
    degenerate: Optional[np.ndarray] = None  # (N,) bool: near-degenerate ray


def trace(tree: Octree, rays: np.ndarray, K: int, mode: str = "dda") -> Hits:
    """First K hit leaves per ray, in ascending t_in."""
    rays = np.ascontiguousarray(rays, dtype=np.float32).reshape(-1, 6)
    N = rays.shape[0]
    rank = np.empty((N, K), dtype=np.int32)
    tin = np.empty((N, K), dtype=np.float64)
    tout = np.empty((N, K), dtype=np.float64)
    nh = np.empty(N, dtype=np.int32)
    codes = tree.codes if tree.n_leaves else np.zeros(1, dtype=np.uint64)
    if mode == "brute":
        lib().oracle_trace_brute(_p(codes), tree.n_leaves, tree.depth, _p(rays), N, K,
                                 _p(rank), _p(tin), _p(tout), _p(nh))
        return Hits(rank, tin, tout, nh)
    ts = np.empty(N, dtype=np.float64)
    te = np.empty(N, dtype=np.float64)
    walked = np.empty(N, dtype=np.int64)
    deg = np.empty(N, dtype=np.int32)
    lib().oracle_trace_dda(_p(codes), tree.n_leaves, tree.depth, _p(rays), N, K,
                           _p(rank), _p(tin), _p(tout), _p(nh), _p(ts), _p(te), _p(walked), _p(deg))
    return Hits(rank, tin, tout, nh, ts, te, walked, deg.astype(bool))


# ----------------------------------------------------------------------------
# Ray parameterisation (Sec. 4.1)
# ----------------------------------------------------------------------------
def voxel_centre_radius(ijk: np.ndarray, depth: int):
    h = 2.0 ** -depth
    return (ijk.astype(np.float64) + 0.5) * h, 0.5 * np.sqrt(3.0) * h


def sphere_params(o: np.ndarray, d: np.ndarray, c: np.ndarray, R: float):
    """r = [p~1 | p~2]: the ray's entry and exit points on the sphere of
    radius R about c, relative to c, scaled to unit norm. Rows are samples.

    The roots of |o + t d - c|^2 = R^2 are found from the foot of the
    perpendicular t_f = -d.(o-c)/|d|^2 and the half chord
    sqrt((R^2 - |q|^2)/|d|^2), q = (o - c) + t_f d, which avoids the
    cancellation of the textbook form; p = o + t d.
    """
    oc = o - c
    dd = np.sum(d * d, axis=1)
    tf = -np.sum(d * oc, axis=1) / dd
    q = oc + tf[:, None] * d
    half = np.sqrt(np.maximum(R * R - np.sum(q * q, axis=1), 0.0) / dd)
    t1, t2 = tf - half, tf + half
    p1 = o + t1[:, None] * d - c
    p2 = o + t2[:, None] * d - c
    p1 /= np.linalg.norm(p1, axis=1, keepdims=True)
    p2 /= np.linalg.norm(p2, axis=1, keepdims=True)
    return p1, p2


# ----------------------------------------------------------------------------
# Per-sample network
# ----------------------------------------------------------------------------
def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float64 values to the nearest bfloat16 (ties to even), via the
    float32 value's bit pattern."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def fp16_round(x: np.ndarray) -> np.ndarray:
    """Round float64 values to the nearest IEEE half (ties to even)."""
    return np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)


def _rounder(lowp):
    if lowp in (None, False):
        return None
    if lowp in (True, "bf16"):
        return bf16_round
    if lowp == "fp16":
        return fp16_round
    raise ValueError(lowp)


def split_params(flat: np.ndarray, dims: Sequence[Tuple[int, int]]):
    out, off = [], 0
    flat = np.asarray(flat, dtype=np.float64)
    for o, i in dims:
        W = flat[off:off + o * i].reshape(o, i)
        off += o * i
        b = flat[off:off + o]
        off += o
        out.append((W, b))
    return out


def layer_dims(feat_dim: int, hidden: int, n_hidden: int, out_dim: int = 4):
    dims = [feat_dim + 9] + [hidden] * n_hidden + [out_dim]
    return [(dims[i + 1], dims[i]) for i in range(len(dims) - 1)]


def mlp_forward(h0: np.ndarray, layers, bf16=False):
    """Returns (inputs of every layer, pre-activations of every layer).
    Hidden layers are ReLU; the last layer is linear. With bf16 = True/"bf16"
    (or "fp16") each layer's input activations and weights are rounded to that
    16-bit format first and the products and sums stay in float64 (the biases
    are not rounded)."""
    rnd = _rounder(bf16)
    xs, pres = [], []
    x = h0
    for li, (W, b) in enumerate(layers):
        xin = rnd(x) if rnd else x
        Wl = rnd(W) if rnd else W
        pre = xin @ Wl.T + b
        xs.append(x)
        pres.append(pre)
        x = np.maximum(pre, 0.0) if li + 1 < len(layers) else pre
    return xs, pres


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


# ----------------------------------------------------------------------------
# Rendering
# ----------------------------------------------------------------------------
@dataclass
class Render:
    rgb: np.ndarray     # (N, 3)
    depth: np.ndarray   # (N,)
    hits: Hits
    ray_of: np.ndarray  # (S,) ray index of each sample (samples grouped by ray, in hit order)
    slot: np.ndarray    # (S,) hit index within its ray
    h0: np.ndarray      # (S, in_dim) network inputs
    xs: list
    pres: list
    out: np.ndarray     # (S, 4) raw network outputs
    colour: np.ndarray  # (S, 3) sigmoid(out[:, :3])
    tau: np.ndarray     # (S,) relu(out[:, 3])
    tmid: np.ndarray    # (S,)
    T: np.ndarray       # (N, K+1) transmittance before each hit; T[:, n] is the residual
    w: np.ndarray       # (N, K) compositing weights T_i * alpha_i


def aabb_params(o: np.ndarray, d: np.ndarray, t_in: np.ndarray, t_out: np.ndarray, c: np.ndarray, h: float):
    """The other reading of "voxel origin": r = [x~1 | x~2], the ray's entry
    and exit points of the voxel box itself, x_i = o + t_i d with (t_in,
    t_out) the slab segment (entry clipped at t = 0), in voxel-local
    coordinates (x_i - c) / (h / 2), each component in [-1, 1]."""
    x1 = o + t_in[:, None] * d
    x2 = o + t_out[:, None] * d
    return (x1 - c) / (0.5 * h), (x2 - c) / (0.5 * h)


def sample_inputs(tree: Octree, rays: np.ndarray, hits: Hits, features: np.ndarray, rparam: str = "sphere"):
    """Network inputs h0 = [z | d | p~1 | p~2] of every hit, samples grouped by
    ray in hit order. rparam = "sphere": the bounding-sphere parameterisation
    (Sec. 4.1); "aabb": the voxel-box reading (aabb_params)."""
    N, K = hits.rank.shape
    ray_of, slot = np.nonzero(hits.rank >= 0)
    rank = hits.rank[ray_of, slot]
    o = rays[ray_of, :3].astype(np.float64)
    d = rays[ray_of, 3:].astype(np.float64)
    ijk = tree.leaf_ijk()[rank]
    c, R = voxel_centre_radius(ijk, tree.depth)
    if rparam == "sphere":
        p1, p2 = sphere_params(o, d, c, R)
    elif rparam == "aabb":
        p1, p2 = aabb_params(o, d, hits.t_in[ray_of, slot], hits.t_out[ray_of, slot], c, 2.0 ** -tree.depth)
    else:
        raise ValueError(rparam)
    z = np.asarray(features)[rank].astype(np.float64)
    h0 = np.concatenate([z, d, p1, p2], axis=1)
    tmid = 0.5 * (hits.t_in[ray_of, slot] + hits.t_out[ray_of, slot])
    return ray_of, slot, rank, h0, tmid


def composite(N: int, K: int, ray_of, slot, colour, tau, tmid, bg):
    """Eq. 3 over the first K hits, plus the residual transmittance times bg."""
    tau_k = np.zeros((N, K))
    col_k = np.zeros((N, K, 3))
    tm_k = np.zeros((N, K))
    tau_k[ray_of, slot] = tau
    col_k[ray_of, slot] = colour
    tm_k[ray_of, slot] = tmid
    T = np.ones((N, K + 1))
    for i in range(K):
        T[:, i + 1] = T[:, i] * np.exp(-tau_k[:, i])
    w = T[:, :K] * (1.0 - np.exp(-tau_k))
    rgb = np.sum(w[:, :, None] * col_k, axis=1) + T[:, K:K + 1] * np.asarray(bg, dtype=np.float64)[None, :]
    depth = np.sum(w * tm_k, axis=1)
    return rgb, depth, T, w


def render(tree: Octree, features: np.ndarray, params: np.ndarray, dims, rays: np.ndarray,
           K: int, bg=(0.0, 0.0, 0.0), bf16=False, hits: Optional[Hits] = None,
           feat_bf16_storage: bool = False, rparam: str = "sphere") -> Render:
    rays = np.ascontiguousarray(rays, dtype=np.float32).reshape(-1, 6)
    N = rays.shape[0]
    if hits is None:
        hits = trace(tree, rays, K)
    feats = np.asarray(features, dtype=np.float32)
    ray_of, slot, rank, h0, tmid = sample_inputs(tree, rays, hits, feats, rparam)
    layers = split_params(params, dims)
    xs, pres = mlp_forward(h0, layers, bf16=bf16)
    out = pres[-1]
    colour = sigmoid(out[:, :3])
    tau = np.maximum(out[:, 3], 0.0)
    rgb, depth, T, w = composite(N, K, ray_of, slot, colour, tau, tmid, bg)
    return Render(rgb, depth, hits, ray_of, slot, h0, xs, pres, out, colour, tau, tmid, T, w)


# ----------------------------------------------------------------------------
# Training: loss, adjoint, finite differences, Adam
# ----------------------------------------------------------------------------
DEPTH_WEIGHT = 0.1


def loss(rgb, depth, rgb_t, depth_t, mask, norm=None) -> float:
    """Mean over rays of sum_ch (C - C*)^2 + 0.1 * m * |D - D*|. With `norm`
    the sum is divided by norm instead of the ray count: the share of one
    shard of a batch of `norm` rays, whose shares sum to the batch's mean."""
    N = rgb.shape[0] if norm is None else norm
    e = np.sum((rgb - rgb_t) ** 2) + DEPTH_WEIGHT * np.sum(mask * np.abs(depth - depth_t))
    return float(e / N)


def backward(tree: Octree, r: Render, params: np.ndarray, dims, rgb_t, depth_t, mask, bg,
             n_leaves: int, feat_dim: int, bf16=False, norm=None):
    """Hand-derived adjoint of loss(render(...), norm=norm). Returns
    (dL/dfeatures (dense, n_leaves x F), dL/dparams (flat, same layout as
    params), dC, dD)."""
    N, K = r.hits.rank.shape
    M = N if norm is None else norm
    bg = np.asarray(bg, dtype=np.float64)
    dC = 2.0 * (r.rgb - rgb_t) / M
    dD = DEPTH_WEIGHT * mask * np.sign(r.depth - depth_t) / M
    # per-slot arrays
    col_k = np.zeros((N, K, 3))
    tm_k = np.zeros((N, K))
    col_k[r.ray_of, r.slot] = r.colour
    tm_k[r.ray_of, r.slot] = r.tmid
    wc = r.w[:, :, None] * col_k
    wt = r.w * tm_k
    # S_i = sum_{j>i} w_j c_j + T_{K} bg ; U_i = sum_{j>i} w_j t_j  (empty slots have w = 0)
    S = np.zeros((N, K, 3))
    U = np.zeros((N, K))
    accS = r.T[:, K:K + 1] * bg[None, :]
    accU = np.zeros(N)
    for i in range(K - 1, -1, -1):
        S[:, i] = accS
        U[:, i] = accU
        accS = accS + wc[:, i]
        accU = accU + wt[:, i]
    Tn = r.T[:, 1:]  # T_{i+1}
    dcol = r.w[:, :, None] * dC[:, None, :]
    dtau = np.sum(dC[:, None, :] * (Tn[:, :, None] * col_k - S), axis=2) + dD[:, None] * (Tn * tm_k - U)
    # through the output activations
    dout = np.zeros_like(r.out)
    dout[:, :3] = dcol[r.ray_of, r.slot] * r.colour * (1.0 - r.colour)
    dout[:, 3] = dtau[r.ray_of, r.slot] * (r.out[:, 3] > 0)
    # through the network
    rnd = _rounder(bf16)
    layers = split_params(params, dims)
    grads = []
    delta = dout
    for li in range(len(layers) - 1, -1, -1):
        W, b = layers[li]
        xin = rnd(r.xs[li]) if rnd else r.xs[li]
        Wl = rnd(W) if rnd else W
        dW = delta.T @ xin
        db = delta.sum(axis=0)
        grads.append((dW, db))
        dx = delta @ Wl
        if li > 0:
            delta = dx * (r.pres[li - 1] > 0)
        else:
            dz = dx[:, :feat_dim]
    grads.reverse()
    flat = np.concatenate([np.concatenate([g[0].reshape(-1), g[1]]) for g in grads])
    dfeat = np.zeros((n_leaves, feat_dim))
    rank = r.hits.rank[r.ray_of, r.slot]
    np.add.at(dfeat, rank, dz)
    return dfeat, flat, dC, dD


def kink_pattern(r: Render, depth_t, mask):
    """Everything whose flip makes the loss non-differentiable: every hidden
    ReLU, the optical-thickness ReLU and the sign of D - D* on masked rays."""
    parts = [(p > 0) for p in r.pres[:-1]]
    parts.append(r.out[:, 3] > 0)
    parts.append(np.sign(r.depth - depth_t) * (mask > 0))
    return parts


def same_pattern(a, b) -> bool:
    return all(np.array_equal(x, y) for x, y in zip(a, b))


def adam(params, grads, m, v, step: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One bias-corrected Adam step (Kingma & Ba, Algorithm 1). Returns the new
    (params, m, v)."""
    p = np.asarray(params, dtype=np.float64)
    g = np.asarray(grads, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v
