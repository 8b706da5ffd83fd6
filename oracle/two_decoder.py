"""The paper's two-decoder SVLF in float64. TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import this module. It shares no code with the CUDA path.

Definitions followed (arXiv 2205.07058):

* Sec. 4.1 "Scene volume": every octree vertex (corner of a leaf voxel) holds
  one feature vector, shared by the voxels that meet there; a point p inside
  voxel v gets psi(p; Z), the trilinear interpolation of v's eight corner
  features.
* Sec. 4.2: the features split into Z^T (optical thickness) and Z^C (colour).
  For a hit voxel with intersection points x1 (entry) and x2 (exit),
  tau, eta = F^T(r, [psi(x1; Z^T) | psi(x2; Z^T)]) (Eq. 1), the surface point
  is x_s = eta x1 + (1 - eta) x2, and c = F^C(r, psi(x_s; Z^C)) (Eq. 2);
  r = [p~1 | p~2] is the bounding-sphere parameterisation of Sec. 4.1.
* Sec. 4.5 "Architecture": ReLU MLPs; ReLU on tau, sigmoid on eta and c.
* Sec. 4.3, Eq. 3: compositing over the hits in order along the ray.

Readings taken where the paper is silent: the network inputs are ordered
features first, [psi(x1) | psi(x2) | r] and [psi(x_s) | r] (the order of a
first layer's inputs is a permutation of its weight columns; features first
keeps feature groups aligned as in the single-network form [z | d | r]); the
vertex ids are the ranks of the corner lattice points sorted by
their Morton code (corner (a, b, c) of leaf (i, j, k) is (i+a, j+b, k+c), slot
a + 2b + 4c); trilinear weights use the point's position inside the voxel
clamped to [0, 1]^3; the depth of a hit is the ray parameter of x_s,
t_s = eta t_in + (1 - eta) t_out, and the ray's depth is sum_i w_i t_s,i.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional, Sequence, Tuple

import numpy as np

from . import oracle as O


# ----------------------------------------------------------------------------
# Vertex table (Sec. 4.1)
# ----------------------------------------------------------------------------
def _morton3(ijk: np.ndarray, bits: int) -> np.ndarray:
    code = np.zeros(ijk.shape[0], dtype=np.uint64)
    for b in range(bits):
        for a in range(3):
            code |= ((ijk[:, a].astype(np.uint64) >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + a)
    return code


CORNERS = np.array([[a, b, c] for c in (0, 1) for b in (0, 1) for a in (0, 1)], dtype=np.int64)  # slot a+2b+4c


@dataclass
class VertexTable:
    leaf_vertices: np.ndarray  # (n_leaves, 8) int64: vertex id of corner slot a + 2b + 4c
    vertex_ijk: np.ndarray     # (n_vertices, 3) int64 lattice coordinates (0 .. 2^L)

    @property
    def n_vertices(self) -> int:
        return int(self.vertex_ijk.shape[0])


def vertex_table(tree: O.Octree) -> VertexTable:
    """Every corner of every leaf, de-duplicated; ids in Morton order of the
    corner coordinates (L + 1 bits per axis)."""
    ijk = tree.leaf_ijk()
    corners = (ijk[:, None, :] + CORNERS[None, :, :]).reshape(-1, 3)
    codes = _morton3(corners, tree.depth + 1)
    uniq, inverse = np.unique(codes, return_inverse=True)
    first = np.zeros(uniq.shape[0], dtype=np.int64)
    first[inverse] = np.arange(codes.shape[0])
    return VertexTable(inverse.reshape(-1, 8).astype(np.int64), corners[first])


def trilinear_weights(p: np.ndarray, ijk: np.ndarray, depth: int) -> np.ndarray:
    """(S, 8) weights of the eight corners of voxel ijk for points p (S, 3)."""
    u = np.clip(p * (2.0 ** depth) - ijk.astype(np.float64), 0.0, 1.0)
    w = np.ones((p.shape[0], 8))
    for s, (a, b, c) in enumerate(CORNERS):
        w[:, s] = ((u[:, 0] if a else 1.0 - u[:, 0]) * (u[:, 1] if b else 1.0 - u[:, 1]) *
                   (u[:, 2] if c else 1.0 - u[:, 2]))
    return w


def psi(p: np.ndarray, rank: np.ndarray, tree: O.Octree, vt: VertexTable, Z: np.ndarray) -> np.ndarray:
    """Trilinear interpolation of the corner features of leaf `rank` at p."""
    ijk = tree.leaf_ijk()[rank]
    w = trilinear_weights(p, ijk, tree.depth)
    Zc = np.asarray(Z, dtype=np.float64)[vt.leaf_vertices[rank]]  # (S, 8, F)
    return np.einsum("sv,svf->sf", w, Zc)


# ----------------------------------------------------------------------------
# Networks and rendering (Sec. 4.2, 4.3, 4.5)
# ----------------------------------------------------------------------------
def dims_t(feat_t: int, hidden: int, n_hidden: int):
    """F^T: [psi(x1) | psi(x2) | p~1 | p~2] -> (tau_pre, eta_pre)."""
    d = [6 + 2 * feat_t] + [hidden] * n_hidden + [2]
    return [(d[i + 1], d[i]) for i in range(len(d) - 1)]


def dims_c(feat_c: int, hidden: int, n_hidden: int):
    """F^C: [psi(x_s) | p~1 | p~2] -> colour pre-activations."""
    d = [6 + feat_c] + [hidden] * n_hidden + [3]
    return [(d[i + 1], d[i]) for i in range(len(d) - 1)]


@dataclass
class Render2:
    rgb: np.ndarray
    depth: np.ndarray
    hits: O.Hits
    ray_of: np.ndarray
    slot: np.ndarray
    tau: np.ndarray
    eta: np.ndarray
    colour: np.ndarray
    t_s: np.ndarray
    x1: np.ndarray
    x2: np.ndarray
    x_s: np.ndarray
    h_t: np.ndarray  # F^T inputs
    h_c: np.ndarray  # F^C inputs
    w: np.ndarray    # compositing weights (N, K)
    T: np.ndarray    # transmittance (N, K + 1)
    rank: np.ndarray
    t_in: np.ndarray
    t_out: np.ndarray
    xs_t: list       # every F^T layer's input
    pres_t: list     # every F^T layer's pre-activation
    xs_c: list
    pres_c: list
    dirs: np.ndarray  # ray direction of every sample


@dataclass
class Eval2:
    """The two decoders on a list of (ray, voxel, segment) samples."""
    rank: np.ndarray
    t_in: np.ndarray
    t_out: np.ndarray
    dirs: np.ndarray
    x1: np.ndarray
    x2: np.ndarray
    tau: np.ndarray
    eta: np.ndarray
    x_s: np.ndarray
    t_s: np.ndarray
    colour: np.ndarray
    h_t: np.ndarray
    h_c: np.ndarray
    xs_t: list
    pres_t: list
    xs_c: list
    pres_c: list


def eval_samples(tree: O.Octree, vt: VertexTable, z_t, z_c, params_t, params_c, d_t, d_c, o, d, rank, t_in,
                 t_out, lowp=False) -> Eval2:
    """Eq. 1-2 on samples: ray origin o and direction d (S x 3), hit leaf rank,
    segment [t_in, t_out]."""
    c, R = O.voxel_centre_radius(tree.leaf_ijk()[rank], tree.depth)
    p1, p2 = O.sphere_params(o, d, c, R)
    x1 = o + t_in[:, None] * d
    x2 = o + t_out[:, None] * d
    h_t = np.concatenate([psi(x1, rank, tree, vt, z_t), psi(x2, rank, tree, vt, z_t), p1, p2], axis=1)
    xs_t, pres_t = O.mlp_forward(h_t, O.split_params(params_t, d_t), bf16=lowp)
    tau = np.maximum(pres_t[-1][:, 0], 0.0)
    eta = O.sigmoid(pres_t[-1][:, 1])
    x_s = eta[:, None] * x1 + (1.0 - eta[:, None]) * x2
    t_s = eta * t_in + (1.0 - eta) * t_out
    h_c = np.concatenate([psi(x_s, rank, tree, vt, z_c), p1, p2], axis=1)
    xs_c, pres_c = O.mlp_forward(h_c, O.split_params(params_c, d_c), bf16=lowp)
    colour = O.sigmoid(pres_c[-1])
    return Eval2(rank, t_in, t_out, d, x1, x2, tau, eta, x_s, t_s, colour, h_t, h_c, xs_t, pres_t, xs_c, pres_c)


def render2(tree: O.Octree, vt: VertexTable, z_t: np.ndarray, z_c: np.ndarray, params_t: np.ndarray,
            params_c: np.ndarray, d_t, d_c, rays: np.ndarray, K: int, bg=(0.0, 0.0, 0.0), lowp=False,
            hits: Optional[O.Hits] = None) -> Render2:
    """Two-decoder render of every ray. lowp = "bf16" / "fp16" rounds each
    layer's inputs and weights to that format (products and sums in float64)."""
    rays = np.ascontiguousarray(rays, dtype=np.float32).reshape(-1, 6)
    N = rays.shape[0]
    if hits is None:
        hits = O.trace(tree, rays, K)
    ray_of, slot = np.nonzero(hits.rank >= 0)
    rank = hits.rank[ray_of, slot]
    o = rays[ray_of, :3].astype(np.float64)
    d = rays[ray_of, 3:].astype(np.float64)
    e = eval_samples(tree, vt, z_t, z_c, params_t, params_c, d_t, d_c, o, d, rank, hits.t_in[ray_of, slot],
                     hits.t_out[ray_of, slot], lowp)
    rgb, depth, T, w = O.composite(N, K, ray_of, slot, e.colour, e.tau, e.t_s, bg)
    return Render2(rgb, depth, hits, ray_of, slot, e.tau, e.eta, e.colour, e.t_s, e.x1, e.x2, e.x_s, e.h_t, e.h_c,
                   w, T, rank, e.t_in, e.t_out, e.xs_t, e.pres_t, e.xs_c, e.pres_c, d)


# ----------------------------------------------------------------------------
# Adjoint (derived by hand from the definitions above, Eq. 3 and the loss)
# ----------------------------------------------------------------------------
def trilinear_weight_gradients(p: np.ndarray, ijk: np.ndarray, depth: int) -> np.ndarray:
    """(S, 8, 3): d w_corner / d p inside the voxel (0 along an axis where the
    position is clamped)."""
    n = 2.0 ** depth
    u_raw = p * n - ijk.astype(np.float64)
    u = np.clip(u_raw, 0.0, 1.0)
    inside = (u_raw > 0.0) & (u_raw < 1.0)
    g = np.zeros((p.shape[0], 8, 3))
    for s, corner in enumerate(CORNERS):
        f = [u[:, a] if corner[a] else 1.0 - u[:, a] for a in range(3)]
        for a in range(3):
            sign = 1.0 if corner[a] else -1.0
            others = f[(a + 1) % 3] * f[(a + 2) % 3]
            g[:, s, a] = np.where(inside[:, a], sign * others * n, 0.0)
    return g


def _mlp_backward(delta, xs, pres, layers, lowp):
    """Returns (flat dparams, dL/d(network input))."""
    rnd = O._rounder(lowp)
    grads = []
    dx = None
    for li in range(len(layers) - 1, -1, -1):
        W, b = layers[li]
        xin = rnd(xs[li]) if rnd else xs[li]
        Wl = rnd(W) if rnd else W
        grads.append((delta.T @ xin, delta.sum(axis=0)))
        dx = delta @ Wl
        if li > 0:
            delta = dx * (pres[li - 1] > 0)
    grads.reverse()
    return np.concatenate([np.concatenate([g[0].reshape(-1), g[1]]) for g in grads]), dx


def adjoint_core(tree: O.Octree, vt: VertexTable, e, z_c, params_t, params_c, d_t, d_c, dcol, dtau, dts,
                 deta_direct, feat_t: int, feat_c: int, lowp=False):
    """Adjoint of the two decoders on samples `e` (Eval2 or Render2) given the
    loss's gradients w.r.t. every sample's colour (S x 3), tau, depth
    parameter t_s and (directly) eta. Returns (dZ^T, dZ^C, dparams_t, dparams_c)."""
    ijk = tree.leaf_ijk()[e.rank]
    dparams_c, dhc = _mlp_backward(dcol * e.colour * (1.0 - e.colour), e.xs_c, e.pres_c,
                                   O.split_params(params_c, d_c), lowp)
    dpsi_c = dhc[:, :feat_c]
    wgt_s = trilinear_weights(e.x_s, ijk, tree.depth)
    dzc = np.zeros((vt.n_vertices, feat_c))
    np.add.at(dzc, vt.leaf_vertices[e.rank].reshape(-1),
              (wgt_s[:, :, None] * dpsi_c[:, None, :]).reshape(-1, feat_c))
    # through x_s = o + t_s d: d psi / d x_s from the corner weights' gradients
    gw = trilinear_weight_gradients(e.x_s, ijk, tree.depth)                  # (S, 8, 3)
    zdot = np.einsum("svf,sf->sv", np.asarray(z_c, np.float64)[vt.leaf_vertices[e.rank]], dpsi_c)
    dxs = np.einsum("sv,sva->sa", zdot, gw)
    dts = dts + np.einsum("sa,sa->s", dxs, e.dirs)  # x_s = o + t_s d
    deta = dts * (e.t_in - e.t_out) + deta_direct  # t_s = eta t_in + (1 - eta) t_out
    delta_t = np.stack([dtau * (e.pres_t[-1][:, 0] > 0), deta * e.eta * (1.0 - e.eta)], axis=1)
    dparams_t, dht = _mlp_backward(delta_t, e.xs_t, e.pres_t, O.split_params(params_t, d_t), lowp)
    w1 = trilinear_weights(e.x1, ijk, tree.depth)
    w2 = trilinear_weights(e.x2, ijk, tree.depth)
    contrib = w1[:, :, None] * dht[:, None, :feat_t] + w2[:, :, None] * dht[:, None, feat_t:2 * feat_t]
    dzt = np.zeros((vt.n_vertices, feat_t))
    np.add.at(dzt, vt.leaf_vertices[e.rank].reshape(-1), contrib.reshape(-1, feat_t))
    return dzt, dzc, dparams_t, dparams_c


def backward2(tree: O.Octree, vt: VertexTable, r: Render2, z_c: np.ndarray, params_t, params_c, d_t, d_c,
              rgb_t, depth_t, mask, bg, feat_t: int, feat_c: int, lowp=False, deta_direct=None):
    """Gradient of loss(render2(...)) (the loss of the single-network form:
    mean over rays of the squared colour error + 0.1 masked |D - D*|), plus
    an optional direct gradient w.r.t. each sample's eta.
    Returns (dZ^T (n_vertices x feat_t), dZ^C, dparams_t, dparams_c, dC, dD)."""
    N, K = r.hits.rank.shape
    bg = np.asarray(bg, dtype=np.float64)
    dC = 2.0 * (r.rgb - rgb_t) / N
    dD = O.DEPTH_WEIGHT * mask * np.sign(r.depth - depth_t) / N
    col_k = np.zeros((N, K, 3))
    ts_k = np.zeros((N, K))
    col_k[r.ray_of, r.slot] = r.colour
    ts_k[r.ray_of, r.slot] = r.t_s
    wc = r.w[:, :, None] * col_k
    wt = r.w * ts_k
    S = np.zeros((N, K, 3))
    U = np.zeros((N, K))
    accS = r.T[:, K:K + 1] * bg[None, :]
    accU = np.zeros(N)
    for i in range(K - 1, -1, -1):
        S[:, i] = accS
        U[:, i] = accU
        accS = accS + wc[:, i]
        accU = accU + wt[:, i]
    Tn = r.T[:, 1:]
    dcol = (r.w[:, :, None] * dC[:, None, :])[r.ray_of, r.slot]
    dtau = (np.sum(dC[:, None, :] * (Tn[:, :, None] * col_k - S), axis=2) + dD[:, None] * (Tn * ts_k - U))[r.ray_of, r.slot]
    dts = (r.w * dD[:, None])[r.ray_of, r.slot]  # D = sum_i w_i t_s,i
    dd = np.zeros(r.rank.shape[0]) if deta_direct is None else deta_direct
    dzt, dzc, dpt, dpc = adjoint_core(tree, vt, r, z_c, params_t, params_c, d_t, d_c, dcol, dtau, dts, dd,
                                      feat_t, feat_c, lowp)
    return dzt, dzc, dpt, dpc, dC, dD


def kink_pattern2(r: Render2, depth_t, mask):
    """Every hidden ReLU of both networks, the tau ReLU and the sign of D - D*."""
    parts = [(p > 0) for p in r.pres_t[:-1]] + [(p > 0) for p in r.pres_c[:-1]]
    parts.append(r.pres_t[-1][:, 0] > 0)
    parts.append(np.sign(r.depth - depth_t) * (mask > 0))
    return parts


# ----------------------------------------------------------------------------
# Staged training (Sec. 4.4, Eq. 4)
# ----------------------------------------------------------------------------
def eta_target(t_in, t_out, t_star):
    """Within-voxel depth of the true surface point o + t* d on the segment
    [t_in, t_out]: x* = eta x1 + (1 - eta) x2 (clamped to [0, 1])."""
    return np.clip((t_out - t_star) / (t_out - t_in), 0.0, 1.0)


@dataclass
class SurfaceSamples:
    ray: np.ndarray
    rank: np.ndarray
    t_in: np.ndarray
    t_out: np.ndarray
    eta_gt: np.ndarray


def surface_samples(tree: O.Octree, rays: np.ndarray, depth_t: np.ndarray, mask: np.ndarray) -> SurfaceSamples:
    """Stage 1 ("voxel training"): for each ray with a known surface depth D*,
    the voxel containing the surface point x* = o + D* d (floor of x* 2^L),
    kept when it is a leaf and the ray's segment through it has positive
    length."""
    rays = np.asarray(rays, dtype=np.float32).reshape(-1, 6)
    n = 1 << tree.depth
    sel = np.nonzero((np.asarray(mask) > 0) & np.isfinite(depth_t))[0]
    o = rays[sel, :3].astype(np.float64)
    d = rays[sel, 3:].astype(np.float64)
    t_star = np.asarray(depth_t, np.float64)[sel]
    xs = o + t_star[:, None] * d
    ijk = np.clip(np.floor(xs * n).astype(np.int64), 0, n - 1)
    leaves = tree.leaf_ijk()
    lookup = {tuple(v): i for i, v in enumerate(leaves)}
    rank = np.array([lookup.get(tuple(v), -1) for v in ijk], dtype=np.int64)
    h = 1.0 / n
    lo = ijk * h
    with np.errstate(divide="ignore", invalid="ignore"):
        ta = (lo - o) / d
        tb = (lo + h - o) / d
    ta = np.where(d == 0, -np.inf, ta)
    tb = np.where(d == 0, np.inf, tb)
    t_in = np.maximum(np.max(np.minimum(ta, tb), axis=1), 0.0)
    t_out = np.min(np.maximum(ta, tb), axis=1)
    keep = (rank >= 0) & (t_out > t_in)
    return SurfaceSamples(sel[keep], rank[keep], t_in[keep], t_out[keep],
                          eta_target(t_in[keep], t_out[keep], t_star[keep]))


def surface_loss(tree, vt, z_t, z_c, params_t, params_c, d_t, d_c, rays, rgb_t, depth_t, mask, lam_eta, lam_tau,
                 feat_t, feat_c, lowp=False, with_grad=True):
    """Eq. 4 on the surface voxels of a batch of N rays, divided by N:
    (1/N) sum_v |c_v - c*|^2 + lam_eta (eta_v - eta*)^2 + lam_tau exp(-tau_v)^2.
    Returns (loss, samples, eval, grads or None)."""
    rays = np.asarray(rays, dtype=np.float32).reshape(-1, 6)
    N = rays.shape[0]
    ss = surface_samples(tree, rays, depth_t, mask)
    o = rays[ss.ray, :3].astype(np.float64)
    d = rays[ss.ray, 3:].astype(np.float64)
    e = eval_samples(tree, vt, z_t, z_c, params_t, params_c, d_t, d_c, o, d, ss.rank, ss.t_in, ss.t_out, lowp)
    ct = np.asarray(rgb_t, np.float64)[ss.ray]
    et = np.exp(-e.tau)
    L = float(np.sum(np.sum((e.colour - ct) ** 2, axis=1) + lam_eta * (e.eta - ss.eta_gt) ** 2
                     + lam_tau * et * et) / N)
    if not with_grad:
        return L, ss, e, None
    dcol = 2.0 * (e.colour - ct) / N
    dtau = -2.0 * lam_tau * et * et / N
    deta = 2.0 * lam_eta * (e.eta - ss.eta_gt) / N
    grads = adjoint_core(tree, vt, e, z_c, params_t, params_c, d_t, d_c, dcol, dtau, np.zeros(ss.ray.size), deta,
                         feat_t, feat_c, lowp)
    return L, ss, e, grads


def eta_term(r: Render2, depth_t, mask, lam_eta):
    """Stages 2-3: lam_eta (eta_v - eta*)^2 / N over each ray's surface voxel
    among its hits (the hit whose segment contains D*). Returns (loss term,
    per-sample direct dL/deta)."""
    N = r.hits.rank.shape[0]
    t_star = np.asarray(depth_t, np.float64)[r.ray_of]
    on = (np.asarray(mask)[r.ray_of] > 0) & (r.t_in <= t_star) & (t_star <= r.t_out) & (r.t_out > r.t_in)
    # one surface voxel per ray: the first hit containing D*
    first = np.zeros_like(on)
    seen = set()
    for i in np.nonzero(on)[0]:
        if r.ray_of[i] not in seen:
            seen.add(r.ray_of[i])
            first[i] = True
    eg = eta_target(r.t_in, r.t_out, t_star)
    L = float(lam_eta * np.sum(((r.eta - eg) ** 2)[first]) / N)
    deta = np.where(first, 2.0 * lam_eta * (r.eta - eg) / N, 0.0)
    return L, deta
