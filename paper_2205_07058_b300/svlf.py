"""Python binding of libsvlf (the C ABI in include/svlf.h).

Argument marshalling only: every step of the render/train path runs in the
library's CUDA kernels. PyTorch supplies device memory and the current CUDA
stream. Importing this module on a machine without the built library raises;
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsvlf.so")

SVLF_OK = 0
SVLF_ERR_ARG = -1
SVLF_ERR_CUDA = -2
SVLF_ERR_DEVICE = -3
SVLF_ERR_UNSUPPORTED = -4
SVLF_ERR_WORKSPACE = -5

SVLF_DEV_STEP_LIMIT = 1
SVLF_DEV_BAD_INDEX = 2
SVLF_DEV_SAMPLE_OVERFLOW = 4
SVLF_DEV_WAIT_TIMEOUT = 8

FP32, BF16, FP16 = 0, 1, 2
RPARAM_SPHERE, RPARAM_AABB = 0, 1  # ray parameterisation of the network input (svlf_render_opts.rparam_mode)
FEAT_F32, FEAT_BF16 = 0, 1
PRECISIONS = {"fp32": FP32, "bf16": BF16, "fp16": FP16}


class SvlfError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"{fn} failed: {code} ({status_string(code)})")
        self.code = code


class MlpDesc(ctypes.Structure):
    _fields_ = [("feat_dim", ctypes.c_int), ("hidden", ctypes.c_int), ("n_hidden", ctypes.c_int),
                ("out_dim", ctypes.c_int), ("precision", ctypes.c_int), ("feat_dtype", ctypes.c_int)]


class TwoDecoderDescC(ctypes.Structure):
    _fields_ = [("feat_t", ctypes.c_int), ("feat_c", ctypes.c_int), ("hidden_t", ctypes.c_int),
                ("n_hidden_t", ctypes.c_int), ("hidden_c", ctypes.c_int), ("n_hidden_c", ctypes.c_int),
                ("precision", ctypes.c_int), ("feat_dtype", ctypes.c_int)]


class RenderOpts(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int), ("bg", ctypes.c_float * 3), ("rparam_mode", ctypes.c_int),
                ("image_width", ctypes.c_int)]


class SceneDesc(ctypes.Structure):
    _fields_ = [("tree", ctypes.c_void_p), ("features", ctypes.c_void_p), ("mlp_params", ctypes.c_void_p),
                ("rays", ctypes.c_void_p), ("n_rays", ctypes.c_int64), ("rgb", ctypes.c_void_p),
                ("depth", ctypes.c_void_p), ("d_rgb", ctypes.c_void_p), ("d_depth", ctypes.c_void_p),
                ("d_features", ctypes.c_void_p), ("d_mlp_params", ctypes.c_void_p)]


class Tuning(ctypes.Structure):
    _fields_ = [("mlp_warpgroups", ctypes.c_int), ("mlp_epilogue_batch", ctypes.c_int),
                ("trace_budget", ctypes.c_int), ("trace_block", ctypes.c_int),
                ("trace_refill", ctypes.c_int), ("mlp_bwd_warpgroups", ctypes.c_int)]


class Camera(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_float * 3), ("fwd", ctypes.c_float * 3), ("right", ctypes.c_float * 3),
                ("up", ctypes.c_float * 3), ("tan_half_fov", ctypes.c_float)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


EXPORTS = [
    "svlf_build_octree", "svlf_octree_leaf_ijk", "svlf_octree_info", "svlf_free_octree",
    "svlf_workspace_size", "svlf_render_rays", "svlf_render_rays_backward", "svlf_loss",
    "svlf_adam_step", "svlf_get_device_status", "svlf_status_string", "svlf_selftest_mma", "svlf_selftest_wait",
    "svlf_profile_enable", "svlf_profile_report", "svlf_workspace_samples",
    "svlf_render_rays_static", "svlf_workspace_size_batched", "svlf_render_rays_batched",
    "svlf_render_rays_backward_batched", "svlf_set_tuning", "svlf_get_tuning",
    "svlf_octree_build_vertices", "svlf_octree_leaf_vertices", "svlf_octree_parent_index", "svlf_selftest_ffma",
    "svlf_workspace_samples_batched", "svlf_workspace_scene_samples", "svlf_pinhole_rays",
    "svlf_workspace_size_two_decoder",
    "svlf_render_rays_two_decoder", "svlf_render_rays_backward_two_decoder", "svlf_surface_loss_two_decoder",
    "svlf_eta_loss_two_decoder", "svlf_build_octree_from_depth", "svlf_set_step_limit",
    "svlf_adam_step_device", "svlf_step_advance", "svlf_loss_shard", "svlf_build_octree_host",
]

_lib = None


def lib():
    """Load libsvlf.so (built in-tree by build_lib.py). Raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libsvlf.so not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, i32, f32, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_float, ctypes.c_size_t
    P = ctypes.POINTER
    L.svlf_build_octree.argtypes = [vp, i64, i32, vp, P(vp), P(i64)]
    L.svlf_build_octree_host.argtypes = [vp, i64, i32, vp, P(vp), P(i64)]
    L.svlf_octree_leaf_ijk.argtypes = [vp, vp, vp]
    L.svlf_build_octree_from_depth.argtypes = [vp, vp, i64, i32, vp, P(vp), P(i64)]
    L.svlf_octree_info.argtypes = [vp, P(i32), P(i64), P(i64), P(i64)]
    L.svlf_free_octree.argtypes = [vp]
    L.svlf_workspace_size.argtypes = [P(MlpDesc), i64, i32, P(sz)]
    L.svlf_render_rays.argtypes = [vp, vp, vp, P(MlpDesc), vp, i64, P(RenderOpts), vp, vp, vp, vp,
                                   vp, sz, vp]
    L.svlf_render_rays_backward.argtypes = [vp, vp, vp, P(MlpDesc), vp, i64, P(RenderOpts), vp,
                                            vp, vp, vp, vp, sz, vp]
    L.svlf_loss.argtypes = [vp, vp, vp, vp, vp, i64, f32, vp, vp, vp, vp]
    L.svlf_loss_shard.argtypes = [vp, vp, vp, vp, vp, i64, i64, f32, vp, vp, vp, vp]
    L.svlf_adam_step.argtypes = [vp, vp, vp, vp, i64, f32, f32, f32, f32, i64, vp, vp]
    L.svlf_adam_step_device.argtypes = [vp, vp, vp, vp, i64, f32, f32, f32, f32, vp, vp, vp]
    L.svlf_step_advance.argtypes = [vp, vp]
    L.svlf_get_device_status.argtypes = [vp, P(i32)]
    L.svlf_set_step_limit.argtypes = [i64]
    L.svlf_selftest_mma.argtypes = [vp, vp, vp, i32, i32, i32, i32, i32, i32, vp]
    L.svlf_workspace_size_batched.argtypes = [P(MlpDesc), i64, i32, i32, P(sz)]
    L.svlf_render_rays_batched.argtypes = [P(SceneDesc), i32, P(MlpDesc), P(RenderOpts), vp, sz, vp]
    L.svlf_render_rays_backward_batched.argtypes = [P(SceneDesc), i32, P(MlpDesc), P(RenderOpts), vp, sz, vp]
    L.svlf_render_rays_static.argtypes = [vp, vp, vp, P(MlpDesc), vp, i64, P(RenderOpts), vp, vp, vp]
    L.svlf_set_tuning.argtypes = [P(Tuning)]
    L.svlf_get_tuning.argtypes = [P(Tuning)]
    L.svlf_profile_enable.argtypes = [i32]
    L.svlf_profile_report.argtypes = [P(KernelStat), i32, P(i32)]
    L.svlf_workspace_samples.argtypes = [vp, P(MlpDesc), i64, i32, P(i64), vp]
    L.svlf_octree_build_vertices.argtypes = [vp, P(i64), vp]
    L.svlf_octree_leaf_vertices.argtypes = [vp, vp, vp]
    L.svlf_octree_parent_index.argtypes = [vp, vp, P(i64), vp]
    L.svlf_selftest_ffma.argtypes = [vp, ctypes.c_int, i64, vp]
    L.svlf_selftest_wait.argtypes = [i64, ctypes.c_int, vp, vp]
    L.svlf_workspace_samples_batched.argtypes = [vp, P(MlpDesc), P(i64), i32, i32, P(i64), vp]
    L.svlf_workspace_scene_samples.argtypes = [vp, P(MlpDesc), P(i64), i32, i32, P(i64), vp]
    L.svlf_pinhole_rays.argtypes = [P(Camera), i32, i32, i32, vp, vp]
    L.svlf_workspace_size_two_decoder.argtypes = [P(TwoDecoderDescC), i64, i32, P(sz)]
    L.svlf_render_rays_two_decoder.argtypes = [vp, vp, vp, vp, vp, P(TwoDecoderDescC), vp, i64, P(RenderOpts),
                                               vp, vp, vp, vp, vp, sz, vp]
    L.svlf_render_rays_backward_two_decoder.argtypes = [vp, vp, vp, vp, vp, P(TwoDecoderDescC), vp, i64,
                                                        P(RenderOpts), vp, vp, vp, vp, vp, vp, vp, sz, vp]
    L.svlf_surface_loss_two_decoder.argtypes = [vp, vp, vp, vp, vp, P(TwoDecoderDescC), vp, i64, vp, vp, vp, f32,
                                                f32, vp, vp, vp, vp, vp, vp, sz, vp]
    L.svlf_eta_loss_two_decoder.argtypes = [vp, P(TwoDecoderDescC), vp, i64, P(RenderOpts), vp, vp, f32, vp, vp,
                                            sz, vp]
    L.svlf_status_string.argtypes = [i32]
    L.svlf_status_string.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name != "svlf_status_string":
            getattr(L, name).restype = i32
    _lib = L
    return L


def status_string(code: int) -> str:
    return lib().svlf_status_string(int(code)).decode()


def _check(fn: str, rc: int):
    if rc != SVLF_OK:
        raise SvlfError(fn, rc)


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


# ---------------------------------------------------------------------------
# octree
# ---------------------------------------------------------------------------
class Octree:
    """Library-owned sparse octree (svlf_build_octree)."""

    def __init__(self, leaf_ijk: torch.Tensor, depth: int, stream=None, host: bool = False):
        """Octree over the leaves (n x 3 ijk), built on the GPU (or, with
        host=True, by the library's independent host construction)."""
        ijk = leaf_ijk.to(device="cuda", dtype=torch.int32).contiguous()
        h = ctypes.c_void_p()
        n = ctypes.c_int64()
        fn = "svlf_build_octree_host" if host else "svlf_build_octree"
        _check(fn, getattr(lib(), fn)(
            _ptr(ijk), ijk.shape[0], int(depth), _stream(stream), ctypes.byref(h), ctypes.byref(n)))
        self.handle = h
        self.depth = int(depth)
        self.n_leaves = int(n.value)

    @classmethod
    def from_depth(cls, rays: torch.Tensor, depth: torch.Tensor, depth_levels: int, stream=None) -> "Octree":
        """Octree of the voxels the depth maps' surface points fall in, built on the GPU."""
        r = rays.to(device="cuda", dtype=torch.float32).contiguous()
        d = depth.to(device="cuda", dtype=torch.float32).contiguous()
        h = ctypes.c_void_p()
        n = ctypes.c_int64()
        _check("svlf_build_octree_from_depth", lib().svlf_build_octree_from_depth(
            _ptr(r), _ptr(d), r.shape[0], int(depth_levels), _stream(stream), ctypes.byref(h), ctypes.byref(n)))
        t = cls.__new__(cls)
        t.handle = h
        t.depth = int(depth_levels)
        t.n_leaves = int(n.value)
        return t

    def info(self):
        d, nl, nn, nb = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check("svlf_octree_info", lib().svlf_octree_info(self.handle, ctypes.byref(d), ctypes.byref(nl),
                                                           ctypes.byref(nn), ctypes.byref(nb)))
        return {"depth": d.value, "n_leaves": nl.value, "n_nodes": nn.value, "n_bricks": nb.value}

    def leaf_ijk(self, stream=None) -> torch.Tensor:
        out = torch.empty((self.n_leaves, 3), dtype=torch.int32, device="cuda")
        _check("svlf_octree_leaf_ijk", lib().svlf_octree_leaf_ijk(self.handle, _ptr(out), _stream(stream)))
        return out

    def parent_index(self, stream=None) -> torch.Tensor:
        """The dense parent index (n_entries x 2 int32 on the device; the uint32
        words reinterpreted): node words, or empty boxes (lo, hi)."""
        n = ctypes.c_int64()
        _check("svlf_octree_parent_index", lib().svlf_octree_parent_index(self.handle, None, ctypes.byref(n), None))
        out = torch.empty((n.value, 2), dtype=torch.int32, device="cuda")
        if n.value:
            _check("svlf_octree_parent_index", lib().svlf_octree_parent_index(self.handle, _ptr(out), ctypes.byref(n),
                                                                               _stream(stream)))
        return out

    def build_vertices(self, stream=None) -> int:
        """Vertex table of the two-decoder form; returns the vertex count."""
        n = ctypes.c_int64()
        _check("svlf_octree_build_vertices", lib().svlf_octree_build_vertices(self.handle, ctypes.byref(n),
                                                                               _stream(stream)))
        self.n_vertices = int(n.value)
        return self.n_vertices

    def leaf_vertices(self, stream=None) -> torch.Tensor:
        out = torch.empty((self.n_leaves, 8), dtype=torch.int32, device="cuda")
        _check("svlf_octree_leaf_vertices", lib().svlf_octree_leaf_vertices(self.handle, _ptr(out), _stream(stream)))
        return out

    def free(self):
        if self.handle:
            lib().svlf_free_octree(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# rendering
# ---------------------------------------------------------------------------
@dataclass
class Network:
    feat_dim: int
    hidden: int
    n_hidden: int
    precision: int = FP32
    feat_dtype: int = FEAT_F32

    def desc(self) -> MlpDesc:
        return MlpDesc(self.feat_dim, self.hidden, self.n_hidden, 4, self.precision, self.feat_dtype)


def workspace_size(net: Network, n_rays: int, K: int) -> int:
    b = ctypes.c_size_t()
    d = net.desc()
    _check("svlf_workspace_size", lib().svlf_workspace_size(ctypes.byref(d), int(n_rays), int(K), ctypes.byref(b)))
    return int(b.value)


def alloc_workspace(net: Network, n_rays: int, K: int) -> torch.Tensor:
    """A 256-byte aligned device buffer of svlf_workspace_size bytes."""
    return torch.empty(workspace_size(net, n_rays, K) + 256, dtype=torch.uint8, device="cuda")


def _ws_ptr(ws: torch.Tensor):
    p = ws.data_ptr()
    aligned = (p + 255) & ~255
    return ctypes.c_void_p(aligned), ws.numel() - (aligned - p)


def _opts(K: int, bg: Sequence[float], rparam: int = RPARAM_SPHERE, image_width: int = 0) -> RenderOpts:
    o = RenderOpts()
    o.K = int(K)
    for i in range(3):
        o.bg[i] = float(bg[i])
    o.rparam_mode = int(rparam)
    o.image_width = int(image_width)
    return o


# ---------------------------------------------------------------------------
# argument checks: the C ABI takes raw device pointers, so a table of the wrong
# dtype or shape would be read out of bounds on the GPU; the binding refuses it
# ---------------------------------------------------------------------------
def _param_count(dims) -> int:
    """Flat parameter count of layers [(out, in), ...]: W (out x in) then b."""
    return sum(o * i + o for o, i in dims)


def _net_dims(net: "Network"):
    return [(net.hidden, net.feat_dim + 9)] + [(net.hidden, net.hidden)] * (net.n_hidden - 1) + [(4, net.hidden)]


def _td_dims(net: "TwoDecoder"):
    dt = [(net.hidden_t, 2 * net.feat_t + 6)] + [(net.hidden_t, net.hidden_t)] * (net.n_hidden_t - 1) + \
        [(2, net.hidden_t)]
    dc = [(net.hidden_c, net.feat_c + 6)] + [(net.hidden_c, net.hidden_c)] * (net.n_hidden_c - 1) + \
        [(3, net.hidden_c)]
    return dt, dc


def _check_table(name: str, t: Optional[torch.Tensor], rows: Optional[int], cols: int, feat_dtype: int,
                 grad: bool = False):
    """A feature table (or its float32 gradient) of at least `rows` x `cols`."""
    if t is None:
        return
    want = torch.float32 if grad or feat_dtype != FEAT_BF16 else torch.bfloat16
    if t.dtype != want:
        raise ValueError(f"{name}: dtype {t.dtype}, expected {want} (feat_dtype {feat_dtype})")
    if t.dim() != 2 or t.shape[1] != cols or (rows is not None and t.shape[0] < rows):
        raise ValueError(f"{name}: shape {tuple(t.shape)}, expected ({rows}, {cols})")


def _check_params(name: str, t: Optional[torch.Tensor], dims):
    if t is None:
        return
    n = _param_count(dims)
    if t.dtype != torch.float32 or t.numel() < n:
        raise ValueError(f"{name}: {t.numel()} x {t.dtype}, expected at least {n} x torch.float32")


def _check_rays(rays: torch.Tensor):
    if rays.dtype != torch.float32 or rays.dim() != 2 or rays.shape[1] != 6:
        raise ValueError(f"rays: {tuple(rays.shape)} x {rays.dtype}, expected (N, 6) x torch.float32")


def _check_single(tree, features, params, net, rays, d_features=None, d_params=None):
    _check_rays(rays)
    _check_table("features", features, tree.n_leaves, net.feat_dim, net.feat_dtype)
    _check_table("d_features", d_features, tree.n_leaves, net.feat_dim, net.feat_dtype, grad=True)
    dims = _net_dims(net)
    _check_params("params", params, dims)
    _check_params("d_params", d_params, dims)


def _check_two_decoder(tree, z_t, z_c, params_t, params_c, net, rays, d_z_t=None, d_z_c=None, d_params_t=None,
                       d_params_c=None):
    _check_rays(rays)
    nv = getattr(tree, "n_vertices", None)
    _check_table("z_t", z_t, nv, net.feat_t, net.feat_dtype)
    _check_table("z_c", z_c, nv, net.feat_c, net.feat_dtype)
    _check_table("d_z_t", d_z_t, nv, net.feat_t, net.feat_dtype, grad=True)
    _check_table("d_z_c", d_z_c, nv, net.feat_c, net.feat_dtype, grad=True)
    dt, dc = _td_dims(net)
    _check_params("params_t", params_t, dt)
    _check_params("params_c", params_c, dc)
    _check_params("d_params_t", d_params_t, dt)
    _check_params("d_params_c", d_params_c, dc)


def svlf_render_rays(tree: Octree, features: torch.Tensor, params: torch.Tensor, net: Network,
                     rays: torch.Tensor, K: int, bg=(0.0, 0.0, 0.0), workspace: Optional[torch.Tensor] = None,
                     want_hits: bool = False, out: Optional[tuple] = None, stream=None, rparam: int = RPARAM_SPHERE,
                     image_width: int = 0):
    """Returns (rgb (N,3), depth (N,), hits (N,K) or None, t_io (N,K,2) or None, workspace).
    image_width > 0: the rays are rows of images that wide (traversal order
    only; svlf_render_opts.image_width)."""
    _check_single(tree, features, params, net, rays)
    N = rays.shape[0]
    if workspace is None:
        workspace = alloc_workspace(net, N, K)
    if out is None:
        rgb = torch.empty((N, 3), dtype=torch.float32, device="cuda")
        depth = torch.empty((N,), dtype=torch.float32, device="cuda")
    else:
        rgb, depth = out
    hits = torch.empty((N, K), dtype=torch.int32, device="cuda") if want_hits else None
    t_io = torch.empty((N, K, 2), dtype=torch.float32, device="cuda") if want_hits else None
    d = net.desc()
    o = _opts(K, bg, rparam, image_width)
    wp, wb = _ws_ptr(workspace)
    _check("svlf_render_rays", lib().svlf_render_rays(
        tree.handle, _ptr(features), _ptr(params), ctypes.byref(d), _ptr(rays), N, ctypes.byref(o),
        _ptr(rgb), _ptr(depth), _ptr(hits), _ptr(t_io), wp, wb, _stream(stream)))
    return rgb, depth, hits, t_io, workspace


@dataclass
class TwoDecoder:
    """Shapes of the two-decoder form (defaults: the paper's Sec. 4.5 sizes)."""
    feat_t: int = 64
    feat_c: int = 32
    hidden_t: int = 128
    n_hidden_t: int = 1
    hidden_c: int = 128
    n_hidden_c: int = 3
    precision: int = BF16
    feat_dtype: int = FEAT_F32

    def desc(self) -> TwoDecoderDescC:
        return TwoDecoderDescC(self.feat_t, self.feat_c, self.hidden_t, self.n_hidden_t, self.hidden_c,
                               self.n_hidden_c, self.precision, self.feat_dtype)


def workspace_size_two_decoder(net: TwoDecoder, n_rays: int, K: int) -> int:
    b = ctypes.c_size_t()
    d = net.desc()
    _check("svlf_workspace_size_two_decoder",
           lib().svlf_workspace_size_two_decoder(ctypes.byref(d), int(n_rays), int(K), ctypes.byref(b)))
    return int(b.value)


def svlf_render_rays_two_decoder(tree: Octree, z_t: torch.Tensor, z_c: torch.Tensor, params_t: torch.Tensor,
                                 params_c: torch.Tensor, net: TwoDecoder, rays: torch.Tensor, K: int,
                                 bg=(0.0, 0.0, 0.0), workspace: Optional[torch.Tensor] = None,
                                 want_hits: bool = False, out: Optional[tuple] = None, stream=None,
                                 image_width: int = 0):
    """Two-decoder render (the octree's vertex table must be built).
    Returns (rgb, depth, hits or None, t_io or None, workspace)."""
    _check_two_decoder(tree, z_t, z_c, params_t, params_c, net, rays)
    N = rays.shape[0]
    if workspace is None:
        workspace = torch.empty(workspace_size_two_decoder(net, N, K) + 256, dtype=torch.uint8, device="cuda")
    if out is None:
        rgb = torch.empty((N, 3), dtype=torch.float32, device="cuda")
        depth = torch.empty((N,), dtype=torch.float32, device="cuda")
    else:
        rgb, depth = out
    hits = torch.empty((N, K), dtype=torch.int32, device="cuda") if want_hits else None
    t_io = torch.empty((N, K, 2), dtype=torch.float32, device="cuda") if want_hits else None
    d = net.desc()
    o = _opts(K, bg, image_width=image_width)
    wp, wb = _ws_ptr(workspace)
    _check("svlf_render_rays_two_decoder", lib().svlf_render_rays_two_decoder(
        tree.handle, _ptr(z_t), _ptr(z_c), _ptr(params_t), _ptr(params_c), ctypes.byref(d), _ptr(rays), N,
        ctypes.byref(o), _ptr(rgb), _ptr(depth), _ptr(hits), _ptr(t_io), wp, wb, _stream(stream)))
    return rgb, depth, hits, t_io, workspace


def svlf_render_rays_backward_two_decoder(tree: Octree, z_t, z_c, params_t, params_c, net: TwoDecoder,
                                          rays: torch.Tensor, K: int, bg, d_rgb: torch.Tensor, d_depth: torch.Tensor,
                                          d_z_t=None, d_z_c=None, d_params_t=None, d_params_c=None,
                                          workspace: torch.Tensor = None, stream=None):
    """Accumulates the gradients (those passed) of the two-decoder render whose
    workspace is given."""
    _check_two_decoder(tree, z_t, z_c, params_t, params_c, net, rays, d_z_t, d_z_c, d_params_t, d_params_c)
    d = net.desc()
    o = _opts(K, bg)
    wp, wb = _ws_ptr(workspace)
    _check("svlf_render_rays_backward_two_decoder", lib().svlf_render_rays_backward_two_decoder(
        tree.handle, _ptr(z_t), _ptr(z_c), _ptr(params_t), _ptr(params_c), ctypes.byref(d), _ptr(rays),
        rays.shape[0], ctypes.byref(o), _ptr(d_rgb), _ptr(d_depth), _ptr(d_z_t), _ptr(d_z_c), _ptr(d_params_t),
        _ptr(d_params_c), wp, wb, _stream(stream)))


def svlf_surface_loss_two_decoder(tree: Octree, z_t, z_c, params_t, params_c, net: TwoDecoder, rays, rgb_target,
                                  depth_target, mask, lambda_eta: float, lambda_tau: float, loss: torch.Tensor,
                                  d_z_t=None, d_z_c=None, d_params_t=None, d_params_c=None, workspace=None,
                                  stream=None):
    """Stage 1 of the staged training (Eq. 4 on the rays' surface voxels);
    adds to `loss` (1-element float64) and accumulates the given gradients.
    Returns the workspace."""
    _check_two_decoder(tree, z_t, z_c, params_t, params_c, net, rays, d_z_t, d_z_c, d_params_t, d_params_c)
    N = rays.shape[0]
    if workspace is None:
        workspace = torch.empty(workspace_size_two_decoder(net, N, 1) + 256, dtype=torch.uint8, device="cuda")
    d = net.desc()
    wp, wb = _ws_ptr(workspace)
    _check("svlf_surface_loss_two_decoder", lib().svlf_surface_loss_two_decoder(
        tree.handle, _ptr(z_t), _ptr(z_c), _ptr(params_t), _ptr(params_c), ctypes.byref(d), _ptr(rays), N,
        _ptr(rgb_target), _ptr(depth_target), _ptr(mask), float(lambda_eta), float(lambda_tau), _ptr(loss),
        _ptr(d_z_t), _ptr(d_z_c), _ptr(d_params_t), _ptr(d_params_c), wp, wb, _stream(stream)))
    return workspace


def svlf_eta_loss_two_decoder(tree: Octree, net: TwoDecoder, rays, K: int, depth_target, mask, lambda_eta: float,
                              loss: torch.Tensor, workspace: torch.Tensor, stream=None):
    """Stages 2-3: the eta term on the surface voxels among the hits of the
    render whose workspace is given (call before its backward)."""
    d = net.desc()
    o = _opts(K, (0.0, 0.0, 0.0))
    wp, wb = _ws_ptr(workspace)
    _check("svlf_eta_loss_two_decoder", lib().svlf_eta_loss_two_decoder(
        tree.handle, ctypes.byref(d), _ptr(rays), rays.shape[0], ctypes.byref(o), _ptr(depth_target), _ptr(mask),
        float(lambda_eta), _ptr(loss), wp, wb, _stream(stream)))


def svlf_render_rays_static(tree: Octree, features: torch.Tensor, params: torch.Tensor, net: Network,
                            rays: torch.Tensor, K: int, bg=(0.0, 0.0, 0.0), out: Optional[tuple] = None,
                            stream=None, rparam: int = RPARAM_SPHERE, image_width: int = 0):
    """Render without a workspace (the library's fixed scratch array); for
    callers that may not allocate device memory. Returns (rgb, depth)."""
    _check_single(tree, features, params, net, rays)
    N = rays.shape[0]
    if out is None:
        out = (torch.empty((N, 3), dtype=torch.float32, device="cuda"),
               torch.empty((N,), dtype=torch.float32, device="cuda"))
    rgb, depth = out
    d = net.desc()
    o = _opts(K, bg, rparam, image_width)
    _check("svlf_render_rays_static", lib().svlf_render_rays_static(
        tree.handle, _ptr(features), _ptr(params), ctypes.byref(d), _ptr(rays), N, ctypes.byref(o),
        _ptr(rgb), _ptr(depth), _stream(stream)))
    return rgb, depth


@dataclass
class BatchScene:
    """One scene of a batched call; tensors are CUDA and contiguous."""
    tree: "Octree"
    features: torch.Tensor
    params: torch.Tensor
    rays: torch.Tensor
    rgb: Optional[torch.Tensor] = None
    depth: Optional[torch.Tensor] = None
    d_rgb: Optional[torch.Tensor] = None
    d_depth: Optional[torch.Tensor] = None
    d_features: Optional[torch.Tensor] = None
    d_params: Optional[torch.Tensor] = None

    def desc(self) -> SceneDesc:
        v = lambda t: None if t is None else _ptr(t)
        return SceneDesc(self.tree.handle, v(self.features), v(self.params), v(self.rays), self.rays.shape[0],
                         v(self.rgb), v(self.depth), v(self.d_rgb), v(self.d_depth), v(self.d_features),
                         v(self.d_params))


def workspace_size_batched(net: Network, total_rays: int, n_scenes: int, K: int) -> int:
    b = ctypes.c_size_t()
    d = net.desc()
    _check("svlf_workspace_size_batched", lib().svlf_workspace_size_batched(
        ctypes.byref(d), int(total_rays), int(n_scenes), int(K), ctypes.byref(b)))
    return int(b.value)


def alloc_workspace_batched(net: Network, scenes: Sequence[BatchScene], K: int) -> torch.Tensor:
    total = sum(s.rays.shape[0] for s in scenes)
    return torch.empty(workspace_size_batched(net, total, len(scenes), K) + 256, dtype=torch.uint8, device="cuda")


def svlf_render_rays_batched(scenes: Sequence[BatchScene], net: Network, K: int, bg=(0.0, 0.0, 0.0),
                             workspace: Optional[torch.Tensor] = None, stream=None, rparam: int = RPARAM_SPHERE,
                             image_width: int = 0):
    """Render every scene in one call; fills each scene's rgb/depth (allocated
    here when missing). Returns the workspace (needed by the backward)."""
    for s in scenes:
        _check_single(s.tree, s.features, s.params, net, s.rays)
    for s in scenes:
        if s.rgb is None:
            s.rgb = torch.empty((s.rays.shape[0], 3), dtype=torch.float32, device="cuda")
        if s.depth is None:
            s.depth = torch.empty((s.rays.shape[0],), dtype=torch.float32, device="cuda")
    if workspace is None:
        workspace = alloc_workspace_batched(net, scenes, K)
    arr = (SceneDesc * len(scenes))(*[s.desc() for s in scenes])
    d = net.desc()
    o = _opts(K, bg, rparam, image_width)
    wp, wb = _ws_ptr(workspace)
    _check("svlf_render_rays_batched", lib().svlf_render_rays_batched(
        arr, len(scenes), ctypes.byref(d), ctypes.byref(o), wp, wb, _stream(stream)))
    return workspace


def svlf_workspace_samples_batched(workspace: torch.Tensor, net: Network, scenes: Sequence[BatchScene], K: int,
                                   stream=None) -> int:
    """Samples the last batched call over `scenes` wrote into `workspace`."""
    rays = (ctypes.c_int64 * len(scenes))(*[int(s.rays.shape[0]) for s in scenes])
    d = net.desc()
    n = ctypes.c_int64()
    wp, _ = _ws_ptr(workspace)
    _check("svlf_workspace_samples_batched", lib().svlf_workspace_samples_batched(
        wp, ctypes.byref(d), rays, len(scenes), int(K), ctypes.byref(n), _stream(stream)))
    return n.value


def svlf_workspace_scene_samples(workspace: torch.Tensor, net: Network, scenes: Sequence[BatchScene], K: int,
                                 stream=None) -> list:
    """Samples the last batched call over `scenes` wrote into `workspace`, per scene."""
    rays = (ctypes.c_int64 * len(scenes))(*[int(s.rays.shape[0]) for s in scenes])
    per = (ctypes.c_int64 * len(scenes))()
    d = net.desc()
    wp, _ = _ws_ptr(workspace)
    _check("svlf_workspace_scene_samples", lib().svlf_workspace_scene_samples(
        wp, ctypes.byref(d), rays, len(scenes), int(K), per, _stream(stream)))
    return [int(x) for x in per]


def svlf_render_rays_backward_batched(scenes: Sequence[BatchScene], net: Network, K: int, bg, workspace,
                                      stream=None, rparam: int = RPARAM_SPHERE):
    for s in scenes:
        _check_single(s.tree, s.features, s.params, net, s.rays, s.d_features, s.d_params)
    arr = (SceneDesc * len(scenes))(*[s.desc() for s in scenes])
    d = net.desc()
    o = _opts(K, bg, rparam)
    wp, wb = _ws_ptr(workspace)
    _check("svlf_render_rays_backward_batched", lib().svlf_render_rays_backward_batched(
        arr, len(scenes), ctypes.byref(d), ctypes.byref(o), wp, wb, _stream(stream)))


def svlf_render_rays_backward(tree: Octree, features: torch.Tensor, params: torch.Tensor, net: Network,
                              rays: torch.Tensor, K: int, bg, d_rgb: torch.Tensor, d_depth: torch.Tensor,
                              d_features: Optional[torch.Tensor], d_params: Optional[torch.Tensor],
                              workspace: torch.Tensor, stream=None, rparam: int = RPARAM_SPHERE):
    _check_single(tree, features, params, net, rays, d_features, d_params)
    d = net.desc()
    o = _opts(K, bg, rparam)
    wp, wb = _ws_ptr(workspace)
    _check("svlf_render_rays_backward", lib().svlf_render_rays_backward(
        tree.handle, _ptr(features), _ptr(params), ctypes.byref(d), _ptr(rays), rays.shape[0],
        ctypes.byref(o), _ptr(d_rgb), _ptr(d_depth), _ptr(d_features), _ptr(d_params), wp, wb,
        _stream(stream)))


def svlf_loss(rgb, depth, rgb_t, depth_t, mask, depth_weight: float, d_rgb, d_depth, loss_accum, stream=None,
              n_total: Optional[int] = None):
    """Training loss and its output gradients. With n_total (a data-parallel
    shard of a batch of n_total rays) the sum is divided by n_total."""
    if n_total is None:
        _check("svlf_loss", lib().svlf_loss(_ptr(rgb), _ptr(depth), _ptr(rgb_t), _ptr(depth_t), _ptr(mask),
                                            rgb.shape[0], float(depth_weight), _ptr(d_rgb), _ptr(d_depth),
                                            _ptr(loss_accum), _stream(stream)))
    else:
        _check("svlf_loss_shard", lib().svlf_loss_shard(
            _ptr(rgb), _ptr(depth), _ptr(rgb_t), _ptr(depth_t), _ptr(mask), rgb.shape[0], int(n_total),
            float(depth_weight), _ptr(d_rgb), _ptr(d_depth), _ptr(loss_accum), _stream(stream)))


def svlf_adam_step(params, grads, m, v, step: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                   bf16_shadow: Optional[torch.Tensor] = None, stream=None):
    _check("svlf_adam_step", lib().svlf_adam_step(_ptr(params), _ptr(grads), _ptr(m), _ptr(v), params.numel(),
                                                  float(lr), float(beta1), float(beta2), float(eps), int(step),
                                                  _ptr(bf16_shadow), _stream(stream)))


def svlf_adam_step_device(params, grads, m, v, step: torch.Tensor, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                          bf16_shadow: Optional[torch.Tensor] = None, stream=None):
    """Adam with the step count read from `step` (a 1-element int64 CUDA
    tensor) when the kernel runs: capturable in a CUDA graph."""
    if step.dtype != torch.int64 or step.numel() != 1:
        raise ValueError("step: expected a 1-element torch.int64 tensor")
    _check("svlf_adam_step_device", lib().svlf_adam_step_device(
        _ptr(params), _ptr(grads), _ptr(m), _ptr(v), params.numel(), float(lr), float(beta1), float(beta2),
        float(eps), _ptr(step), _ptr(bf16_shadow), _stream(stream)))


def svlf_step_advance(step: torch.Tensor, stream=None):
    """step += 1 on the device (the counter svlf_adam_step_device reads)."""
    if step.dtype != torch.int64 or step.numel() != 1:
        raise ValueError("step: expected a 1-element torch.int64 tensor")
    _check("svlf_step_advance", lib().svlf_step_advance(_ptr(step), _stream(stream)))


def svlf_selftest_mma(A: torch.Tensor, B: torch.Tensor, a_mn_major=False, b_mn_major=False, flags=0,
                      stream=None):
    """D = A @ B.T (A: 128 x K, B: N x K, bf16 or fp16) through one tcgen05 tile."""
    D = torch.empty((128, B.shape[0]), dtype=torch.float32, device="cuda")
    _check("svlf_selftest_mma", lib().svlf_selftest_mma(
        _ptr(A), _ptr(B), _ptr(D), B.shape[0], A.shape[1], int(a_mn_major), int(b_mn_major),
        int(A.dtype == torch.bfloat16), int(flags), _stream(stream)))
    return D


def cameras(eye, fwd, right, up, tan_half_fov):
    """Camera array for svlf_pinhole_rays from (n, 3) basis arrays and (n,) tan(fov/2)."""
    eye, fwd, right, up = (np.asarray(x, dtype=np.float64).reshape(-1, 3) for x in (eye, fwd, right, up))
    th = np.broadcast_to(np.asarray(tan_half_fov, dtype=np.float64), (eye.shape[0],))
    arr = (Camera * eye.shape[0])()
    for i in range(eye.shape[0]):
        arr[i] = Camera((ctypes.c_float * 3)(*eye[i]), (ctypes.c_float * 3)(*fwd[i]),
                        (ctypes.c_float * 3)(*right[i]), (ctypes.c_float * 3)(*up[i]), float(th[i]))
    return arr


def svlf_pinhole_rays(cams, width: int, height: int, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Rays of len(cams) pinhole views of width x height, generated on the device."""
    n = len(cams) * width * height
    if out is None:
        out = torch.empty((n, 6), dtype=torch.float32, device="cuda")
    _check("svlf_pinhole_rays", lib().svlf_pinhole_rays(cams, len(cams), int(width), int(height), _ptr(out),
                                                         _stream(stream)))
    return out


def svlf_measure_ffma_tflops(iters: int = 20000, repeats: int = 5) -> float:
    """Measured float32 FMA throughput of this GPU (TFLOP/s), from the library's
    FMA kernel timed with CUDA events: the FP32 SIMT roofline's denominator."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks = sms * 8
    out = torch.empty(blocks, device="cuda")
    _check("svlf_selftest_ffma", lib().svlf_selftest_ffma(_ptr(out), blocks, int(iters), _stream(None)))
    best = None
    for _ in range(repeats):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        _check("svlf_selftest_ffma", lib().svlf_selftest_ffma(_ptr(out), blocks, int(iters), _stream(None)))
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        best = ms if best is None else min(best, ms)
    return blocks * 256 * iters * 32 / (best / 1e3) / 1e12


def svlf_selftest_wait(limit_cycles: int, arrive: bool = False, stream=None):
    """Runs the bounded-wait self-test; returns (completed, clocks waited).
    Without `arrive` the wait gives up and latches SVLF_DEV_WAIT_TIMEOUT."""
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    _check("svlf_selftest_wait", lib().svlf_selftest_wait(int(limit_cycles), 1 if arrive else 0, _ptr(out),
                                                          _stream(stream)))
    r = out.cpu()
    return bool(r[0].item()), int(r[1].item())


def svlf_set_tuning(mlp_warpgroups=0, mlp_epilogue_batch=0, trace_budget=0, trace_block=0, trace_refill=0,
                    mlp_bwd_warpgroups=0):
    t = Tuning(int(mlp_warpgroups), int(mlp_epilogue_batch), int(trace_budget), int(trace_block),
               int(trace_refill), int(mlp_bwd_warpgroups))
    _check("svlf_set_tuning", lib().svlf_set_tuning(ctypes.byref(t)))


def svlf_get_tuning() -> dict:
    t = Tuning()
    _check("svlf_get_tuning", lib().svlf_get_tuning(ctypes.byref(t)))
    return {f: getattr(t, f) for f, _ in Tuning._fields_}


def svlf_profile_enable(on: bool = True):
    _check("svlf_profile_enable", lib().svlf_profile_enable(int(on)))


def svlf_profile_report() -> dict:
    """{kernel name: (launches, total ms)} since the last report (synchronises)."""
    arr = (KernelStat * 64)()
    n = ctypes.c_int()
    _check("svlf_profile_report", lib().svlf_profile_report(arr, 64, ctypes.byref(n)))
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(min(n.value, 64))}


def svlf_workspace_samples(workspace: torch.Tensor, net: Network, n_rays: int, K: int, stream=None) -> int:
    d = net.desc()
    wp, _ = _ws_ptr(workspace)
    n = ctypes.c_int64()
    _check("svlf_workspace_samples", lib().svlf_workspace_samples(wp, ctypes.byref(d), int(n_rays), int(K),
                                                                   ctypes.byref(n), _stream(stream)))
    return int(n.value)


def svlf_get_device_status(stream=None) -> int:
    """Reads and clears the device status word after the work queued on
    `stream` (default: the current stream); synchronises that stream."""
    s = ctypes.c_int()
    _check("svlf_get_device_status", lib().svlf_get_device_status(_stream(stream), ctypes.byref(s)))
    return int(s.value)


def svlf_set_step_limit(max_steps: int = 0):
    """Traversal safety bound per ray (0 = the default 3 * 2^L + 64)."""
    _check("svlf_set_step_limit", lib().svlf_set_step_limit(int(max_steps)))


# ---------------------------------------------------------------------------
# autograd
# ---------------------------------------------------------------------------
class SvlfRender(torch.autograd.Function):
    """rgb, depth = render(features, params); backward through the library's
    hand-written kernels (activations recomputed, not stored)."""

    @staticmethod
    def forward(ctx, features, params, tree, net, rays, K, bg, rparam=RPARAM_SPHERE, image_width=0):
        rgb, depth, _, _, ws = svlf_render_rays(tree, features, params, net, rays, K, bg, rparam=rparam,
                                                image_width=image_width)
        ctx.save_for_backward(features, params, rays)
        ctx.tree, ctx.net, ctx.K, ctx.bg, ctx.ws, ctx.rparam = tree, net, K, bg, ws, rparam
        return rgb, depth

    @staticmethod
    def backward(ctx, g_rgb, g_depth):
        features, params, rays = ctx.saved_tensors
        df = torch.zeros(features.shape, dtype=torch.float32, device="cuda") if ctx.needs_input_grad[0] else None
        dp = torch.zeros_like(params) if ctx.needs_input_grad[1] else None
        svlf_render_rays_backward(ctx.tree, features, params, ctx.net, rays, ctx.K, ctx.bg,
                                  g_rgb.contiguous(), g_depth.contiguous(), df, dp, ctx.ws, rparam=ctx.rparam)
        ctx.ws = None
        return df, dp, None, None, None, None, None, None, None


def render(features, params, tree: Octree, net: Network, rays, K: int, bg=(0.0, 0.0, 0.0),
           rparam: int = RPARAM_SPHERE, image_width: int = 0):
    return SvlfRender.apply(features, params, tree, net, rays, K, tuple(bg), rparam, image_width)
