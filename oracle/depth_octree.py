"""Occupied voxels from depth maps (Sec. 4.1 "Scene volume": the scene is
partitioned into a voxel grid from the dataset's depth maps and only voxels
holding a surface are kept; Sec. 4.5 builds it at 128^3). TEST
INFRASTRUCTURE ONLY; shares no code with the CUDA path.

Each pixel's ray (origin o, unit direction d) and depth D give the surface
point x = o + D d; its voxel at depth L is floor(x 2^L) per axis, clamped to
[0, 2^L - 1]. Pixels with a non-finite or non-positive depth are skipped.
Floating point decides an integer here, so the point is formed in float32
exactly as the kernel forms it: the product D d rounded, then the sum
rounded (no fused multiply-add), then the exact scaling by 2^L.
"""
from __future__ import annotations

import numpy as np


def depth_voxels(rays: np.ndarray, depth: np.ndarray, L: int) -> np.ndarray:
    """Sorted (lexicographic i, j, k) unique voxels hit by the depth maps."""
    rays = np.asarray(rays, dtype=np.float32).reshape(-1, 6)
    D = np.asarray(depth, dtype=np.float32).reshape(-1)
    ok = np.isfinite(D) & (D > 0)
    o = rays[ok, :3]
    d = rays[ok, 3:]
    x = (o + (D[ok, None] * d).astype(np.float32)).astype(np.float32)
    n = 1 << L
    cell = np.floor(x * np.float32(n)).astype(np.int64)
    cell = np.clip(cell, 0, n - 1)
    return np.unique(cell, axis=0)
