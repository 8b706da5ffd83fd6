"""The traversal's dense parent index: node words where the level L-3 node
exists, and for every empty parent cell an empty box that holds the cell, holds
its largest empty octree block, and cannot grow by one layer on any face
(checked on host-built and GPU-built trees; the GPU build must equal the
host build entry for entry)."""
import numpy as np
import pytest
import torch

from paper_2205_07058_b300 import inputs as I
from tests.gpu_common import requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


def _unpack(v):
    v = v.astype(np.int64)
    return np.stack([v & 0xFF, (v >> 8) & 0xFF, (v >> 16) & 0xFF], axis=-1)


def _check_index(pidx, leaf_ijk, L):
    G = 1 << (L - 3)
    occ = np.zeros((G, G, G), bool)  # [z, y, x]
    q = leaf_ijk.astype(np.int64) >> 3
    occ[q[:, 2], q[:, 1], q[:, 0]] = True
    w = pidx.reshape(G, G, G, 2).view(np.uint32) if pidx.dtype != np.uint32 else pidx.reshape(G, G, G, 2)
    mask = w[..., 0] >> 24
    assert np.array_equal(mask != 0, occ)
    # node words: the mask bit of each child brick that holds a leaf
    b = leaf_ijk.astype(np.int64) >> 2
    bit = (b[:, 0] & 1) | ((b[:, 1] & 1) << 1) | ((b[:, 2] & 1) << 2)
    expect = np.zeros((G, G, G), np.uint32)
    np.bitwise_or.at(expect, (q[:, 2], q[:, 1], q[:, 0]), (1 << bit).astype(np.uint32))
    assert np.array_equal(mask, expect)
    assert np.all(w[..., 1][occ] == 0)
    # empty cells: boxes
    S = np.zeros((G + 1, G + 1, G + 1), np.int64)
    S[1:, 1:, 1:] = occ.astype(np.int64).cumsum(0).cumsum(1).cumsum(2)

    def count(lo, hi):  # lo, hi: (..., 3) as (x, y, z)
        x0, y0, z0 = lo[..., 0], lo[..., 1], lo[..., 2]
        x1, y1, z1 = hi[..., 0], hi[..., 1], hi[..., 2]
        return (S[z1, y1, x1] - S[z0, y1, x1] - S[z1, y0, x1] - S[z1, y1, x0] + S[z0, y0, x1] + S[z0, y1, x0]
                + S[z1, y0, x0] - S[z0, y0, x0])

    zz, yy, xx = np.nonzero(~occ)
    lo = _unpack(w[zz, yy, xx, 0])
    hi = _unpack(w[zz, yy, xx, 1])
    cell = np.stack([xx, yy, zz], axis=-1)
    assert np.all((lo <= cell) & (cell < hi) & (hi <= G))
    assert np.all(count(lo, hi) == 0)
    # holds the largest empty octree block around the cell
    for e in (1 << np.arange(L - 2)):
        blo = cell & ~(e - 1)
        empty = count(blo, blo + e) == 0
        aligned_ok = np.all((lo <= blo) & (blo + e <= hi), axis=-1)
        assert np.all(aligned_ok | ~empty)
    # maximal: every face is at the grid border or its next layer holds a leaf
    for a in range(3):
        l2, h2 = lo.copy(), hi.copy()
        l2[:, a] = lo[:, a] - 1
        h2[:, a] = lo[:, a]
        border = lo[:, a] == 0
        assert np.all(border | (count(np.maximum(l2, 0), h2) > 0))
        l2, h2 = lo.copy(), hi.copy()
        l2[:, a] = hi[:, a]
        h2[:, a] = hi[:, a] + 1
        border = hi[:, a] == G
        assert np.all(border | (count(l2, np.minimum(h2, G)) > 0))


@pytest.mark.parametrize("L,n_sph,n_box", [(6, 8, 2), (9, 64, 32), (4, 3, 0)])
def test_parent_index_boxes_host_build(L, n_sph, n_box):
    from paper_2205_07058_b300 import svlf
    sc = I.make_scene(np.random.default_rng(70 + L), L, n_sph, n_box)
    tree = svlf.Octree(torch.from_numpy(sc.leaf_ijk), L, host=True)
    pidx = tree.parent_index().cpu().numpy().view(np.uint32)
    assert pidx.shape == ((1 << (L - 3)) ** 3, 2)
    _check_index(pidx, sc.leaf_ijk, L)


def test_parent_index_small_and_empty_trees():
    from paper_2205_07058_b300 import svlf
    t2 = svlf.Octree(torch.tensor([[1, 2, 3]], dtype=torch.int32), 2)
    assert t2.parent_index().shape == (0, 2)
    t3 = svlf.Octree(torch.tensor([[7, 0, 5]], dtype=torch.int32), 3)
    p3 = t3.parent_index().cpu().numpy().view(np.uint32)
    assert p3.shape == (1, 2) and (p3[0, 0] >> 24) != 0 and p3[0, 1] == 0
    te = svlf.Octree(torch.zeros((0, 3), dtype=torch.int32), 6)
    assert te.parent_index().shape == (0, 2)


@pytest.mark.parametrize("L", [5, 7, 9])
def test_parent_index_gpu_build_equals_host_build(L):
    from paper_2205_07058_b300 import svlf
    rng = np.random.default_rng(90 + L)
    sc = I.make_scene(rng, L, 10, 4)
    az, el = I.random_view_angles(rng, 3)
    rays = np.concatenate([I.pinhole_rays(az[v], el[v], 96, 96) for v in range(3)])
    depth, mask = I.analytic_depth(rays, sc)
    depth = np.where(mask > 0, depth, np.nan).astype(np.float32)
    gt = svlf.Octree.from_depth(torch.from_numpy(rays), torch.from_numpy(depth), L)
    leaves = gt.leaf_ijk()
    ht = svlf.Octree(leaves, L, host=True)
    pg = gt.parent_index().cpu().numpy()
    ph = ht.parent_index().cpu().numpy()
    assert np.array_equal(pg, ph)
    _check_index(ph.view(np.uint32), leaves.cpu().numpy(), L)
