"""Octree built on the GPU from depth maps (Sec. 4.1, 4.5) against the
oracle's voxels, the host build of the same leaves, and traversal parity."""
import numpy as np
import pytest
import torch

from oracle import depth_octree as DO
from oracle import oracle as O
from paper_2205_07058_b300 import inputs as I
from tests.gpu_common import compare_hits, random_rays, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


def _depth_maps(seed, L, n_sph, n_box, views, res):
    rng = np.random.default_rng(seed)
    sc = I.make_scene(rng, L, n_sph, n_box)
    az, el = I.random_view_angles(rng, views)
    rays = np.concatenate([I.pinhole_rays(az[v], el[v], res, res) for v in range(views)])
    depth, mask = I.analytic_depth(rays, sc)
    return rays, np.where(mask > 0, depth, np.nan).astype(np.float32)


def _morton(ijk, L):
    code = np.zeros(ijk.shape[0], dtype=np.uint64)
    for b in range(L):
        for a in range(3):
            code |= ((ijk[:, a].astype(np.uint64) >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + a)
    return code


@pytest.mark.parametrize("L,views,res", [(7, 4, 128), (2, 1, 32), (3, 1, 48), (5, 2, 64), (10, 2, 256)])
def test_leaves_nodes_and_traversal(L, views, res):
    from paper_2205_07058_b300 import svlf
    rays, depth = _depth_maps(1013 + L, L, 12, 6, views, res)
    tree = svlf.Octree.from_depth(torch.from_numpy(rays), torch.from_numpy(depth), L)
    torch.cuda.synchronize()
    vox = DO.depth_voxels(rays, depth, L)
    assert tree.n_leaves == vox.shape[0] > 0
    # rank order = Morton order of the oracle's voxels
    ref = vox[np.argsort(_morton(vox, L))]
    assert np.array_equal(tree.leaf_ijk().cpu().numpy(), ref)
    # the same structure as the library's host construction of those leaves
    host = svlf.Octree(torch.from_numpy(ref.astype(np.int32)), L, host=True)
    assert tree.info() == host.info()
    assert torch.equal(tree.parent_index(), host.parent_index())
    # hit lists on the GPU-built tree, bit-exact against the oracle's walk
    rng = np.random.default_rng(L)
    probe = np.concatenate([rays[rng.choice(rays.shape[0], min(4000, rays.shape[0]), replace=False)],
                            random_rays(rng, 4000)])
    K = 6
    net = svlf.Network(8, 32, 1, svlf.FP32)
    feats = torch.zeros(tree.n_leaves, 8, device="cuda")
    params = torch.zeros(I.MLPShape(8, 32, 1).n_params, device="cuda")
    _, _, hits, tio, _ = svlf.svlf_render_rays(tree, feats, params, net, torch.from_numpy(probe).cuda(), K,
                                               want_hits=True)
    torch.cuda.synchronize()
    assert svlf.svlf_get_device_status() == 0
    oh = O.trace(O.build_octree(ref, L), probe, K)
    compare_hits(oh, hits.cpu().numpy(), tio.cpu().numpy())
    assert (oh.n > 0).sum() > 300


def test_empty_and_invalid_depths():
    from paper_2205_07058_b300 import svlf
    rays = torch.from_numpy(I.pinhole_rays(0.4, 0.3, 16, 16))
    depth = torch.full((rays.shape[0],), float("nan"))
    depth[:10] = -1.0
    tree = svlf.Octree.from_depth(rays, depth, 6)
    assert tree.n_leaves == 0
    rgb, dep, _, _, _ = svlf.svlf_render_rays(tree, torch.zeros(1, 8, device="cuda"),
                                              torch.zeros(I.MLPShape(8, 32, 1).n_params, device="cuda"),
                                              svlf.Network(8, 32, 1, svlf.FP32), rays.cuda(), 4, bg=(0.25, 0.5, 1.0))
    assert torch.all(rgb.cpu() == torch.tensor([0.25, 0.5, 1.0])) and torch.all(dep == 0)
    with pytest.raises(svlf.SvlfError):
        svlf.Octree.from_depth(rays, depth, 11)


@pytest.mark.parametrize("L,n_sph,n_box", [(2, 1, 0), (3, 2, 1), (6, 8, 3), (9, 24, 8), (10, 8, 4)])
def test_leaf_list_build_on_gpu_equals_host_construction(L, n_sph, n_box):
    """svlf_build_octree (on the GPU) and svlf_build_octree_host give the same
    arrays: sizes, leaf coordinates in rank order, the parent index entry for
    entry; the leaf list is shuffled and holds duplicates."""
    from paper_2205_07058_b300 import svlf
    rng = np.random.default_rng(300 + L)
    sc = I.make_scene(rng, L, n_sph, n_box)
    ijk = sc.leaf_ijk[rng.permutation(sc.n_leaves)]
    ijk = np.concatenate([ijk, ijk[: max(1, sc.n_leaves // 7)]]).astype(np.int32)
    gpu = svlf.Octree(torch.from_numpy(ijk), L)
    host = svlf.Octree(torch.from_numpy(ijk), L, host=True)
    torch.cuda.synchronize()
    assert gpu.n_leaves == host.n_leaves == sc.n_leaves
    assert gpu.info() == host.info()
    assert torch.equal(gpu.leaf_ijk(), host.leaf_ijk())
    assert np.array_equal(gpu.leaf_ijk().cpu().numpy(), sc.leaf_ijk)
    assert torch.equal(gpu.parent_index(), host.parent_index())


def test_leaf_list_build_rejects_out_of_range_and_handles_empty():
    from paper_2205_07058_b300 import svlf
    for bad in ([[0, 0, 4]], [[-1, 0, 0]], [[1, 1, 1], [0, 9, 0]]):
        with pytest.raises(svlf.SvlfError) as e:
            svlf.Octree(torch.tensor(bad, dtype=torch.int32), 2)
        assert e.value.code == svlf.SVLF_ERR_ARG
    empty = svlf.Octree(torch.zeros((0, 3), dtype=torch.int32), 5)
    assert empty.n_leaves == 0 and empty.info()["n_bricks"] == 0
    assert svlf.svlf_get_device_status() == 0
