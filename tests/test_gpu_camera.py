"""Pinhole rays generated on the device against the host generator the
workloads use, and a render from them against the oracle on the same rays."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2205_07058_b300 import inputs as I
from tests.gpu_common import compare_hits, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


def _cams(views, fov_deg=40.0):
    from paper_2205_07058_b300 import svlf
    basis = [I.camera_basis(a, e) for a, e in views]
    eye, fwd, right, up = (np.stack([b[k] for b in basis]) for k in range(4))
    return svlf.cameras(eye, fwd, right, up, math.tan(math.radians(fov_deg) / 2.0))


@pytest.mark.parametrize("w,h", [(64, 64), (97, 31)])
def test_pinhole_rays_match_host_generator(w, h):
    from paper_2205_07058_b300 import svlf
    views = [(math.radians(30.0), math.radians(20.0)), (math.radians(200.0), math.radians(-35.0)),
             (math.radians(123.0), math.radians(70.0))]
    cams = _cams(views)
    rays = svlf.svlf_pinhole_rays(cams, w, h).cpu().numpy()
    ref = np.concatenate([I.pinhole_rays(a, e, w, h) for a, e in views])
    assert rays.shape == ref.shape
    assert np.array_equal(rays[:, :3], ref[:, :3])
    assert np.abs(rays[:, 3:] - ref[:, 3:]).max() <= 2e-6
    assert np.abs(np.linalg.norm(rays[:, 3:].astype(np.float64), axis=1) - 1.0).max() <= 1e-6


def test_many_views_and_bad_arguments():
    from paper_2205_07058_b300 import svlf
    views = [(0.1 * i, 0.01 * i) for i in range(70)]  # more than one launch's worth of cameras
    rays = svlf.svlf_pinhole_rays(_cams(views), 8, 4).cpu().numpy()
    ref = np.concatenate([I.pinhole_rays(a, e, 8, 4) for a, e in views])
    assert np.abs(rays - ref).max() <= 2e-6
    with pytest.raises(svlf.SvlfError):
        svlf.svlf_pinhole_rays(_cams(views[:1]), 0, 4)


def test_render_from_device_rays_matches_oracle(tiny):
    from paper_2205_07058_b300 import svlf
    rays_d = svlf.svlf_pinhole_rays(_cams([(math.radians(30.0), math.radians(20.0))]), 64, 64)
    rays = rays_d.cpu().numpy()
    tree = svlf.Octree(torch.from_numpy(tiny.scene.leaf_ijk), tiny.scene.depth)
    f = torch.from_numpy(tiny.features).cuda()
    p = torch.from_numpy(tiny.params).cuda()
    net = svlf.Network(16, 64, 2, svlf.FP32)
    rgb, depth, hits, tio, _ = svlf.svlf_render_rays(tree, f, p, net, rays_d, 4, want_hits=True)
    torch.cuda.synchronize()
    oh = O.trace(O.build_octree(tiny.scene.leaf_ijk, tiny.scene.depth), rays, 4)
    compare_hits(oh, hits.cpu().numpy(), tio.cpu().numpy())
    ref = O.render(O.build_octree(tiny.scene.leaf_ijk, tiny.scene.depth), tiny.features, tiny.params,
                   O.layer_dims(16, 64, 2), rays, 4)
    ok = ~ref.hits.degenerate
    assert np.abs(rgb.cpu().numpy()[ok] - ref.rgb[ok]).max() <= 1e-5
