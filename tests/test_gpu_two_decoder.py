"""The paper's two-decoder SVLF (vertex features, trilinear interpolation,
F^T -> tau, eta; F^C at the surface point) on the GPU against the oracle."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from oracle import two_decoder as T2
from paper_2205_07058_b300 import inputs as I
from tests.gpu_common import compare_hits, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


def _net(rng, dims, bias_std=0.2):
    out = []
    for o, i in dims:
        out.append(rng.standard_normal(o * i) * math.sqrt(2.0 / i))
        out.append(rng.standard_normal(o) * bias_std)
    return np.concatenate(out).astype(np.float32)


def _setup(seed, depth, n_sph, n_box, views, res, ft=64, fc=32, ht=128, nt=1, hc=128, nc=3):
    from paper_2205_07058_b300 import svlf
    rng = np.random.default_rng(seed)
    sc = I.make_scene(rng, depth, n_sph, n_box)
    tree_o = O.build_octree(sc.leaf_ijk, depth)
    vt = T2.vertex_table(tree_o)
    zt = I.make_features(rng, vt.n_vertices, ft)
    zc = I.make_features(rng, vt.n_vertices, fc)
    dt, dc = T2.dims_t(ft, ht, nt), T2.dims_c(fc, hc, nc)
    pt, pc = _net(rng, dt), _net(rng, dc)
    az, el = I.random_view_angles(rng, views)
    rays = np.concatenate([I.pinhole_rays(az[v], el[v], res, res) for v in range(views)])
    tree = svlf.Octree(torch.from_numpy(sc.leaf_ijk), depth)
    return dict(sc=sc, tree_o=tree_o, vt=vt, zt=zt, zc=zc, dt=dt, dc=dc, pt=pt, pc=pc, rays=rays, tree=tree,
                shape=(ft, fc, ht, nt, hc, nc))


@pytest.fixture(scope="module")
def small():
    return _setup(1007, 7, 10, 4, 2, 96)


def test_vertex_table_matches_oracle(small):
    n = small["tree"].build_vertices()
    assert n == small["vt"].n_vertices
    lv = small["tree"].leaf_vertices().cpu().numpy()
    assert np.array_equal(lv, small["vt"].leaf_vertices)


def _gpu(w, prec, K, bg=(0.0, 0.0, 0.0), feat_bf16=False, params=None, image_width=0):
    from paper_2205_07058_b300 import svlf
    w["tree"].build_vertices()
    ft, fc, ht, nt, hc, nc = w["shape"]
    net = svlf.TwoDecoder(ft, fc, ht, nt, hc, nc, svlf.PRECISIONS[prec],
                          svlf.FEAT_BF16 if feat_bf16 else svlf.FEAT_F32)
    cast = (lambda a: torch.from_numpy(a).to(torch.bfloat16).cuda()) if feat_bf16 else (lambda a: torch.from_numpy(a).cuda())
    pt, pc = params if params is not None else (w["pt"], w["pc"])
    rgb, depth, hits, tio, _ = svlf.svlf_render_rays_two_decoder(
        w["tree"], cast(w["zt"]), cast(w["zc"]), torch.from_numpy(pt).cuda(), torch.from_numpy(pc).cuda(),
        net, torch.from_numpy(w["rays"]).cuda(), K, bg=bg, want_hits=True, image_width=image_width)
    torch.cuda.synchronize()
    assert svlf.svlf_get_device_status() == 0
    return rgb.cpu().numpy(), depth.cpu().numpy(), hits.cpu().numpy(), tio.cpu().numpy()


def test_tile_walk_is_bit_identical(small):
    """The views walked in 8 x 4 pixel tiles (image_width 96): colours, depth,
    hit lists and segments bit-identical to the walk in the rays' own order
    (the samples reach the two passes in another order only)."""
    a = _gpu(small, "bf16", 6, (0.1, 0.2, 0.3))
    b = _gpu(small, "bf16", 6, (0.1, 0.2, 0.3), image_width=96)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("prec,feat_bf16", [("bf16", False), ("fp16", False), ("bf16", True)])
def test_render_matches_emulating_oracle(small, prec, feat_bf16):
    w = small
    K = 6
    bg = (0.1, 0.2, 0.3)
    rgb, depth, hits, tio = _gpu(w, prec, K, bg, feat_bf16)
    zt, zc = w["zt"], w["zc"]
    if feat_bf16:  # the stored values the GPU reads
        zt = torch.from_numpy(zt).to(torch.bfloat16).float().numpy()
        zc = torch.from_numpy(zc).to(torch.bfloat16).float().numpy()
    ref = T2.render2(w["tree_o"], w["vt"], zt, zc, w["pt"], w["pc"], w["dt"], w["dc"], w["rays"], K, bg=bg,
                     lowp=prec)
    n_ok, n_deg, _ = compare_hits(ref.hits, hits, tio)
    ok = ~ref.hits.degenerate
    assert (ref.hits.n[ok] > 0).sum() > 1500
    err = np.abs(rgb[ok] - ref.rgb[ok]).max(axis=1)
    derr = np.abs(depth[ok] - ref.depth[ok]) / (1 + ref.depth[ok])
    f64 = T2.render2(w["tree_o"], w["vt"], zt, zc, w["pt"], w["pc"], w["dt"], w["dc"], w["rays"], K, bg=bg,
                     hits=ref.hits)
    print(prec, "bf16 storage" if feat_bf16 else "fp32 storage", "colour max / p99", err.max(), np.quantile(err, 0.99),
          "depth max", derr.max(), "| vs FP64: colour max", np.abs(rgb[ok] - f64.rgb[ok]).max())
    assert err.max() <= 2e-3 and derr.max() <= 2e-3
    assert np.quantile(err, 0.99) <= 2e-4


@pytest.mark.parametrize("ft,fc,feat_bf16", [(8, 8, False), (8, 8, True), (24, 40, False), (24, 40, True)])
def test_render_feature_widths(ft, fc, feat_bf16):
    """The cooperative corner gather at the widths where its lane groups change
    shape: rows of 1 and 2 16-byte segments (1 and 2 lanes per sample), 3, 5
    and 6 segments (groups of 4 and 8 with idle lanes) and 10 (lanes taking a
    second segment), in float32 and bfloat16 storage."""
    w = _setup(1011, 6, 6, 3, 1, 80, ft=ft, fc=fc, ht=64, nt=1, hc=64, nc=2)
    K = 5
    rgb, depth, hits, tio = _gpu(w, "bf16", K, (0.0, 0.0, 0.0), feat_bf16)
    zt, zc = w["zt"], w["zc"]
    if feat_bf16:
        zt = torch.from_numpy(zt).to(torch.bfloat16).float().numpy()
        zc = torch.from_numpy(zc).to(torch.bfloat16).float().numpy()
    ref = T2.render2(w["tree_o"], w["vt"], zt, zc, w["pt"], w["pc"], w["dt"], w["dc"], w["rays"], K, lowp="bf16")
    compare_hits(ref.hits, hits, tio)
    ok = ~ref.hits.degenerate
    assert (ref.hits.n[ok] > 0).sum() > 300
    err = np.abs(rgb[ok] - ref.rgb[ok]).max(axis=1)
    derr = np.abs(depth[ok] - ref.depth[ok]) / (1 + ref.depth[ok])
    print(ft, fc, "bf16 storage" if feat_bf16 else "fp32 storage", "colour max", err.max(), "depth max", derr.max())
    assert err.max() <= 2e-3 and derr.max() <= 2e-3


def test_constant_networks_closed_form(small):
    """Zero weights: every hit has tau = relu(b_tau), eta = sigmoid(b_eta),
    c = sigmoid(b_c), so the image depends only on the hit segments."""
    w = small
    K = 5
    def zero_net(dims, out_b):
        parts = []
        for li, (o, i) in enumerate(dims):
            parts.append(np.zeros(o * i, np.float32))
            parts.append(np.asarray(out_b, np.float32) if li + 1 == len(dims) else np.zeros(o, np.float32))
        return np.concatenate(parts)
    pt = zero_net(w["dt"], [0.8, -0.7])
    pc = zero_net(w["dc"], [0.3, -1.2, 2.0])
    bg = (0.5, 0.5, 0.5)
    rgb, depth, hits, tio = _gpu(w, "bf16", K, bg, params=(pt, pc))
    ref = T2.render2(w["tree_o"], w["vt"], w["zt"], w["zc"], pt, pc, w["dt"], w["dc"], w["rays"], K, bg=bg)
    ok = ~ref.hits.degenerate
    np.testing.assert_allclose(rgb[ok], ref.rgb[ok], rtol=0, atol=2e-6)
    np.testing.assert_allclose(depth[ok], ref.depth[ok], rtol=0, atol=2e-6 * (1 + ref.depth[ok].max()))


def test_many_tiles_per_cta_sampled():
    """Depth 9 scene, 2 views of 800^2 (1.28 M rays): every CTA runs many
    tiles; 3000 sampled rays against the bf16-emulating oracle."""
    w = _setup(1008, 9, 48, 24, 2, 800)
    K = 8
    rgb, depth, hits, tio = _gpu(w, "bf16", K)
    sample = np.random.default_rng(3).choice(w["rays"].shape[0], 3000, replace=False)
    ref = T2.render2(w["tree_o"], w["vt"], w["zt"], w["zc"], w["pt"], w["pc"], w["dt"], w["dc"],
                     w["rays"][sample], K, lowp="bf16")
    ok = ~ref.hits.degenerate
    assert np.array_equal(hits[sample][ok], ref.hits.rank[ok])
    assert (ref.hits.n[ok] > 0).sum() > 300
    err = np.abs(rgb[sample][ok] - ref.rgb[ok]).max()
    derr = (np.abs(depth[sample][ok] - ref.depth[ok]) / (1 + ref.depth[ok])).max()
    assert err <= 2e-3 and derr <= 2e-3, (err, derr)


def test_argument_errors():
    from paper_2205_07058_b300 import svlf
    rng = np.random.default_rng(9)
    ijk = torch.from_numpy(np.unique(rng.integers(0, 8, size=(40, 3)), axis=0).astype(np.int32))
    tree = svlf.Octree(ijk, 3)
    net = svlf.TwoDecoder(16, 8, 32, 1, 32, 1)
    zt = torch.zeros((1000, 16), device="cuda")
    zc = torch.zeros((1000, 8), device="cuda")
    p = torch.zeros(10000, device="cuda")
    rays = torch.from_numpy(I.pinhole_rays(0.3, 0.2, 8, 8)).cuda()
    with pytest.raises(svlf.SvlfError) as e:  # vertex table not built
        svlf.svlf_render_rays_two_decoder(tree, zt, zc, p, p, net, rays, 4)
    assert e.value.code == svlf.SVLF_ERR_ARG
    tree.build_vertices()
    with pytest.raises(svlf.SvlfError) as e:
        svlf.svlf_render_rays_two_decoder(tree, zt, zc, p, p, svlf.TwoDecoder(16, 8, 32, 1, 32, 1, svlf.FP32), rays,
                                          4)
    assert e.value.code == svlf.SVLF_ERR_UNSUPPORTED
    with pytest.raises(svlf.SvlfError) as e:
        svlf.svlf_render_rays_two_decoder(tree, torch.zeros((1000, 12), device="cuda"), zc, p, p,
                                          svlf.TwoDecoder(12, 8, 32, 1, 32, 1), rays, 4)
    assert e.value.code == svlf.SVLF_ERR_UNSUPPORTED
    # a table whose dtype or width disagrees with the descriptor is refused before any launch
    with pytest.raises(ValueError):
        svlf.svlf_render_rays_two_decoder(tree, zt.bfloat16(), zc.bfloat16(), p, p, net, rays, 4)
    with pytest.raises(ValueError):
        svlf.svlf_render_rays_two_decoder(tree, zt, zt, p, p, net, rays, 4)


def _rel(g, r):
    return float(np.linalg.norm(g - r) / np.linalg.norm(r))


@pytest.mark.parametrize("prec,ft,fc,feat_bf16", [("bf16", 32, 16, False), ("fp16", 32, 16, False),
                                                  ("bf16", 64, 40, False), ("bf16", 32, 16, True)])
def test_backward_matches_oracle_adjoint(prec, ft, fc, feat_bf16):
    """Gradients of Z^T, Z^C and both networks through the GPU render + loss +
    backward against the oracle's adjoint with the same operand rounding.
    Near-degenerate rays are dropped and the L1 depth term is masked where
    |D - D*| is within float32 noise (its kink). The shapes cover the corner
    scatter's 32-column blocks: one block, two full blocks (Z^T 64) and a
    partly filled second block (Z^C 40); bfloat16 tables are read as such and
    their gradients stay float32."""
    from paper_2205_07058_b300 import svlf
    rng = np.random.default_rng(1009)
    sc = I.make_scene(rng, 7, 10, 4)
    tree_o = O.build_octree(sc.leaf_ijk, 7)
    vt = T2.vertex_table(tree_o)
    dt, dc = T2.dims_t(ft, 64, 1), T2.dims_c(fc, 64, 2)
    zt = (rng.standard_normal((vt.n_vertices, ft)) * 0.3).astype(np.float32)
    zc = (rng.standard_normal((vt.n_vertices, fc)) * 0.3).astype(np.float32)
    if feat_bf16:  # the oracle sees the tables the GPU reads
        zt = torch.from_numpy(zt).to(torch.bfloat16).float().numpy()
        zc = torch.from_numpy(zc).to(torch.bfloat16).float().numpy()
    pt, pc = _net(rng, dt, 0.3), _net(rng, dc, 0.3)
    az, el = I.random_view_angles(rng, 40)
    rays = I.training_rays(np.random.default_rng(2), 40, 200, 10000, az, el)
    K = 6
    rays = rays[~O.trace(tree_o, rays, K).degenerate]
    rgb_t = np.random.default_rng(3).uniform(0, 1, size=(rays.shape[0], 3)).astype(np.float32)
    depth_t, mask = I.analytic_depth(rays, sc)
    ref64 = T2.render2(tree_o, vt, zt, zc, pt, pc, dt, dc, rays, K)
    mask = np.where(np.abs(ref64.depth - depth_t) < 1e-4, 0.0, mask).astype(np.float32)
    assert (ref64.hits.n > 0).sum() > 1000
    # GPU
    tree = svlf.Octree(torch.from_numpy(sc.leaf_ijk), 7)
    tree.build_vertices()
    net = svlf.TwoDecoder(ft, fc, 64, 1, 64, 2, svlf.PRECISIONS[prec],
                          svlf.FEAT_BF16 if feat_bf16 else svlf.FEAT_F32)
    g = {k: torch.from_numpy(v).cuda() for k, v in dict(zt=zt, zc=zc, pt=pt, pc=pc, rays=rays).items()}
    if feat_bf16:
        g["zt_k"], g["zc_k"] = g["zt"].bfloat16(), g["zc"].bfloat16()
    else:
        g["zt_k"], g["zc_k"] = g["zt"], g["zc"]
    rgb, depth, _, _, ws = svlf.svlf_render_rays_two_decoder(tree, g["zt_k"], g["zc_k"], g["pt"], g["pc"], net,
                                                             g["rays"], K)
    d_rgb, d_depth = torch.empty_like(rgb), torch.empty_like(depth)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    svlf.svlf_loss(rgb, depth, torch.from_numpy(rgb_t).cuda(), torch.from_numpy(depth_t).cuda(),
                   torch.from_numpy(mask).cuda(), 0.1, d_rgb, d_depth, loss)
    grads = {k: torch.zeros_like(g[k]) for k in ("zt", "zc", "pt", "pc")}
    svlf.svlf_render_rays_backward_two_decoder(tree, g["zt_k"], g["zc_k"], g["pt"], g["pc"], net, g["rays"], K,
                                               (0.0, 0.0, 0.0), d_rgb, d_depth, grads["zt"], grads["zc"],
                                               grads["pt"], grads["pc"], ws)
    torch.cuda.synchronize()
    assert svlf.svlf_get_device_status() == 0
    gpu = {k: v.cpu().numpy() for k, v in grads.items()}
    # oracle adjoint with the same rounding, and in FP64
    res = {}
    for lowp in (prec, False):
        r = T2.render2(tree_o, vt, zt, zc, pt, pc, dt, dc, rays, K, lowp=lowp, hits=ref64.hits)
        res[lowp] = T2.backward2(tree_o, vt, r, zc, pt, pc, dt, dc, rgb_t, depth_t, mask, (0, 0, 0), ft, fc,
                                 lowp=lowp)
    names = ["zt", "zc", "pt", "pc"]
    errs = {n: _rel(gpu[n], res[prec][i]) for i, n in enumerate(names)}
    errs64 = {n: _rel(gpu[n], res[False][i]) for i, n in enumerate(names)}
    print(prec, "two-decoder gradients vs emulating oracle", errs, "| vs FP64", errs64)
    for n in names:
        assert errs[n] <= 2e-2, (n, errs[n])
    # every layer of both networks
    for flat, ref, dims in ((gpu["pt"], res[prec][2], dt), (gpu["pc"], res[prec][3], dc)):
        off = 0
        for o, i in dims:
            for m in (o * i, o):
                assert _rel(flat[off:off + m], ref[off:off + m]) <= 5e-2
                off += m


# ---------------------------------------------------------------- staged training (Sec. 4.4, Eq. 4)
def _staged_setup(seed=1010):
    from paper_2205_07058_b300 import svlf
    rng = np.random.default_rng(seed)
    sc = I.make_scene(rng, 7, 10, 4)
    tree_o = O.build_octree(sc.leaf_ijk, 7)
    vt = T2.vertex_table(tree_o)
    ft, fc = 32, 16
    dt, dc = T2.dims_t(ft, 64, 1), T2.dims_c(fc, 64, 2)
    zt = (rng.standard_normal((vt.n_vertices, ft)) * 0.3).astype(np.float32)
    zc = (rng.standard_normal((vt.n_vertices, fc)) * 0.3).astype(np.float32)
    pt, pc = _net(rng, dt, 0.3), _net(rng, dc, 0.3)
    az, el = I.random_view_angles(rng, 40)
    rays = I.training_rays(np.random.default_rng(2), 40, 200, 12000, az, el)
    rgb_t = np.random.default_rng(3).uniform(0, 1, size=(rays.shape[0], 3)).astype(np.float32)
    depth_t, mask = I.analytic_depth(rays, sc)
    tree = svlf.Octree(torch.from_numpy(sc.leaf_ijk), 7)
    tree.build_vertices()
    return dict(sc=sc, tree_o=tree_o, vt=vt, ft=ft, fc=fc, dt=dt, dc=dc, zt=zt, zc=zc, pt=pt, pc=pc, rays=rays,
                rgb_t=rgb_t, depth_t=depth_t, mask=mask, tree=tree)


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_surface_loss_matches_oracle(prec):
    """Stage 1: Eq. 4 over the rays' surface voxels (point lookup) and its
    gradients, against the oracle with the same operand rounding."""
    from paper_2205_07058_b300 import svlf
    w = _staged_setup()
    lam_eta, lam_tau = 0.8, 0.4
    net = svlf.TwoDecoder(w["ft"], w["fc"], 64, 1, 64, 2, svlf.PRECISIONS[prec])
    g = {k: torch.from_numpy(w[k]).cuda() for k in ("zt", "zc", "pt", "pc", "rays", "rgb_t", "depth_t", "mask")}
    grads = {k: torch.zeros_like(g[k]) for k in ("zt", "zc", "pt", "pc")}
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    ws = svlf.svlf_surface_loss_two_decoder(w["tree"], g["zt"], g["zc"], g["pt"], g["pc"], net, g["rays"], g["rgb_t"],
                                            g["depth_t"], g["mask"], lam_eta, lam_tau, loss, grads["zt"], grads["zc"],
                                            grads["pt"], grads["pc"])
    torch.cuda.synchronize()
    assert svlf.svlf_get_device_status() == 0
    n_gpu = svlf.svlf_workspace_samples(ws, svlf.Network(32, 64, 1, svlf.BF16), w["rays"].shape[0], 1)
    L, ss, _, ref = T2.surface_loss(w["tree_o"], w["vt"], w["zt"], w["zc"], w["pt"], w["pc"], w["dt"], w["dc"],
                                    w["rays"], w["rgb_t"], w["depth_t"], w["mask"], lam_eta, lam_tau, w["ft"], w["fc"],
                                    lowp=prec)
    assert ss.ray.size > 1000
    assert abs(n_gpu - ss.ray.size) <= max(2, ss.ray.size // 500)  # surface points on a voxel face may round apart
    print(prec, "surface samples", n_gpu, ss.ray.size, "loss", loss.item(), L)
    assert abs(loss.item() - L) <= 2e-3 * abs(L)
    for i, k in enumerate(("zt", "zc", "pt", "pc")):
        e = _rel(grads[k].cpu().numpy(), ref[i])
        print(prec, k, e)
        assert e <= 2e-2, (k, e)


@pytest.mark.parametrize("prec", ["bf16"])
def test_volume_stage_eta_term_matches_oracle(prec):
    """Stages 2-3: two-decoder render + the workload loss + the eta term on
    each ray's surface voxel among its hits; loss and gradients against the
    oracle (Z^C and F^C frozen as in stage 2: their gradients not asked for)."""
    from paper_2205_07058_b300 import svlf
    w = _staged_setup(1011)
    K = 6
    lam_eta = 0.7
    rays = w["rays"][~O.trace(w["tree_o"], w["rays"], K).degenerate]
    rgb_t = w["rgb_t"][:rays.shape[0]]
    depth_t, mask = I.analytic_depth(rays, w["sc"])
    ref64 = T2.render2(w["tree_o"], w["vt"], w["zt"], w["zc"], w["pt"], w["pc"], w["dt"], w["dc"], rays, K)
    mask = np.where(np.abs(ref64.depth - depth_t) < 1e-4, 0.0, mask).astype(np.float32)
    net = svlf.TwoDecoder(w["ft"], w["fc"], 64, 1, 64, 2, svlf.PRECISIONS[prec])
    g = {k: torch.from_numpy(v).cuda() for k, v in dict(zt=w["zt"], zc=w["zc"], pt=w["pt"], pc=w["pc"], rays=rays,
                                                        rgb_t=rgb_t, depth_t=depth_t, mask=mask).items()}
    rgb, depth, _, _, ws = svlf.svlf_render_rays_two_decoder(w["tree"], g["zt"], g["zc"], g["pt"], g["pc"], net,
                                                             g["rays"], K)
    d_rgb, d_depth = torch.empty_like(rgb), torch.empty_like(depth)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    svlf.svlf_loss(rgb, depth, g["rgb_t"], g["depth_t"], g["mask"], 0.1, d_rgb, d_depth, loss)
    svlf.svlf_eta_loss_two_decoder(w["tree"], net, g["rays"], K, g["depth_t"], g["mask"], lam_eta, loss, ws)
    gzt, gpt = torch.zeros_like(g["zt"]), torch.zeros_like(g["pt"])
    svlf.svlf_render_rays_backward_two_decoder(w["tree"], g["zt"], g["zc"], g["pt"], g["pc"], net, g["rays"], K,
                                               (0.0, 0.0, 0.0), d_rgb, d_depth, gzt, None, gpt, None, ws)
    torch.cuda.synchronize()
    assert svlf.svlf_get_device_status() == 0
    r = T2.render2(w["tree_o"], w["vt"], w["zt"], w["zc"], w["pt"], w["pc"], w["dt"], w["dc"], rays, K, lowp=prec,
                   hits=ref64.hits)
    Le, deta = T2.eta_term(r, depth_t, mask, lam_eta)
    L = O.loss(r.rgb, r.depth, rgb_t, depth_t, mask) + Le
    assert np.count_nonzero(deta) > 500
    print(prec, "loss", loss.item(), L, "eta term", Le)
    assert abs(loss.item() - L) <= 2e-3 * abs(L)
    ref = T2.backward2(w["tree_o"], w["vt"], r, w["zc"], w["pt"], w["pc"], w["dt"], w["dc"], rgb_t, depth_t, mask,
                       (0, 0, 0), w["ft"], w["fc"], lowp=prec, deta_direct=deta)
    ez, ep = _rel(gzt.cpu().numpy(), ref[0]), _rel(gpt.cpu().numpy(), ref[2])
    print(prec, "gradients: Z^T", ez, "F^T", ep)
    assert ez <= 2e-2 and ep <= 2e-2
