"""Batched form: many scenes of uneven octree size in one launch per kernel,
against one call per scene and against the oracle; CUDA-graph capture."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2205_07058_b300 import inputs as I
from tests.gpu_common import requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]

SHAPE = I.MLPShape(32, 128, 3)


def _scenes(n=5, seed=40, shape=SHAPE):
    """Scenes of depth 6..9 with different primitive counts, features,
    networks and views (a few thousand rays each, some with none)."""
    from paper_2205_07058_b300 import svlf
    rng = np.random.default_rng(seed)
    SHAPE_ = shape
    out = []
    for i in range(n):
        depth = [6, 7, 8, 9, 7][i % 5]
        sc = I.make_scene(rng, depth, int(rng.integers(2, 10)), int(rng.integers(0, 4)))
        feats = I.make_features(rng, sc.n_leaves, 32)
        params = I.make_mlp(rng, SHAPE_, bias_std=0.2)
        az, el = I.random_view_angles(rng, 1)
        res = [48, 64, 32, 40, 0][i % 5]
        rays = I.pinhole_rays(az[0], el[0], res, res) if res else np.zeros((0, 6), np.float32)
        out.append(dict(scene=sc, feats=feats, params=params, rays=rays,
                        tree=svlf.Octree(torch.from_numpy(sc.leaf_ijk), depth)))
    return out


def _batch(scenes):
    from paper_2205_07058_b300 import svlf
    return [svlf.BatchScene(s["tree"], torch.from_numpy(s["feats"]).cuda(), torch.from_numpy(s["params"]).cuda(),
                            torch.from_numpy(s["rays"]).cuda()) for s in scenes]


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_batched_render_matches_single_calls_and_oracle(prec):
    from paper_2205_07058_b300 import svlf
    scenes = _scenes()
    net = svlf.Network(32, 128, 3, svlf.PRECISIONS[prec])
    bg = (0.1, 0.2, 0.3)
    batch = _batch(scenes)
    svlf.svlf_render_rays_batched(batch, net, 8, bg=bg)
    torch.cuda.synchronize()
    assert svlf.svlf_get_device_status() == 0
    for s, b in zip(scenes, batch):
        if s["rays"].shape[0] == 0:
            assert b.rgb.shape == (0, 3)
            continue
        rgb, depth, _, _, _ = svlf.svlf_render_rays(b.tree, b.features, b.params, net, b.rays, 8, bg=bg)
        torch.testing.assert_close(b.rgb, rgb, rtol=0, atol=1e-6)
        torch.testing.assert_close(b.depth, depth, rtol=0, atol=1e-6)
        tree = O.build_octree(s["scene"].leaf_ijk, s["scene"].depth)
        emu = O.render(tree, s["feats"], s["params"], O.layer_dims(32, 128, 3), s["rays"], 8, bg=bg, bf16=prec)
        ok = ~emu.hits.degenerate
        assert np.abs(b.rgb.cpu().numpy()[ok] - emu.rgb[ok]).max() <= 2e-3


@pytest.mark.parametrize("prec,nh", [("bf16", 3), ("fp16", 3), ("bf16", 4)])
def test_batched_backward_matches_single_calls(prec, nh):
    """nh = 4 streams the hidden layers' weights through two shared-memory
    slots, across scene changes inside a CTA's range of tiles."""
    from paper_2205_07058_b300 import svlf
    scenes = _scenes(seed=41, shape=I.MLPShape(32, 128, nh))
    net = svlf.Network(32, 128, nh, svlf.PRECISIONS[prec])
    batch = _batch(scenes)
    ws = svlf.svlf_render_rays_batched(batch, net, 8)
    rng = np.random.default_rng(0)
    for b in batch:
        n = b.rays.shape[0]
        b.d_rgb = torch.from_numpy(rng.standard_normal((n, 3)).astype(np.float32) * 1e-3).cuda()
        b.d_depth = torch.from_numpy(rng.standard_normal(n).astype(np.float32) * 1e-4).cuda()
        b.d_features = torch.zeros_like(b.features)
        b.d_params = torch.zeros_like(b.params)
    svlf.svlf_render_rays_backward_batched(batch, net, 8, (0, 0, 0), ws)
    torch.cuda.synchronize()
    assert svlf.svlf_get_device_status() == 0
    for b in batch:
        if b.rays.shape[0] == 0:
            assert torch.all(b.d_params == 0)
            continue
        _, _, _, _, w1 = svlf.svlf_render_rays(b.tree, b.features, b.params, net, b.rays, 8)
        df = torch.zeros_like(b.features)
        dp = torch.zeros_like(b.params)
        svlf.svlf_render_rays_backward(b.tree, b.features, b.params, net, b.rays, 8, (0, 0, 0), b.d_rgb,
                                       b.d_depth, df, dp, w1)
        torch.cuda.synchronize()
        assert (torch.linalg.norm(b.d_params - dp) / torch.linalg.norm(dp)).item() <= 1e-4
        assert (torch.linalg.norm(b.d_features - df) / torch.linalg.norm(df)).item() <= 1e-4


@pytest.mark.parametrize("prec,nh", [("bf16", 3), ("fp16", 3), ("bf16", 4)])
def test_batched_backward_matches_oracle_adjoint(prec, nh):
    """The batched backward against the oracle's adjoint scene by scene (the
    oracle rounding activations and weights to the same 16-bit format), on the
    training loss of each scene's own rays (L2 colour + 0.1 masked L1 depth,
    mean over the scene's rays). Near-degenerate rays are dropped beforehand,
    and the depth term is masked where |D - D*| is within rounding noise (the
    L1 kink). Tolerance: the single-scene tensor-core gradient tests' 1e-2
    normwise."""
    from paper_2205_07058_b300 import svlf
    shape = I.MLPShape(32, 128, nh)
    dims = O.layer_dims(32, 128, nh)
    scenes = _scenes(seed=49, shape=shape)
    trees_o = []
    for s in scenes:
        t = O.build_octree(s["scene"].leaf_ijk, s["scene"].depth)
        trees_o.append(t)
        if s["rays"].shape[0]:
            s["rays"] = s["rays"][~O.trace(t, s["rays"], 8).degenerate]
    net = svlf.Network(32, 128, nh, svlf.PRECISIONS[prec])
    batch = _batch(scenes)
    ws = svlf.svlf_render_rays_batched(batch, net, 8)
    rng = np.random.default_rng(11)
    refs = []
    for s, t, b in zip(scenes, trees_o, batch):
        n = s["rays"].shape[0]
        rgb_t = rng.uniform(0, 1, size=(n, 3)).astype(np.float32)
        depth_t, mask = I.analytic_depth(s["rays"], s["scene"])
        r = O.render(t, s["feats"], s["params"], dims, s["rays"], 8, bf16=prec)
        mask = np.where(np.abs(r.depth - depth_t) < 1e-4, 0.0, mask).astype(np.float32)
        b.d_rgb = torch.empty((n, 3), device="cuda")
        b.d_depth = torch.empty((n,), device="cuda")
        b.d_features = torch.zeros_like(b.features)
        b.d_params = torch.zeros_like(b.params)
        if n:
            loss = torch.zeros(1, dtype=torch.float64, device="cuda")
            svlf.svlf_loss(b.rgb, b.depth, torch.from_numpy(rgb_t).cuda(), torch.from_numpy(depth_t).cuda(),
                           torch.from_numpy(mask).cuda(), 0.1, b.d_rgb, b.d_depth, loss)
            refs.append(O.backward(t, r, s["params"], dims, rgb_t.astype(np.float64), depth_t.astype(np.float64),
                                   mask.astype(np.float64), (0, 0, 0), t.n_leaves, 32, bf16=prec)[:2])
        else:
            refs.append(None)
    svlf.svlf_render_rays_backward_batched(batch, net, 8, (0, 0, 0), ws)
    torch.cuda.synchronize()
    assert svlf.svlf_get_device_status() == 0
    checked = 0
    for b, ref in zip(batch, refs):
        if ref is None:
            assert torch.all(b.d_params == 0) and torch.all(b.d_features == 0)
            continue
        dfr, dpr = ref
        df, dp = b.d_features.cpu().numpy().astype(np.float64), b.d_params.cpu().numpy().astype(np.float64)
        assert np.isfinite(df).all() and np.isfinite(dp).all()
        assert np.any(dpr)  # the seed gives every scene samples with tau > 0
        e_f = np.linalg.norm(df - dfr) / np.linalg.norm(dfr)
        e_p = np.linalg.norm(dp - dpr) / np.linalg.norm(dpr)
        assert e_f <= 1e-2 and e_p <= 1e-2, (e_f, e_p)
        checked += 1
    assert checked == 4


def test_batched_render_under_cuda_graph():
    from paper_2205_07058_b300 import svlf
    scenes = _scenes(seed=42)
    net = svlf.Network(32, 128, 3, svlf.BF16)
    batch = _batch(scenes)
    ws = svlf.svlf_render_rays_batched(batch, net, 8)  # allocates outputs, warms up
    torch.cuda.synchronize()
    ref = [b.rgb.clone() for b in batch]
    for b in batch:
        b.rgb.zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            svlf.svlf_render_rays_batched(batch, net, 8, workspace=ws)
    for _ in range(2):
        for b in batch:
            b.rgb.zero_()
        g.replay()
        torch.cuda.synchronize()
        for b, r in zip(batch, ref):
            torch.testing.assert_close(b.rgb, r, rtol=0, atol=1e-6)


def test_batched_trace_refill_shapes_agree():
    """Warps that mix rays of several chunks and scenes (refill below 32) give
    the same images, bit for bit, as warps that finish a chunk first."""
    from paper_2205_07058_b300 import svlf
    scenes = _scenes(seed=41)
    net = svlf.Network(32, 128, 3, svlf.BF16)
    out = {}
    try:
        for refill in (32, 16, 1, 0):
            svlf.svlf_set_tuning(trace_refill=refill, trace_budget=4)
            batch = _batch(scenes)
            svlf.svlf_render_rays_batched(batch, net, 8)
            torch.cuda.synchronize()
            assert svlf.svlf_get_device_status() == 0
            out[refill] = [(b.rgb.clone(), b.depth.clone()) for b in batch]
    finally:
        svlf.svlf_set_tuning()
    for refill in (16, 1, 0):
        for (c0, d0), (c1, d1) in zip(out[32], out[refill]):
            assert torch.equal(c0, c1) and torch.equal(d0, d1)


def test_scene_without_rays_may_omit_its_parameters():
    """A scene with no rays is skipped whole: its parameter pointer may be null."""
    from paper_2205_07058_b300 import svlf
    scenes = _scenes(n=3, seed=43)
    net = svlf.Network(32, 128, 3, svlf.BF16)
    batch = _batch(scenes)
    ref = [None] * len(batch)
    svlf.svlf_render_rays_batched(batch, net, 8)
    torch.cuda.synchronize()
    ref = [(b.rgb.clone(), b.depth.clone()) for b in batch]
    empty = svlf.BatchScene(batch[0].tree, batch[0].features, None, torch.zeros((0, 6), device="cuda"))
    batch2 = [batch[0], empty, batch[1], batch[2]]
    for b in (batch[0], batch[1], batch[2]):
        b.rgb = None
        b.depth = None
    svlf.svlf_render_rays_batched(batch2, net, 8)
    torch.cuda.synchronize()
    assert svlf.svlf_get_device_status() == 0
    for (c0, d0), b in zip(ref, (batch2[0], batch2[2], batch2[3])):
        assert torch.equal(c0, b.rgb) and torch.equal(d0, b.depth)


def test_workspace_samples_batched_equals_per_scene_counts():
    from paper_2205_07058_b300 import svlf
    scenes = _scenes(seed=44)
    net = svlf.Network(32, 128, 3, svlf.BF16)
    batch = _batch(scenes)
    ws = svlf.svlf_render_rays_batched(batch, net, 8)
    torch.cuda.synchronize()
    total = svlf.svlf_workspace_samples_batched(ws, net, batch, 8)
    expect = 0
    for b in batch:
        n = b.rays.shape[0]
        if n == 0:
            continue
        _, _, hits, _, _ = svlf.svlf_render_rays(b.tree, b.features, b.params, net, b.rays, 8, want_hits=True)
        expect += int((hits >= 0).sum())
    assert total == expect > 0


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_scene_without_output_gradients_takes_no_part(prec):
    """A training step's two kinds of rays in one batched call: rays that are
    only rendered (a scene whose d_rgb and d_depth are NULL) and rays that are
    trained on, over the same octree, features and network. The rendered
    outputs equal single calls, the gradients equal the single-scene backward
    of the trained rays alone (up to the order of float32 atomic additions),
    and a scene with exactly one of d_rgb, d_depth is refused."""
    from paper_2205_07058_b300 import svlf
    rng = np.random.default_rng(52)
    sc = I.make_scene(rng, 8, 12, 4)
    feats = torch.from_numpy(I.make_features(rng, sc.n_leaves, 32)).cuda()
    params = torch.from_numpy(I.make_mlp(rng, SHAPE, bias_std=0.2)).cuda()
    tree = svlf.Octree(torch.from_numpy(sc.leaf_ijk), 8)
    az, el = I.random_view_angles(rng, 3)
    view = torch.from_numpy(np.concatenate([I.pinhole_rays(az[v], el[v], 96, 96) for v in range(2)])).cuda()
    train = torch.from_numpy(I.training_rays(np.random.default_rng(3), 3, 128, 6000, az, el)).cuda()
    net = svlf.Network(32, 128, 3, svlf.PRECISIONS[prec])
    K = 8
    nt = train.shape[0]
    rgb_t = torch.from_numpy(np.random.default_rng(4).uniform(0, 1, size=(nt, 3)).astype(np.float32)).cuda()
    depth_t, mask = I.analytic_depth(train.cpu().numpy(), sc)
    depth_t, mask = torch.from_numpy(depth_t).cuda(), torch.from_numpy(mask).cuda()

    def loss_grads(rgb, depth):
        d_rgb, d_depth = torch.empty_like(rgb), torch.empty_like(depth)
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        svlf.svlf_loss(rgb, depth, rgb_t, depth_t, mask, 0.1, d_rgb, d_depth, loss)
        return d_rgb, d_depth

    # one call for both: the view scene takes no part in the backward
    batch = [svlf.BatchScene(tree, feats, params, view), svlf.BatchScene(tree, feats, params, train)]
    ws = svlf.svlf_render_rays_batched(batch, net, K)
    batch[1].d_rgb, batch[1].d_depth = loss_grads(batch[1].rgb, batch[1].depth)
    batch[1].d_features = torch.zeros_like(feats)
    batch[1].d_params = torch.zeros_like(params)
    svlf.svlf_render_rays_backward_batched(batch, net, K, (0.0, 0.0, 0.0), ws)
    torch.cuda.synchronize()
    assert svlf.svlf_get_device_status() == 0
    # single calls
    per = svlf.svlf_workspace_scene_samples(ws, net, batch, K)
    assert sum(per) == svlf.svlf_workspace_samples_batched(ws, net, batch, K)
    vrgb, vdepth, _, _, vws = svlf.svlf_render_rays(tree, feats, params, net, view, K)
    trgb, tdepth, _, _, tws = svlf.svlf_render_rays(tree, feats, params, net, train, K)
    assert per == [svlf.svlf_workspace_samples(vws, net, view.shape[0], K),
                   svlf.svlf_workspace_samples(tws, net, train.shape[0], K)]
    d_rgb, d_depth = loss_grads(trgb, tdepth)
    df, dp = torch.zeros_like(feats), torch.zeros_like(params)
    svlf.svlf_render_rays_backward(tree, feats, params, net, train, K, (0.0, 0.0, 0.0), d_rgb, d_depth, df, dp, tws)
    torch.cuda.synchronize()
    torch.testing.assert_close(batch[0].rgb, vrgb, rtol=0, atol=1e-6)
    torch.testing.assert_close(batch[0].depth, vdepth, rtol=0, atol=1e-6)
    torch.testing.assert_close(batch[1].rgb, trgb, rtol=0, atol=1e-6)
    for a, b in ((batch[1].d_features, df), (batch[1].d_params, dp)):
        assert torch.linalg.norm(b) > 0
        e = (torch.linalg.norm(a - b) / torch.linalg.norm(b)).item()
        assert e <= 1e-5, e
    # exactly one of the two output gradients: refused
    batch[0].d_rgb = torch.zeros_like(batch[0].rgb)
    with pytest.raises(svlf.SvlfError) as err:
        svlf.svlf_render_rays_backward_batched(batch, net, K, (0.0, 0.0, 0.0), ws)
    assert err.value.code == svlf.SVLF_ERR_ARG
