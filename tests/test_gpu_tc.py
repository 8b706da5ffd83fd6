"""tcgen05 tensor-core path: the operand-layout self-test against torch, and
the BF16 / FP16 render against the oracle (bf16-emulating and FP64)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2205_07058_b300 import inputs as I
from tests.gpu_common import gpu_inputs, net_for, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("N,K", [(128, 48), (64, 32), (32, 128), (256, 16)])
@pytest.mark.parametrize("a_mn,b_mn", [(False, False), (False, True), (True, True), (True, False)])
def test_mma_operand_layouts(dtype, N, K, a_mn, b_mn):
    from paper_2205_07058_b300 import svlf
    g = torch.Generator(device="cpu").manual_seed(N * 1000 + K)
    A = torch.randn(128, K, generator=g).to(dtype).cuda()
    B = torch.randn(N, K, generator=g).to(dtype).cuda()
    D = svlf.svlf_selftest_mma(A, B, a_mn, b_mn)
    ref = A.double() @ B.double().T
    torch.testing.assert_close(D.double(), ref, rtol=1e-5, atol=1e-4)
    assert svlf.svlf_get_device_status() == 0


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("N,K", [(128, 48), (128, 128), (16, 128), (64, 144), (256, 16)])
@pytest.mark.parametrize("b_mn", [False, True])
def test_mma_a_operand_in_tmem(dtype, N, K, b_mn):
    from paper_2205_07058_b300 import svlf
    g = torch.Generator(device="cpu").manual_seed(N * 1000 + K + 7)
    A = torch.randn(128, K, generator=g).to(dtype).cuda()
    B = torch.randn(N, K, generator=g).to(dtype).cuda()
    D = svlf.svlf_selftest_mma(A, B, False, b_mn, flags=32)
    ref = A.double() @ B.double().T
    torch.testing.assert_close(D.double(), ref, rtol=1e-5, atol=1e-4)
    assert svlf.svlf_get_device_status() == 0


def _render(w, precision, params, bg=(0.0, 0.0, 0.0)):
    from paper_2205_07058_b300 import svlf
    tree, f, p, r = gpu_inputs(w, params=params)
    rgb, depth, hits, _, _ = svlf.svlf_render_rays(tree, f, p, net_for(w, precision), r, w.K, bg=bg,
                                                   want_hits=True)
    torch.cuda.synchronize()
    assert svlf.svlf_get_device_status() == 0
    return rgb.cpu().numpy(), depth.cpu().numpy()


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_render_tensor_core_tiny(tiny, prec):
    from paper_2205_07058_b300 import svlf
    rng = np.random.default_rng(4)
    params = I.make_mlp(rng, tiny.mlp, bias_std=0.5)
    bg = (0.25, 0.5, 0.75)
    precision = svlf.BF16 if prec == "bf16" else svlf.FP16
    rgb, depth = _render(tiny, precision, params, bg)
    tree = O.build_octree(tiny.scene.leaf_ijk, tiny.scene.depth)
    dims = O.layer_dims(16, 64, 2)
    ref64 = O.render(tree, tiny.features, params, dims, tiny.rays, tiny.K, bg=bg)
    ok = ~ref64.hits.degenerate
    if prec == "bf16":
        emu = O.render(tree, tiny.features, params, dims, tiny.rays, tiny.K, bg=bg, bf16=True)
        e_emu = np.abs(rgb[ok] - emu.rgb[ok]).max()
        assert e_emu <= 2e-3, e_emu
    e64 = np.abs(rgb[ok] - ref64.rgb[ok]).max()
    assert e64 <= (2e-3 if prec == "fp16" else 1e-2), e64
    empty = ref64.hits.n == 0
    assert np.array_equal(rgb[empty], np.broadcast_to(np.float32(bg), (empty.sum(), 3)))


def test_launch_shapes_do_not_change_results(tiny):
    """Every tuning candidate gives the same image as the defaults."""
    from paper_2205_07058_b300 import svlf
    from paper_2205_07058_b300.autotune import MLP_CANDIDATES, TRACE_CANDIDATES
    tree, f, p, r = gpu_inputs(tiny)
    net = net_for(tiny, svlf.BF16)
    svlf.svlf_set_tuning()
    ref, dref, _, _, _ = svlf.svlf_render_rays(tree, f, p, net, r, tiny.K)
    try:
        for cand in TRACE_CANDIDATES + MLP_CANDIDATES:
            svlf.svlf_set_tuning(**cand)
            rgb, depth, _, _, _ = svlf.svlf_render_rays(tree, f, p, net, r, tiny.K)
            torch.testing.assert_close(rgb, ref, rtol=0, atol=0)
            torch.testing.assert_close(depth, dref, rtol=0, atol=0)
    finally:
        svlf.svlf_set_tuning()


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_repeated_renders_are_bit_identical(prec):
    """Samples land in different tiles and rows from call to call (the
    traversal reserves them with atomics); every sample's value must not
    depend on where it lands, so repeated renders agree bit for bit."""
    import math
    from paper_2205_07058_b300 import svlf
    rng = np.random.default_rng(77)
    sc = I.make_scene(rng, 7, 24, 8)
    rays = np.concatenate([I.pinhole_rays(math.radians(a), math.radians(e), 384, 384)
                           for a, e in ((15, 10), (200, -20))])
    feats = I.make_features(rng, sc.n_leaves, 32)
    params = I.make_mlp(rng, I.MLPShape(32, 128, 3), bias_std=0.2)
    tree = svlf.Octree(torch.from_numpy(sc.leaf_ijk), sc.depth)
    f, p, r = (torch.from_numpy(x).cuda() for x in (feats, params, rays))
    net = svlf.Network(32, 128, 3, svlf.PRECISIONS[prec])
    ref = None
    for _ in range(6):
        rgb, depth, _, _, _ = svlf.svlf_render_rays(tree, f, p, net, r, 8)
        torch.cuda.synchronize()
        if ref is None:
            ref = (rgb.clone(), depth.clone())
        else:
            assert torch.equal(rgb, ref[0]) and torch.equal(depth, ref[1])
    assert svlf.svlf_get_device_status() == 0


def test_ffma_rate_kernel_is_plausible():
    """The FP32 roofline denominator: the FMA kernel's measured rate lies
    between a tenth of and the nominal 148 SMs x 128 lanes x 2 flop x clock."""
    from paper_2205_07058_b300 import svlf
    tf = svlf.svlf_measure_ffma_tflops(iters=4000, repeats=2)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = sms * 128 * 2 * 2.2e9 / 1e12  # generous clock bound
    assert nominal / 10 < tf < nominal
    assert svlf.svlf_get_device_status() == 0
