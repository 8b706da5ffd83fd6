"""The binding's argument checks (host only): the C ABI takes raw device
pointers, so a feature table or parameter array of the wrong dtype or size must
be refused in Python before any launch could read past it."""
from types import SimpleNamespace

import pytest
import torch

from paper_2205_07058_b300 import svlf


def _single(n_leaves=10, F=32, H=64, nh=2, fdt=svlf.FEAT_F32):
    tree = SimpleNamespace(n_leaves=n_leaves)
    net = svlf.Network(F, H, nh, svlf.BF16, fdt)
    n_par = (F + 9) * H + H + (nh - 1) * (H * H + H) + 4 * H + 4
    return tree, net, n_par


def test_param_count_matches_layout():
    tree, net, n_par = _single()
    assert svlf._param_count(svlf._net_dims(net)) == n_par
    td = svlf.TwoDecoder(64, 32, 128, 1, 128, 3)
    dt, dc = svlf._td_dims(td)
    assert svlf._param_count(dt) == (134 * 128 + 128) + (2 * 128 + 2)
    assert svlf._param_count(dc) == (38 * 128 + 128) + 2 * (128 * 128 + 128) + (3 * 128 + 3)


def test_single_accepts_matching_arguments():
    tree, net, n_par = _single()
    svlf._check_single(tree, torch.zeros(10, 32), torch.zeros(n_par), net, torch.zeros(5, 6),
                       torch.zeros(10, 32), torch.zeros(n_par))
    tree, net, n_par = _single(fdt=svlf.FEAT_BF16)
    svlf._check_single(tree, torch.zeros(10, 32, dtype=torch.bfloat16), torch.zeros(n_par), net, torch.zeros(5, 6),
                       torch.zeros(10, 32))  # the gradient stays float32


@pytest.mark.parametrize("case", ["bf16_table_f32_desc", "f32_table_bf16_desc", "few_rows", "wrong_F",
                                  "short_params", "f64_params", "flat_rays", "short_grad"])
def test_single_refuses_mismatches(case):
    tree, net, n_par = _single(fdt=svlf.FEAT_BF16 if case == "f32_table_bf16_desc" else svlf.FEAT_F32)
    feats = torch.zeros(10, 32)
    params = torch.zeros(n_par)
    rays = torch.zeros(5, 6)
    grad = None
    if case == "bf16_table_f32_desc":
        feats = feats.bfloat16()
    elif case == "few_rows":
        feats = torch.zeros(9, 32)
    elif case == "wrong_F":
        feats = torch.zeros(10, 16)
    elif case == "short_params":
        params = torch.zeros(n_par - 1)
    elif case == "f64_params":
        params = torch.zeros(n_par, dtype=torch.float64)
    elif case == "flat_rays":
        rays = torch.zeros(30)
    elif case == "short_grad":
        grad = torch.zeros(9, 32)
    with pytest.raises(ValueError):
        svlf._check_single(tree, feats, params, net, rays, grad)


def test_two_decoder_checks():
    td = svlf.TwoDecoder(64, 32, 128, 1, 128, 3, svlf.BF16, svlf.FEAT_BF16)
    dt, dc = svlf._td_dims(td)
    tree = SimpleNamespace(n_leaves=4, n_vertices=20)
    zt = torch.zeros(20, 64, dtype=torch.bfloat16)
    zc = torch.zeros(20, 32, dtype=torch.bfloat16)
    pt, pc = torch.zeros(svlf._param_count(dt)), torch.zeros(svlf._param_count(dc))
    rays = torch.zeros(3, 6)
    svlf._check_two_decoder(tree, zt, zc, pt, pc, td, rays, torch.zeros(20, 64), torch.zeros(20, 32), pt, pc)
    with pytest.raises(ValueError):  # float32 tables under a bf16 descriptor
        svlf._check_two_decoder(tree, zt.float(), zc.float(), pt, pc, td, rays)
    with pytest.raises(ValueError):  # fewer rows than vertices
        svlf._check_two_decoder(tree, zt[:19], zc, pt, pc, td, rays)
    with pytest.raises(ValueError):  # F^C parameters too short
        svlf._check_two_decoder(tree, zt, zc, pt, pc[:-1], td, rays)
    with pytest.raises(ValueError):  # bf16 gradient table
        svlf._check_two_decoder(tree, zt, zc, pt, pc, td, rays, zt)
