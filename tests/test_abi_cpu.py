"""The C-ABI library loads and exports every symbol include/svlf.h declares;
host-side argument checks answer without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^(?:int|const char \*)\s*(svlf_\w+)\(", src, re.M))
    return names


@pytest.fixture(scope="module")
def L():
    from paper_2205_07058_b300 import build_lib
    build_lib.build()
    from paper_2205_07058_b300 import svlf
    return svlf.lib()


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert len(names) >= 11
    for n in names:
        assert hasattr(L, n), n


def test_binding_names_cover_the_abi():
    from paper_2205_07058_b300 import svlf
    assert _declared() <= set(svlf.EXPORTS)


def test_every_binding_declares_argument_types(L):
    """Without argtypes ctypes passes Python ints as 32-bit C ints, leaving the
    upper half of an int64_t / size_t argument undefined."""
    from paper_2205_07058_b300 import svlf
    for n in svlf.EXPORTS:
        assert getattr(L, n).argtypes is not None, n


def test_host_side_argument_errors(L):
    from paper_2205_07058_b300 import svlf
    assert svlf.status_string(0) == "ok"
    assert "argument" in svlf.status_string(svlf.SVLF_ERR_ARG)
    d = svlf.MlpDesc(32, 128, 3, 4, svlf.FP32, 0)
    b = ctypes.c_size_t()
    assert L.svlf_workspace_size(ctypes.byref(d), 1000, 8, ctypes.byref(b)) == 0
    assert b.value >= 1000 * 8 * 48
    assert L.svlf_workspace_size(ctypes.byref(d), 1000, 0, ctypes.byref(b)) == svlf.SVLF_ERR_ARG
    o = svlf.RenderOpts()
    o.K = 8
    # null tree -> argument error before any CUDA call
    rc = L.svlf_render_rays(None, None, None, ctypes.byref(d), None, 10, ctypes.byref(o), None, None,
                            None, None, None, 0, None)
    assert rc == svlf.SVLF_ERR_ARG
    assert L.svlf_free_octree(None) == svlf.SVLF_ERR_ARG
    assert L.svlf_adam_step(None, None, None, None, 10, 1e-3, 0.9, 0.999, 1e-8, 1, None, None) \
        == svlf.SVLF_ERR_ARG
    assert L.svlf_adam_step(None, None, None, None, 10, 1e-3, 0.9, 0.999, 1e-8, 0, None, None) \
        == svlf.SVLF_ERR_ARG
    assert L.svlf_get_device_status(None, None) == svlf.SVLF_ERR_ARG
    assert L.svlf_set_step_limit(-1) == svlf.SVLF_ERR_ARG
    assert L.svlf_set_step_limit(1 << 31) == svlf.SVLF_ERR_ARG
    assert L.svlf_set_step_limit(0) == svlf.SVLF_OK


def test_tuning_arguments_are_checked(L):
    from paper_2205_07058_b300 import svlf
    svlf.svlf_set_tuning(3, 2, 32, 128, 8)
    assert svlf.svlf_get_tuning() == {"mlp_warpgroups": 3, "mlp_epilogue_batch": 2, "trace_budget": 32,
                                      "trace_block": 128, "trace_refill": 8, "mlp_bwd_warpgroups": 0}
    with pytest.raises(svlf.SvlfError):
        svlf.svlf_set_tuning(mlp_warpgroups=9)
    with pytest.raises(svlf.SvlfError):
        svlf.svlf_set_tuning(trace_block=100)
    with pytest.raises(svlf.SvlfError):
        svlf.svlf_set_tuning(trace_refill=33)
    with pytest.raises(svlf.SvlfError):
        svlf.svlf_set_tuning(mlp_bwd_warpgroups=3)
    svlf.svlf_set_tuning()  # defaults
    assert svlf.svlf_get_tuning()["trace_budget"] == 64
    assert svlf.svlf_get_tuning()["trace_refill"] == 0
