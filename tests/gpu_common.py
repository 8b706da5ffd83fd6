"""Shared helpers for the GPU parity tests (CUDA path vs the FP64 oracle)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O

requires_gpu = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")


def net_for(w, precision):
    from paper_2205_07058_b300 import svlf
    return svlf.Network(w.mlp.feat_dim, w.mlp.hidden, w.mlp.n_hidden, precision,
                        svlf.FEAT_BF16 if w.feat_bf16 else svlf.FEAT_F32)


def gpu_inputs(w, features=None, params=None, rays=None):
    from paper_2205_07058_b300 import svlf
    tree = svlf.Octree(torch.from_numpy(w.scene.leaf_ijk), w.scene.depth)
    f = torch.from_numpy(w.features if features is None else features).cuda()
    p = torch.from_numpy(w.params if params is None else params).cuda()
    r = torch.from_numpy(w.rays if rays is None else rays).cuda()
    return tree, f, p, r


def compare_hits(oracle_hits, gpu_hits, gpu_tio, atol_t=2e-6):
    """Hit lists bit-exact on rays the oracle does not flag as near-degenerate;
    returns (n_checked, n_degenerate, n_degenerate_mismatch)."""
    deg = oracle_hits.degenerate
    ok = ~deg
    g = gpu_hits
    assert np.array_equal(g[ok], oracle_hits.rank[ok]), \
        f"{(g[ok] != oracle_hits.rank[ok]).any(axis=1).sum()} non-degenerate rays differ"
    m = oracle_hits.rank[ok] >= 0
    tin = gpu_tio[ok][..., 0][m]
    tout = gpu_tio[ok][..., 1][m]
    np.testing.assert_allclose(tin, oracle_hits.t_in[ok][m], rtol=0, atol=atol_t)
    np.testing.assert_allclose(tout, oracle_hits.t_out[ok][m], rtol=0, atol=atol_t)
    mism = int((g[deg] != oracle_hits.rank[deg]).any(axis=1).sum()) if deg.any() else 0
    return int(ok.sum()), int(deg.sum()), mism


def random_rays(rng, n, inside_frac=0.2):
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = 0.5 + 2.5 * rng.standard_normal((n, 3)) / np.sqrt(3)
    m = rng.uniform(size=n) < inside_frac
    o[m] = rng.uniform(0.0, 1.0, size=(m.sum(), 3))
    # aim most outside rays at the cube
    aim = rng.uniform(0.2, 0.8, size=(n, 3))
    v = aim - o
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    use = (~m) & (rng.uniform(size=n) < 0.8)
    d[use] = v[use]
    return np.concatenate([o, d], axis=1).astype(np.float32)
