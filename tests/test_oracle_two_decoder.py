"""Pins of the two-decoder oracle (vertex features, trilinear psi, Eq. 1-2)
against closed forms, brute force and properties that fix them."""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from oracle import two_decoder as T2
from paper_2205_07058_b300 import inputs as I


def _tree(ijk, depth):
    return O.build_octree(np.asarray(ijk, dtype=np.int32).reshape(-1, 3), depth)


def test_vertex_table_small_closed_forms():
    # one leaf: its 8 corners, ids in Morton order = corner slot a + 2b + 4c
    vt = T2.vertex_table(_tree([[0, 0, 0]], 1))
    assert vt.n_vertices == 8
    assert np.array_equal(vt.leaf_vertices[0], np.arange(8))
    # two face neighbours share a face: 12 vertices
    assert T2.vertex_table(_tree([[0, 0, 0], [1, 0, 0]], 2)).n_vertices == 12
    # the full 2x2x2 block of depth 1: the 3^3 lattice
    full = list(itertools.product(range(2), repeat=3))
    assert T2.vertex_table(_tree(full, 1)).n_vertices == 27
    # a diagonal pair sharing one corner: 15
    assert T2.vertex_table(_tree([[0, 0, 0], [1, 1, 1]], 2)).n_vertices == 15


def test_vertex_table_against_brute_force():
    rng = np.random.default_rng(3)
    ijk = np.unique(rng.integers(0, 16, size=(300, 3)), axis=0)
    tree = _tree(ijk, 4)
    vt = T2.vertex_table(tree)
    leaves = tree.leaf_ijk()
    # every corner coordinate once, via a set
    seen = set()
    for l in range(tree.n_leaves):
        for a in (0, 1):
            for b in (0, 1):
                for c in (0, 1):
                    seen.add((leaves[l, 0] + a, leaves[l, 1] + b, leaves[l, 2] + c))
    assert vt.n_vertices == len(seen)
    # the table points every (leaf, slot) at the lattice point leaf + corner(slot)
    for l in range(tree.n_leaves):
        for a in (0, 1):
            for b in (0, 1):
                for c in (0, 1):
                    v = vt.leaf_vertices[l, a + 2 * b + 4 * c]
                    assert tuple(vt.vertex_ijk[v]) == (leaves[l, 0] + a, leaves[l, 1] + b, leaves[l, 2] + c)
    # ids follow Morton order of the lattice points: strictly increasing codes
    bits = 5
    codes = [sum(((int(x) >> i) & 1) << (3 * i + ax) for i in range(bits) for ax, x in enumerate(p))
             for p in vt.vertex_ijk]
    assert all(a < b for a, b in zip(codes, codes[1:]))


def _affine_features(vt, depth, rng, F):
    A = rng.standard_normal((F, 3))
    b = rng.standard_normal(F)
    pos = vt.vertex_ijk.astype(np.float64) * 2.0 ** -depth
    return pos @ A.T + b, A, b


def test_psi_reproduces_affine_fields_and_corners():
    """Trilinear interpolation is exact on affine functions of position and
    returns the corner value at a corner."""
    rng = np.random.default_rng(4)
    depth = 5
    ijk = np.unique(rng.integers(0, 32, size=(200, 3)), axis=0)
    tree = _tree(ijk, depth)
    vt = T2.vertex_table(tree)
    Z, A, b = _affine_features(vt, depth, rng, 6)
    rank = rng.integers(0, tree.n_leaves, size=500)
    p = (tree.leaf_ijk()[rank] + rng.uniform(0, 1, size=(500, 3))) * 2.0 ** -depth
    np.testing.assert_allclose(T2.psi(p, rank, tree, vt, Z), p @ A.T + b, rtol=0, atol=1e-12)
    # corners
    Zr = rng.standard_normal((vt.n_vertices, 4))
    for s, corner in enumerate(T2.CORNERS):
        pc = (tree.leaf_ijk()[rank] + corner) * 2.0 ** -depth
        np.testing.assert_allclose(T2.psi(pc, rank, tree, vt, Zr), Zr[vt.leaf_vertices[rank, s]], atol=1e-15)
    # centre: the mean of the eight corners
    pm = (tree.leaf_ijk()[rank] + 0.5) * 2.0 ** -depth
    np.testing.assert_allclose(T2.psi(pm, rank, tree, vt, Zr), Zr[vt.leaf_vertices[rank]].mean(axis=1), atol=1e-15)


def test_psi_is_continuous_across_shared_faces():
    rng = np.random.default_rng(5)
    tree = _tree([[2, 3, 4], [3, 3, 4]], 3)  # x-neighbours sharing the face x = 3
    vt = T2.vertex_table(tree)
    Z = rng.standard_normal((vt.n_vertices, 5))
    yz = rng.uniform(0, 1, size=(50, 2))
    p = np.column_stack([np.full(50, 3.0), 3.0 + yz[:, 0], 4.0 + yz[:, 1]]) / 8.0
    ranks = {tuple(r): i for i, r in enumerate(tree.leaf_ijk())}
    a = T2.psi(p, np.full(50, ranks[(2, 3, 4)]), tree, vt, Z)
    b = T2.psi(p, np.full(50, ranks[(3, 3, 4)]), tree, vt, Z)
    np.testing.assert_allclose(a, b, atol=1e-14)


@pytest.fixture(scope="module")
def small():
    rng = np.random.default_rng(1006)
    sc = I.make_scene(rng, 6, 8, 2)
    tree = O.build_octree(sc.leaf_ijk, 6)
    vt = T2.vertex_table(tree)
    rays = I.pinhole_rays(np.radians(40.0), np.radians(25.0), 48, 48)
    return sc, tree, vt, rays


def _zero_net(dims, out_bias):
    p = []
    for li, (o, i) in enumerate(dims):
        p.append(np.zeros(o * i))
        p.append(np.asarray(out_bias, dtype=np.float64) if li + 1 == len(dims) else np.zeros(o))
    return np.concatenate(p)


@pytest.mark.parametrize("b_tau,b_eta,b_c", [(0.7, 0.3, -0.4), (-1.0, 2.0, 1.0), (2.5, 40.0, 0.2), (0.4, -40.0, 0.0)])
def test_constant_networks_closed_form(small, b_tau, b_eta, b_c):
    """All weights zero: tau = relu(b_tau), eta = sigmoid(b_eta) and c =
    sigmoid(b_c) on every hit, so with n hits (brute-force hit lists)
    C = c (1 - e^{-n tau}) + e^{-n tau} bg and D = sum_i T_i alpha (eta t_in,i +
    (1 - eta) t_out,i)."""
    sc, tree, vt, rays = small
    K = 5
    dt, dc = T2.dims_t(16, 32, 1), T2.dims_c(8, 32, 2)
    pt = _zero_net(dt, [b_tau, b_eta])
    pc = _zero_net(dc, [b_c] * 3)
    rng = np.random.default_rng(0)
    zt = rng.standard_normal((vt.n_vertices, 16))
    zc = rng.standard_normal((vt.n_vertices, 8))
    bg = (0.2, 0.5, 0.9)
    r = T2.render2(tree, vt, zt, zc, pt, pc, dt, dc, rays, K, bg=bg)
    brute = O.trace(tree, rays, K, mode="brute")
    n = brute.n.astype(np.float64)
    tau = max(b_tau, 0.0)
    eta = 1.0 / (1.0 + np.exp(-b_eta))
    c = 1.0 / (1.0 + np.exp(-b_c))
    exp_rgb = c * (1.0 - np.exp(-n * tau))[:, None] + np.exp(-n * tau)[:, None] * np.asarray(bg)[None, :]
    np.testing.assert_allclose(r.rgb, exp_rgb, rtol=0, atol=1e-12)
    alpha = 1.0 - np.exp(-tau)
    Ti = np.exp(-tau * np.arange(K))[None, :]
    valid = brute.rank >= 0
    ts = eta * brute.t_in + (1.0 - eta) * brute.t_out
    exp_d = np.sum(np.where(valid, Ti * alpha * ts, 0.0), axis=1)
    np.testing.assert_allclose(r.depth, exp_d, rtol=0, atol=1e-12)
    assert (n > 0).sum() > 200


def test_surface_point_on_segment_inside_voxel(small):
    sc, tree, vt, rays = small
    rng = np.random.default_rng(1)
    dt, dc = T2.dims_t(16, 32, 1), T2.dims_c(8, 32, 2)

    # He-style random networks with non-zero biases
    def rand_net(dims):
        out = []
        for o, i in dims:
            out.append(rng.standard_normal(o * i) * np.sqrt(2.0 / i))
            out.append(rng.standard_normal(o) * 0.3)
        return np.concatenate(out)
    pt, pc = rand_net(dt), rand_net(dc)
    zt = rng.standard_normal((vt.n_vertices, 16)) * 0.1
    zc = rng.standard_normal((vt.n_vertices, 8)) * 0.1
    r = T2.render2(tree, vt, zt, zc, pt, pc, dt, dc, rays, 6)
    assert np.all((r.eta > 0) & (r.eta < 1))
    # x_s on the segment [x1, x2] at parameter t_s, and inside the hit voxel
    o = rays[r.ray_of, :3].astype(np.float64)
    d = rays[r.ray_of, 3:].astype(np.float64)
    np.testing.assert_allclose(r.x_s, o + r.t_s[:, None] * d, atol=1e-12)
    rank = r.hits.rank[r.ray_of, r.slot]
    lo = tree.leaf_ijk()[rank] * 2.0 ** -tree.depth
    assert np.all(r.x_s >= lo - 1e-12) and np.all(r.x_s <= lo + 2.0 ** -tree.depth + 1e-12)
    tin = r.hits.t_in[r.ray_of, r.slot]
    tout = r.hits.t_out[r.ray_of, r.slot]
    assert np.all((r.t_s >= tin - 1e-15) & (r.t_s <= tout + 1e-15))


def test_network_inputs_order_by_selection(small):
    """A network that routes one input coordinate to eta's pre-activation
    (through a ReLU unit, with an offset keeping it positive) recovers, for
    affine vertex features, the value of the affine field at x2 computed from
    the brute-force exit parameter: pins the input order [psi(x1) | psi(x2) |
    r] and the exit point."""
    sc, tree, vt, rays = small
    rng = np.random.default_rng(7)
    F = 8
    Z, A, b = _affine_features(vt, tree.depth, rng, F)
    dt, dc = T2.dims_t(F, 32, 1), T2.dims_c(4, 32, 1)
    f_sel = 5
    col = F + f_sel  # psi(x2)[f_sel]
    W0 = np.zeros((32, 6 + 2 * F))
    W0[0, col] = 1.0
    b0 = np.zeros(32)
    b0[0] = 50.0  # keep the unit in the ReLU's linear part
    W1 = np.zeros((2, 32))
    W1[1, 0] = 1.0
    b1 = np.array([0.0, -50.0])
    pt = np.concatenate([W0.ravel(), b0, W1.ravel(), b1])
    pc = _zero_net(dc, [0.0, 0.0, 0.0])
    zc = np.zeros((vt.n_vertices, 4))
    r = T2.render2(tree, vt, Z, zc, pt, pc, dt, dc, rays, 4)
    brute = O.trace(tree, rays, 4, mode="brute")
    o = rays[r.ray_of, :3].astype(np.float64)
    d = rays[r.ray_of, 3:].astype(np.float64)
    x2 = o + brute.t_out[r.ray_of, r.slot][:, None] * d
    expect = x2 @ A[f_sel] + b[f_sel]
    pre_eta = np.log(r.eta / (1.0 - r.eta))
    np.testing.assert_allclose(pre_eta, expect, rtol=0, atol=1e-9)


def test_two_decoder_adjoint_matches_central_differences(small):
    """The hand-derived adjoint (through Eq. 3, both networks, the trilinear
    scatter and the surface point x_s = o + t_s d) against central
    differences in float64, h = 1e-3, on 64 parameters: Z^T and Z^C entries
    of hit voxels' corners, weights of both networks, and always eta's output
    bias and weights (the path through x_s). Perturbations that flip a ReLU,
    the tau ReLU or the sign of D - D* are resampled."""
    sc, tree, vt, rays = small
    K = 4
    ft, fc = 8, 8
    dt, dc = T2.dims_t(ft, 32, 1), T2.dims_c(fc, 32, 2)
    rng = np.random.default_rng(21)

    def rand_net(dims):
        out = []
        for o, i in dims:
            out.append(rng.standard_normal(o * i) * np.sqrt(2.0 / i))
            out.append(rng.standard_normal(o) * 0.3)
        return np.concatenate(out)
    pt, pc = rand_net(dt), rand_net(dc)
    zt = rng.standard_normal((vt.n_vertices, ft)) * 0.5
    zc = rng.standard_normal((vt.n_vertices, fc)) * 0.5
    rgb_t = rng.uniform(0, 1, size=(rays.shape[0], 3))
    depth_t, mask = I.analytic_depth(rays, sc)
    depth_t, mask = depth_t.astype(np.float64), mask.astype(np.float64)
    bg = np.array([0.3, 0.2, 0.1])
    hits = O.trace(tree, rays, K)

    def run(zt_, zc_, pt_, pc_):
        r = T2.render2(tree, vt, zt_, zc_, pt_, pc_, dt, dc, rays, K, bg=bg, hits=hits)
        return O.loss(r.rgb, r.depth, rgb_t, depth_t, mask), r

    L0, r0 = run(zt, zc, pt, pc)
    dzt, dzc, dpt, dpc, _, _ = T2.backward2(tree, vt, r0, zc, pt, pc, dt, dc, rgb_t, depth_t, mask, bg, ft, fc)
    pat0 = T2.kink_pattern2(r0, depth_t, mask)
    hit_vertices = np.unique(vt.leaf_vertices[r0.rank])
    # eta's output row of F^T: the last layer is (2 x 32) then its bias (2)
    n_t = pt.size
    eta_idx = [n_t - 1] + [n_t - 2 - 32 + j for j in range(0, 32, 7)]
    h = 1e-3
    fd, ad, flips, k = [], [], 0, 0
    while len(fd) < 64:
        kind = ["zt", "zc", "pt", "pc"][k % 4]
        if k < len(eta_idx):
            kind, idx = "pt", eta_idx[k]
        elif kind in ("zt", "zc"):
            idx = (rng.choice(hit_vertices), rng.integers(ft if kind == "zt" else fc))
        else:
            idx = rng.integers((pt if kind == "pt" else pc).size)
        k += 1
        vals, ok = [], True
        for sgn in (+1, -1):
            a = {"zt": zt.copy(), "zc": zc.copy(), "pt": pt.copy(), "pc": pc.copy()}
            a[kind][idx] += sgn * h
            Ls, rs = run(a["zt"], a["zc"], a["pt"], a["pc"])
            ok &= O.same_pattern(T2.kink_pattern2(rs, depth_t, mask), pat0)
            vals.append(Ls)
        if not ok:
            flips += 1
            continue
        fd.append((vals[0] - vals[1]) / (2 * h))
        ad.append({"zt": dzt, "zc": dzc, "pt": dpt, "pc": dpc}[kind][idx])
    fd, ad = np.array(fd), np.array(ad)
    scale = np.maximum(np.abs(fd), 1e-3 * np.abs(fd).max())
    rel = np.abs(ad - fd) / scale
    assert rel.max() <= 1e-4, (rel.max(), flips)
    assert np.linalg.norm(ad - fd) / np.linalg.norm(fd) <= 1e-5
    # eta carries gradient: its output bias derivative is not negligible
    assert abs(dpt[n_t - 1]) > 1e-3 * np.abs(dpt).max()


# ---------------------------------------------------------------- staged training (Sec. 4.4, Eq. 4)
def test_surface_voxel_is_a_hit_of_the_ray(small):
    """The stage-1 voxel (the leaf containing o + D* d) is one of the ray's
    hits in the brute-force list, with the same segment; eta* is 1 at the
    entry and 0 at the exit."""
    sc, tree, vt, rays = small
    depth_t, mask = I.analytic_depth(rays, sc)
    ss = T2.surface_samples(tree, rays, depth_t, mask)
    assert ss.ray.size > 0.9 * (mask > 0).sum()
    brute = O.trace(tree, rays[ss.ray], 64, mode="brute")
    for i in range(ss.ray.size):
        j = np.nonzero(brute.rank[i] == ss.rank[i])[0]
        assert j.size == 1
        assert abs(brute.t_in[i, j[0]] - ss.t_in[i]) < 1e-12 and abs(brute.t_out[i, j[0]] - ss.t_out[i]) < 1e-12
    assert np.all((ss.eta_gt >= 0) & (ss.eta_gt <= 1))
    np.testing.assert_allclose(T2.eta_target(ss.t_in, ss.t_out, ss.t_in), 1.0)
    np.testing.assert_allclose(T2.eta_target(ss.t_in, ss.t_out, ss.t_out), 0.0, atol=1e-15)


def test_surface_loss_constant_networks_closed_form(small):
    sc, tree, vt, rays = small
    depth_t, mask = I.analytic_depth(rays, sc)
    rng = np.random.default_rng(31)
    rgb_t = rng.uniform(0, 1, size=(rays.shape[0], 3))
    dt, dc = T2.dims_t(8, 32, 1), T2.dims_c(8, 32, 2)
    b_tau, b_eta, b_c = 0.6, -0.3, np.array([0.2, -0.5, 1.1])
    pt = _zero_net(dt, [b_tau, b_eta])
    pc = _zero_net(dc, b_c)
    zt = rng.standard_normal((vt.n_vertices, 8))
    zc = rng.standard_normal((vt.n_vertices, 8))
    lam_eta, lam_tau = 0.7, 0.3
    L, ss, _, _ = T2.surface_loss(tree, vt, zt, zc, pt, pc, dt, dc, rays, rgb_t, depth_t, mask, lam_eta, lam_tau,
                                  8, 8, with_grad=False)
    c = 1.0 / (1.0 + np.exp(-b_c))
    eta = 1.0 / (1.0 + np.exp(-b_eta))
    brute = O.trace(tree, rays[ss.ray], 64, mode="brute")
    t_in = np.array([brute.t_in[i, np.nonzero(brute.rank[i] == ss.rank[i])[0][0]] for i in range(ss.ray.size)])
    t_out = np.array([brute.t_out[i, np.nonzero(brute.rank[i] == ss.rank[i])[0][0]] for i in range(ss.ray.size)])
    eg = np.clip((t_out - depth_t[ss.ray]) / (t_out - t_in), 0, 1)
    expect = (np.sum((c[None, :] - rgb_t[ss.ray]) ** 2) + lam_eta * np.sum((eta - eg) ** 2)
              + lam_tau * ss.ray.size * np.exp(-2.0 * b_tau)) / rays.shape[0]
    assert abs(L - expect) <= 1e-12 * max(1.0, abs(expect))


def _fd_check(loss_fn, grads, params, rng, kinds, n=48, h=1e-3):
    fd, ad, flips = [], [], 0
    L0, pat0 = loss_fn(params)
    k = 0
    while len(fd) < n:
        kind = kinds[k % len(kinds)]
        k += 1
        a = params[kind]
        idx = tuple(rng.integers(s) for s in a.shape)
        vals, ok = [], True
        for sgn in (+1, -1):
            p2 = {kk: v.copy() for kk, v in params.items()}
            p2[kind][idx] += sgn * h
            Ls, pat = loss_fn(p2)
            ok &= O.same_pattern(pat, pat0)
            vals.append(Ls)
        if not ok:
            flips += 1
            continue
        fd.append((vals[0] - vals[1]) / (2 * h))
        ad.append(grads[kind][idx])
    fd, ad = np.array(fd), np.array(ad)
    scale = np.maximum(np.abs(fd), 1e-3 * np.abs(fd).max())
    return np.abs(ad - fd) / scale, fd, ad


def test_surface_loss_adjoint_matches_central_differences(small):
    """Eq. 4's adjoint (colour, tau and eta terms; eta also through x_s)."""
    sc, tree, vt, rays = small
    depth_t, mask = I.analytic_depth(rays, sc)
    rng = np.random.default_rng(41)
    rgb_t = rng.uniform(0, 1, size=(rays.shape[0], 3))
    ft, fc = 8, 8
    dt, dc = T2.dims_t(ft, 32, 1), T2.dims_c(fc, 32, 2)

    def rand_net(dims):
        return np.concatenate([np.concatenate([rng.standard_normal(o * i) * np.sqrt(2.0 / i),
                                               rng.standard_normal(o) * 0.3]) for o, i in dims])
    P = {"zt": rng.standard_normal((vt.n_vertices, ft)) * 0.5, "zc": rng.standard_normal((vt.n_vertices, fc)) * 0.5,
         "pt": rand_net(dt), "pc": rand_net(dc)}
    lam = (0.8, 0.5)

    def loss_fn(p):
        L, ss, e, _ = T2.surface_loss(tree, vt, p["zt"], p["zc"], p["pt"], p["pc"], dt, dc, rays, rgb_t, depth_t,
                                      mask, lam[0], lam[1], ft, fc, with_grad=False)
        return L, [(x > 0) for x in e.pres_t[:-1]] + [(x > 0) for x in e.pres_c[:-1]] + [e.pres_t[-1][:, 0] > 0]
    L, ss, e, (gzt, gzc, gpt, gpc) = T2.surface_loss(tree, vt, P["zt"], P["zc"], P["pt"], P["pc"], dt, dc, rays,
                                                     rgb_t, depth_t, mask, lam[0], lam[1], ft, fc)
    G = {"zt": gzt, "zc": gzc, "pt": gpt, "pc": gpc}
    # perturb only vertices of surface voxels (others have zero gradient and zero FD)
    verts = np.unique(vt.leaf_vertices[ss.rank])
    sub = {"zt": P["zt"], "zc": P["zc"], "pt": P["pt"], "pc": P["pc"]}
    rel, fd, ad = _fd_check(loss_fn, G, sub, np.random.default_rng(5), ["pt", "pc", "pt", "pc"])
    assert rel.max() <= 1e-4, rel.max()
    # vertex features of surface voxels
    fd2, ad2 = [], []
    for i in range(24):
        kind = "zt" if i % 2 == 0 else "zc"
        v = verts[(i * 7919) % verts.size]
        f = i % (ft if kind == "zt" else fc)
        vals = []
        for sgn in (+1, -1):
            p2 = {kk: vv.copy() for kk, vv in P.items()}
            p2[kind][v, f] += sgn * 1e-3
            vals.append(loss_fn(p2)[0])
        fd2.append((vals[0] - vals[1]) / 2e-3)
        ad2.append(G[kind][v, f])
    fd2, ad2 = np.array(fd2), np.array(ad2)
    assert np.abs(ad2 - fd2).max() <= 1e-4 * max(np.abs(fd2).max(), 1e-12) + 1e-9


def test_volume_stage_eta_term_adjoint(small):
    """Stages 2-3: the composited loss plus lam_eta (eta_v - eta*)^2 on each
    ray's surface voxel among its hits; the eta term's direct gradient flows
    through the same adjoint."""
    sc, tree, vt, rays = small
    depth_t, mask = I.analytic_depth(rays, sc)
    depth_t, mask = depth_t.astype(np.float64), mask.astype(np.float64)
    rng = np.random.default_rng(51)
    rgb_t = rng.uniform(0, 1, size=(rays.shape[0], 3))
    ft, fc = 8, 8
    dt, dc = T2.dims_t(ft, 32, 1), T2.dims_c(fc, 32, 2)

    def rand_net(dims):
        return np.concatenate([np.concatenate([rng.standard_normal(o * i) * np.sqrt(2.0 / i),
                                               rng.standard_normal(o) * 0.3]) for o, i in dims])
    P = {"zt": rng.standard_normal((vt.n_vertices, ft)) * 0.5, "zc": rng.standard_normal((vt.n_vertices, fc)) * 0.5,
         "pt": rand_net(dt), "pc": rand_net(dc)}
    K = 4
    hits = O.trace(tree, rays, K)
    lam_eta = 0.9

    def loss_fn(p):
        r = T2.render2(tree, vt, p["zt"], p["zc"], p["pt"], p["pc"], dt, dc, rays, K, hits=hits)
        Le, _ = T2.eta_term(r, depth_t, mask, lam_eta)
        return O.loss(r.rgb, r.depth, rgb_t, depth_t, mask) + Le, T2.kink_pattern2(r, depth_t, mask)
    r = T2.render2(tree, vt, P["zt"], P["zc"], P["pt"], P["pc"], dt, dc, rays, K, hits=hits)
    Le, deta = T2.eta_term(r, depth_t, mask, lam_eta)
    assert np.count_nonzero(deta) > 100
    gzt, gzc, gpt, gpc, _, _ = T2.backward2(tree, vt, r, P["zc"], P["pt"], P["pc"], dt, dc, rgb_t, depth_t, mask,
                                            (0, 0, 0), ft, fc, deta_direct=deta)
    G = {"zt": gzt, "zc": gzc, "pt": gpt, "pc": gpc}
    rel, fd, ad = _fd_check(loss_fn, G, P, np.random.default_rng(6), ["pt", "pc"])
    assert rel.max() <= 1e-4, rel.max()
    # eta's output bias carries the eta term's gradient
    n_t = P["pt"].size
    r0 = T2.render2(tree, vt, P["zt"], P["zc"], P["pt"], P["pc"], dt, dc, rays, K, hits=hits)
    g_no = T2.backward2(tree, vt, r0, P["zc"], P["pt"], P["pc"], dt, dc, rgb_t, depth_t, mask, (0, 0, 0), ft, fc)[2]
    assert abs(gpt[n_t - 1] - g_no[n_t - 1]) > 1e-6
