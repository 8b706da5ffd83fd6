"""The N > 1 path on CPU with gloo ranks (127.0.0.1): the bench's job time is
the slowest rank's and its value counts every rank's units, ranks render
different views of the same scene, the reference arm runs on rank 0 only;
and data-parallel training (paper_2205_07058_b300/dp.py): shard losses over
the batch's ray count plus one all-reduce of the contiguous gradient buffer
give every rank the oracle gradient of the union batch."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        local_ms = [10.0, 12.5][rank]
        t_max = bench.max_over_ranks(local_ms, dist, "cpu")
        value = bench.job_value(1000, world, 4, t_max)
        W = bench.make_workload(rank, 2, 16)
        dist.barrier()
        out.put((rank, t_max, value, W["scene"].leaf_ijk.shape[0], W["render_rays"][:, 3:].sum(axis=0).tolist()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replicas_and_max_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, v0, n0, d0), (r1, t1, v1, n1, d1) = res
    assert t0 == t1 == 12.5                       # the slowest rank's time on every rank
    assert v0 == v1 == pytest.approx(1000 * 2 * 4 / 12.5e-3)  # every rank's units / job time
    assert n0 == n1                               # the same scene
    assert not np.allclose(d0, d1)                # different views


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench

    class A:
        views, res, warmup, steps = 1, 8, 0, 1
    assert bench.run_reference(A(), rank=1, world=2) is None


def test_replica_views_differ_per_rank():
    sys.path.insert(0, ROOT)
    import bench
    a = bench.replica_views(1, 3)
    b = bench.replica_views(2, 3)
    assert not np.allclose(a[0], b[0])
    assert np.array_equal(bench.replica_views(1, 3)[0], a[0])  # seeded


# ----------------------------------------------------------------------------
# data-parallel training: shard gradients + one all-reduce == the union batch
# ----------------------------------------------------------------------------
def _dp_rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    from paper_2205_07058_b300 import dp
    from paper_2205_07058_b300 import inputs as I
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        w = I.tiny_workload()
        rng = np.random.default_rng(5)
        params = I.make_mlp(rng, w.mlp, bias_std=0.3)
        rays = w.rays
        N = rays.shape[0]
        rgb_t = rng.uniform(0, 1, size=(N, 3))
        depth_t, mask = I.analytic_depth(rays, w.scene)
        sl = dp.shard(N, rank, world)
        tree = O.build_octree(w.scene.leaf_ijk, w.scene.depth)
        dims = O.layer_dims(16, 64, 2)
        r = O.render(tree, w.features, params, dims, rays[sl], w.K)
        df, dpar, _, _ = O.backward(tree, r, params, dims, rgb_t[sl], depth_t[sl].astype(np.float64),
                                    mask[sl].astype(np.float64), (0, 0, 0), tree.n_leaves, 16, norm=N)
        # the oracle's float64 gradients in the product's buffer layout (float64 here)
        buf = dp.GradientBuffer([df.shape, dpar.shape], device="cpu", dtype=torch.float64)
        buf.views[0].copy_(torch.from_numpy(df))
        buf.views[1].copy_(torch.from_numpy(dpar))
        dp.allreduce_gradients(buf)
        out.put((rank, sl.start, sl.stop, buf.views[0].numpy().copy(), buf.views[1].numpy().copy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_data_parallel_gradients_equal_the_union_batch(world):
    """Each gloo rank takes the oracle's adjoint on its shard of the tiny
    view's rays, with the loss divided by the whole batch's ray count (the
    product's shard loss), and the product's exchange (one all-reduce over the
    contiguous gradient buffer) must give every rank the oracle gradient of
    the union batch. world = 3 makes the shards uneven."""
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    from paper_2205_07058_b300 import inputs as I
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dp_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = I.tiny_workload()
    rng = np.random.default_rng(5)
    params = I.make_mlp(rng, w.mlp, bias_std=0.3)
    N = w.rays.shape[0]
    rgb_t = rng.uniform(0, 1, size=(N, 3))
    depth_t, mask = I.analytic_depth(w.rays, w.scene)
    tree = O.build_octree(w.scene.leaf_ijk, w.scene.depth)
    dims = O.layer_dims(16, 64, 2)
    r = O.render(tree, w.features, params, dims, w.rays, w.K)
    df, dpar, _, _ = O.backward(tree, r, params, dims, rgb_t, depth_t.astype(np.float64),
                                mask.astype(np.float64), (0, 0, 0), tree.n_leaves, 16)
    # the shards tile the batch
    assert res[0][1] == 0 and res[-1][2] == N
    assert all(res[i][2] == res[i + 1][1] for i in range(world - 1))
    assert max(x[2] - x[1] for x in res) - min(x[2] - x[1] for x in res) <= 1
    for _, _, _, gf, gp in res:
        np.testing.assert_allclose(gf, df, rtol=0, atol=1e-12 * np.abs(df).max())
        np.testing.assert_allclose(gp, dpar, rtol=0, atol=1e-12 * np.abs(dpar).max())
    # and the shards' losses sum to the batch's mean loss
    parts = []
    for i in range(world):
        sl = slice(res[i][1], res[i][2])
        parts.append(O.loss(r.rgb[sl], r.depth[sl], rgb_t[sl], depth_t[sl], mask[sl], norm=N))
    assert abs(sum(parts) - O.loss(r.rgb, r.depth, rgb_t, depth_t, mask)) <= 1e-14


def test_gradient_buffer_views_are_contiguous_and_aligned():
    sys.path.insert(0, ROOT)
    from paper_2205_07058_b300 import dp
    buf = dp.GradientBuffer([(7, 3), (13,), (2, 2)])
    assert buf.flat.numel() == 24 + 16 + 4
    for v in buf.views:
        assert v.data_ptr() % 16 == 0 and v.is_contiguous()
    buf.views[1].fill_(1.0)
    assert buf.flat.sum().item() == 13.0
    assert [dp.shard(10, r, 3) for r in range(3)] == [slice(0, 4), slice(4, 7), slice(7, 10)]
