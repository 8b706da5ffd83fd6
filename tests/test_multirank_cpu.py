"""The N > 1 path of bench.py on CPU: two gloo ranks (127.0.0.1), one
independent replica each (no data-path collective): the job time is the
slowest rank's, the job value counts every rank's units, replicas render
different views of the same scene, and the reference arm runs on rank 0 only."""
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
