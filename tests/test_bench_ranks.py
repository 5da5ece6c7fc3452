"""bench.py's multi-process path on CPU: two gloo ranks run the same
cross-rank reduction the GPU arm runs over NCCL (max of the times, sum of the
evaluation counts), and the per-rank workloads are independent replicas."""
import os
import socket
from types import SimpleNamespace

import numpy as np
import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _local(rank):
    # [time ms, evals, e2e ms, e2e evals, full evals] of one rank
    return [10.0 + 5.0 * rank, 100.0 + rank, 20.0 - rank, 50.0 + 2.0 * rank, 7.0 * (rank + 1)]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mx, sm = bench.reduce_over_ranks(_local(rank), world, device="cpu")
        q.put((rank, mx.tolist(), sm.tolist()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_max_times_and_summed_counts():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    a, b = np.array(_local(0)), np.array(_local(1))
    for rank, mx, sm in out:
        assert np.array_equal(mx, np.maximum(a, b))
        assert np.array_equal(sm, a + b)


def test_single_rank_reduction_is_a_copy():
    mx, sm = bench.reduce_over_ranks(_local(0), 1)
    assert np.array_equal(mx, _local(0)) and np.array_equal(sm, _local(0))


def test_ranks_are_independent_replicas():
    """Each rank runs its own posterior: campaign events and injections differ
    by rank (seed offsets), so the summed evaluations are distinct work."""
    ev0 = bench.campaign_workloads(0)
    ev1 = bench.campaign_workloads(1)
    assert [w.noise_seed for w in ev0] != [w.noise_seed for w in ev1]
    assert not np.array_equal(ev0[0].injection, ev1[0].injection)


def test_reference_arm_runs_on_rank_zero_only():
    args = SimpleNamespace(workload="cfg1", steps=1, warmup=0, cpu_seconds=1.0)
    assert bench.run_reference(args, 1, 2) is None
