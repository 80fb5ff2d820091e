"""The N > 1 host path of the benchmark on CPU: two gloo ranks, each with its
own (fake) timing, must agree on the max over ranks and on the whole-job
weak-scaling throughput; replica seeds differ per rank."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    from paper_2503_14688_b300 import replicas

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = [100.0 + 50.0 * rank, 2.0 + rank]  # rank 1 is slower
        dist.barrier()
        ms, e2e = replicas.max_over_ranks(mine)
        value = replicas.weak_scaling_value(world, 1024.0 * 1024.0, 10, ms)
        out.put((rank, ms, e2e, value, replicas.replica_seed(7, rank)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_and_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ms0, e0, v0, s0), (r1, ms1, e1, v1, s1) = res
    assert ms0 == ms1 == 150.0 and e0 == e1 == 3.0
    assert v0 == v1 == pytest.approx(2 * 1024 * 1024 * 10 / (150.0 * 1e6))
    assert s0 != s1


def test_without_process_group_values_pass_through():
    from paper_2503_14688_b300 import replicas

    assert replicas.max_over_ranks([1.5, 2.5]) == (1.5, 2.5)
    assert replicas.weak_scaling_value(1, 4.0, 2, 1.0) == 8e-6
