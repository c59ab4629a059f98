"""Multi-GPU host logic of bench.py on CPU: two gloo ranks run as independent replicas
(each its own frame, no data-path collective); timing is the maximum over ranks and the
whole-job rate sums the ranks' units."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [100.0 + 50.0 * rank, 10.0 * (world - rank)]        # rank 1 slower on the first value
    mx = bench.max_over_ranks(ms, world, "cpu")
    value = bench.replica_throughput(1920 * 4, mx[0], world)
    out.put((rank, mx, value, bench.rank_seed_index(7, rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_aggregate_like_bench():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    results = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, mx0, v0, s0), (r1, mx1, v1, s1) = results
    assert mx0 == mx1 == [150.0, 20.0]
    assert v0 == v1 == pytest.approx(2 * 1920 * 4 / 0.150)
    assert (s0, s1) == (7, 8)                                  # distinct frames per replica


def test_single_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([1.0, 2.0], 1, "cpu") == [1.0, 2.0]
    assert bench.replica_throughput(1920, 10.0, 1) == pytest.approx(192000.0)
