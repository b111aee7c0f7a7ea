"""Host logic of the multi-GPU benchmark (replicas only), on CPU ranks.

The solver does not shard: under torchrun every rank advances its own copy
of the workload and the job's time is the maximum over ranks of the timed
region.  These tests run that reduction with the gloo backend at world
size 2 (no GPU), plus the throughput aggregation.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench as B

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r "measured" 10 + r ms for the kernel region and 3 - r s end to end
        vals = B.max_over_ranks([10.0 + rank, 3.0 - rank], dist, device="cpu")
        dist.barrier()
    finally:
        dist.destroy_process_group()
    with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as f:
        f.write(" ".join(repr(v) for v in vals))


def test_max_over_ranks_gloo_world_two(tmp_path):
    import torch.multiprocessing as mp

    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, str(tmp_path)))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    for p in procs:
        if p.is_alive():
            p.kill()
            p.join()
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    for r in range(world):
        vals = [float(v) for v in open(tmp_path / ("rank%d.txt" % r)).read().split()]
        # every rank sees the slowest rank's time for each entry
        assert vals == [10.0 + (world - 1), 3.0]


def test_max_over_ranks_single_process():
    assert bench.max_over_ranks([1.5, 2.5]) == [1.5, 2.5]


@pytest.mark.parametrize("world", [1, 2, 4, 8])
def test_replica_throughput_is_weak_scaling(world):
    K, steps, ms = 999698, 100, 171.5
    one = bench.replica_throughput(1, K, steps, ms)
    assert one == pytest.approx(K * 5 * steps / 0.1715)
    # per-GPU work fixed: the job's value grows with the number of replicas
    assert bench.replica_throughput(world, K, steps, ms) == pytest.approx(world * one)
