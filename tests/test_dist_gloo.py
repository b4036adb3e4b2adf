"""Replica (weak-scaling) host logic with world_size 2 over gloo on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2512_08887_gb300.dist import rank_blocks, whole_job_rate


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    from paper_2512_08887_gb300.dist import max_over_ranks, rank_blocks
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b, e = rank_blocks(64, rank, world)
    t = max_over_ranks(1.5 + rank)                  # rank 1 is the slow one
    dist.barrier()
    q.put((rank, b, e, t))
    dist.destroy_process_group()


def test_two_replicas_partition_blocks_and_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [(b, e) for _, b, e, _ in out] == [(0, 32), (32, 64)]
    assert all(t == 2.5 for *_, t in out)


def test_partition_covers_the_stream_exactly():
    for total in (0, 1, 7, 64, 1001):
        for world in (1, 2, 3, 8):
            spans = [rank_blocks(total, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == total
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
            assert max(e - b for b, e in spans) - min(e - b for b, e in spans) <= 1
    with pytest.raises(ValueError):
        rank_blocks(10, 2, 2)


def test_whole_job_rate_uses_all_ranks_units_over_the_slowest_time():
    assert whole_job_rate(100.0, 4, 2.0) == 200.0
