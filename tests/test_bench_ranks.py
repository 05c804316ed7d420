"""Multi-rank bookkeeping of bench.py on CPU (gloo, world size 2): the ranks
hold the two halves of the weak-scaled chain set (one pair of 2 x 65,536
chains, windows of global chain indices) and the step time is the maximum
over ranks."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank
    out = bench.max_over_ranks(ms, dist)
    from paper_1811_04156_gb300 import api, build
    build.build()
    args = bench.parse_args([])
    sc = bench.scene_for(args, world)
    q.put((rank, out, api.shard_range(sc.pairs, rank, world), sc.total_chains))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_time_reduction_and_seeds():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert [r[1] for r in res] == [150.0, 150.0]
    assert res[0][3] == res[1][3] == 2 * 65_536
    assert res[0][2] == (0, 65_536) and res[1][2] == (65_536, 131_072)


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, None) == 12.5
