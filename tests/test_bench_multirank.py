"""Host-side logic of the multi-rank benchmark, on 2 CPU ranks (gloo):
ranks get distinct seeds (independent frames, no data exchange) and the step
time is the maximum over ranks."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    times = [10.0 + rank, 3.0 * (world - rank)]
    got = bench.max_over_ranks(times, dist, "cpu")
    q.put((rank, bench.rank_seed(rank), got))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_max_and_seeds():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    os.environ["PYTHONPATH"] = root + os.pathsep + os.environ.get("PYTHONPATH", "")
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, g0), (r1, s1, g1) = res
    assert s0 != s1
    assert g0 == g1 == [11.0, 6.0]


def test_single_rank_passthrough():
    import bench

    assert bench.max_over_ranks([1.5, 2.5], None, "cpu") == [1.5, 2.5]
