"""The N > 1 path on CPU: two gloo ranks, as bench.py and the field sweep use them.

bench.py runs one independent instance per rank (replicas, no data-path
collective); only the timing is reduced: the slowest rank's time, and the
whole-job rate = ranks x units / that time.  The field sweep gives rank r the
fields h[r::world]; the union over ranks is the sweep.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_1411_0391_gb300 import sweep
        # timing reduction: rank-dependent times, every rank must see the maximum
        mine = [1.0 + rank, 0.5 * (rank + 1)]
        slow = bench.max_over_ranks(mine, dist, torch.device("cpu"))
        # field slices: a stand-in for the GPU evolution returns the field it was given
        sweep.run_field = lambda h, *a, **k: {"h": h, "rank": rank}
        part = sweep.field_sweep([2.0, 2.5, 3.0, 3.5, 4.0], 2, 8, 0.01, 1, rank=rank, world=world)
        gathered = [None] * world
        dist.all_gather_object(gathered, part)
        out.put((rank, slow, bench.whole_job_rate(world, 3, slow[0]), gathered))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replica_logic():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slow, rate, gathered in res:
        assert slow == [2.0, 1.0]                       # max over ranks, element-wise
        assert rate == pytest.approx(2 * 3 / 2.0)       # all ranks' units / slowest time
        hs = sorted(r["h"] for part in gathered for r in part)
        assert hs == [2.0, 2.5, 3.0, 3.5, 4.0]
        assert [r["h"] for r in gathered[0]] == [2.0, 3.0, 4.0]
        assert all(r["rank"] == i for i, part in enumerate(gathered) for r in part)
