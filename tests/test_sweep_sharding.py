"""Multi-rank RHS sharding, run as world-size-2 gloo ranks on CPU."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1202_3424_gb300.sweep import gather_results, shard_rhs, solve_sweep


def test_shards_cover_every_rhs_once():
    for R in (0, 1, 2, 7, 128, 129):
        for world in (1, 2, 3, 8):
            got = [i for rank in range(world) for i in shard_rhs(R, rank, world)]
            assert got == list(range(R))
            sizes = [len(shard_rhs(R, rk, world)) for rk in range(world)]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, R, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    khat = np.arange(3 * R, dtype=float).reshape(R, 3)
    ehat = -khat

    def fake_block(k, e):  # stands in for a GPU solve of this rank's RHS block
        return [{"rhs": int(row[0] // 3), "rank": rank, "q": float(row.sum() + e_.sum())} for row, e_ in zip(k, e)]

    res = solve_sweep(fake_block, khat, ehat, dist)
    # bench.py's max/sum over ranks use the same collectives on CPU tensors
    import bench
    tmax = bench.max_over_ranks(dist, float(rank + 1))
    tsum = bench.sum_over_ranks(dist, float(rank + 1))
    out[rank] = (res, tmax, tsum)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("R", [5, 128])
def test_two_rank_sweep_gathers_in_order(R):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, R, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for rank in range(2):
        res, tmax, tsum = out[rank]
        assert [r["rhs"] for r in res] == list(range(R))
        assert [r["rank"] for r in res] == [0] * len(shard_rhs(R, 0, 2)) + [1] * len(shard_rhs(R, 1, 2))
        assert tmax == 2.0 and tsum == 3.0
    assert gather_results([1, 2]) == [1, 2]
