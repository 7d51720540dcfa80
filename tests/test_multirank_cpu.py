"""The benchmark's multi-rank path on CPU with gloo (world size 2): each rank
detects its own slot (weak scaling, no collective on the data path), the step
time is the slowest rank's, and the --split slot gather puts the ranks' PRB
shards back in problem order."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2510_01579_gb300 import shard
    local = 10.0 + 5.0 * rank  # ms: rank 1 is the slow one
    m = bench.max_over_ranks(local)
    w = bench.make_workload("ul16x16_16qam_slot", bench.rank_seed(rank), n_sub=4)
    # the --split slot gather: each rank contributes the result rows of its PRB range; every rank
    # gets them all back, ordered by first problem
    sh = shard.shard_slot(np.repeat(np.arange(30), 2), 30, 2, world, rank)
    rows = np.arange(sh["p0"], sh["p1"]) * 10
    g = bench.gather_shards(sh["p0"], rows)
    q.put((rank, m, float(np.abs(w["y"]).sum()), g.tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_step_and_own_slots():
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
    assert [r[1] for r in res] == [15.0, 15.0]
    assert res[0][2] != res[1][2]  # different slots per rank
    assert res[0][3] == res[1][3] == list(range(0, 600, 10))  # shards gathered in problem order


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
