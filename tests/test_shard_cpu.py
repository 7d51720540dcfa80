"""Splitting one slot across GPUs by contiguous PRB ranges (Sec. 3.2: a
slot's subcarriers are spread over the GPUs, which never synchronise), on CPU:
the partition's arithmetic, and a two-rank gloo run in which each rank
detects its shard (the oracle stands in for the GPU) and rank 0 gathers the
shards and finds them equal, bit for bit, to the unsharded slot."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2510_01579_gb300 import shard

N_SYM = 2


@pytest.mark.parametrize("n_prb,world", [(273, 1), (273, 2), (273, 3), (273, 8), (5, 8), (0, 2), (24, 4)])
def test_prb_ranges_cover_contiguously_and_evenly(n_prb, world):
    r = shard.prb_ranges(n_prb, world)
    assert len(r) == world and r[0][0] == 0 and r[-1][1] == n_prb
    assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
    sizes = [b - a for a, b in r]
    assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)


@pytest.mark.parametrize("n_sub,world", [(3276, 2), (3276, 8), (30, 2), (30, 4), (7, 3), (100, 3)])
def test_shards_are_whole_prbs_and_cover_the_slot(n_sub, world):
    bounds = [shard.shard_problems(n_sub, 14, world, r) for r in range(world)]
    assert bounds[0][0] == 0 and bounds[-1][1] == n_sub * 14
    assert all(a[1] == b[0] for a, b in zip(bounds, bounds[1:]))
    for p0, p1 in bounds:  # every boundary is a PRB boundary or the slot's end (empty last shards)
        assert p0 % (12 * 14) == 0 or p0 == n_sub * 14
        assert p1 % (12 * 14) == 0 or p1 == n_sub * 14


def test_channels_rebase_and_straddle_check():
    ci = np.repeat(np.arange(30) // 12, N_SYM)  # PRB-held channels, ragged last PRB
    s = shard.shard_slot(ci, 30, N_SYM, 2, 1)
    assert (s["p0"], s["p1"], s["c0"], s["c1"]) == (48, 60, 2, 3)
    assert np.array_equal(s["chan_index"], np.zeros(12, np.int32))
    with pytest.raises(ValueError):  # a cut inside a PRB would share its channel
        shard.shard_channels(ci, 0, 10)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _detect_shard(w, sh, prm, seed):
    """Detect a shard as its own job (the GPU's role, played by the oracle):
    channels H[c0:c1] with the re-based index, problem p0 + k drawing the
    Philox stream of problem p0 + k."""
    import oracle
    mb, n_t = w["mod_bits"], w["n_t"]
    H = w["H"][sh["c0"]:sh["c1"]]
    out = []
    for k, p in enumerate(range(sh["p0"], sh["p1"])):
        b = oracle.build_detect32(H[sh["chan_index"][k]], w["y"][p], w["noise_var"][p], mb)
        r = oracle.cac_solve(b["Aq"], b["hq"], b["g"], (1 << (mb // 2)) - 1, prm, seed, p)
        out.append((oracle.decode_detect(n_t, mb, b["g"], r["d"]), r["E"], r["n_div"]))
    return out


def _worker(rank, world, port, hold, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        import synth
        w = synth.uplink(41, 4, 4, 4, n_sub=30, n_sym=N_SYM, snr_db=14.0, hold=hold)  # 2.5 PRBs: ragged
        prm = oracle.Params(steps=60)
        sh = shard.shard_slot(w["chan_index"], 30, N_SYM, world, rank)
        mine = _detect_shard(w, sh, prm, 9)
        parts = [None] * world
        dist.all_gather_object(parts, (rank, sh["p0"], sh["p1"], mine))
        ok = None
        if rank == 0:
            parts.sort()
            gathered = [x for _, _, _, rows in parts for x in rows]
            whole = oracle.detect_batch(w["H"], w["y"], w["noise_var"], 4, prm, 9, w["chan_index"])
            P = w["y"].shape[0]
            ok = (len(gathered) == P and [(a, b) for _, a, b, _ in parts] == [(0, 48), (48, 60)] and
                  all(np.array_equal(gathered[p][0], whole["sym"][p]) and gathered[p][1] == whole["E"][p] and
                      gathered[p][2] == whole["n_div"][p] for p in range(P)))
        q.put((rank, ok))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("hold", ["prb", "subcarrier"])
def test_two_ranks_shard_one_slot_equal_to_the_unsharded_slot(hold):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, hold, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] is True
