"""One slot split into PRB-range shards (Sec. 3.2: subcarriers spread over
GPUs with no synchronisation), each shard run as its own job with its
problem_offset: the concatenated shard outputs equal the whole slot's bit for
bit, through mmgap_detect and through the batched launch.  (All shards run on
one GPU here; on several GPUs each rank runs its own shard the same way.)"""
import numpy as np
import pytest
import torch

import synth
from paper_2510_01579_gb300 import shard

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _outs(P, n_t):
    return {"sym": torch.full((P, n_t), 255, dtype=torch.uint8, device=DEV),
            "energy": torch.full((P,), 9, dtype=torch.int32, device=DEV),
            "ndiv": torch.full((P,), -1, dtype=torch.int32, device=DEV)}


@pytest.mark.parametrize("n_t,n_sub,hold,world", [(8, 100, "prb", 3), (16, 61, "subcarrier", 4), (4, 30, "prb", 2)])
def test_shards_equal_the_whole_slot(n_t, n_sub, hold, world):
    import paper_2510_01579_gb300 as pkg
    w = synth.uplink(300 + n_t, n_t, n_t, 4, n_sub=n_sub, n_sym=14, snr_db=15.0, model="kron", hold=hold)
    P = w["y"].shape[0]
    prm = pkg.Params.default(steps=100)
    with pkg.Context(0) as ctx:
        whole = _outs(P, n_t)
        ctx.detect_jobs([ctx.detect_job(T(w["H"]), T(w["y"]), T(w["noise_var"]), 4, 17, whole,
                                        T(w["chan_index"]))], prm)
        parts = _outs(P, n_t)
        batched = _outs(P, n_t)
        jobs, keep = [], []
        for r in range(world):
            sh = shard.shard_slot(w["chan_index"], n_sub, 14, world, r)
            p0, p1 = sh["p0"], sh["p1"]
            if p1 == p0:
                continue
            t = (T(w["H"][sh["c0"]:sh["c1"]]), T(w["y"][p0:p1]), T(w["noise_var"][p0:p1]), T(sh["chan_index"]))
            o = {k: v[p0:p1] for k, v in parts.items()}
            ctx.detect_jobs([ctx.detect_job(*t[:3], 4, 17, o, t[3], problem_offset=p0)], prm)
            ob = {k: v[p0:p1] for k, v in batched.items()}
            jobs.append(ctx.detect_job(*t[:3], 4, 17, ob, t[3], problem_offset=p0))
            keep.append(t)
        with pkg.Batch(0, prm, jobs, keepalive=keep) as b:
            b.run(use_graph=True)
        torch.cuda.synchronize()
    for k in whole:
        assert torch.equal(parts[k], whole[k]), k
        assert torch.equal(batched[k], whole[k]), k
