"""Caller-supplied guess (mmgap_detect_job.guess_in) against the oracle.

The paper makes the guess an input of the pre-processing (Sec. 3.2; the VPP
form of Sec. 3.3 uses the zero guess): the delta-Ising problem is built around
it instead of the MMSE solution.  The builder's outputs around a given guess,
and detection around it, must equal the oracle's bit for bit; the batched
launch and the server must give the per-job path's bits.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)
FIELDS = ("runs", "steps", "f_mvm", "dt", "p", "a", "zeta", "eps", "sigma0", "x_max", "early_exit")


@pytest.fixture(scope="module")
def mm():
    import paper_2510_01579_gb300 as pkg
    ctx = pkg.Context(0)
    yield pkg, ctx
    ctx.close()


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def oparams(prm):
    return oracle.Params(**{f: getattr(prm, f) for f in FIELDS})


def _guesses(w, seed):
    """A valid lattice guess per problem: the transmitted symbols with a few
    dimensions moved to a neighbouring alphabet point."""
    rng = np.random.default_rng(seed)
    n_t, mb = w["n_t"], w["mod_bits"]
    side = 1 << (mb // 2)
    L = side - 1
    sym = w["sym"].astype(int)
    g = np.concatenate([2 * (sym // side) - L, 2 * (sym % side) - L], axis=1)
    move = rng.random(g.shape) < 0.3
    step = np.where(rng.random(g.shape) < 0.5, -2, 2)
    g = np.where(move, np.clip(g + step, -L, L), g)
    return g.astype(np.int8)


@pytest.mark.parametrize("n_r,nt,mb,hold", [(16, 16, 4, "subcarrier"), (8, 8, 6, "problem"), (12, 8, 2, "prb"),
                                            (5, 3, 4, "problem"), (32, 32, 4, "subcarrier")])
def test_build_around_given_guess_bit_exact(mm, n_r, nt, mb, hold):
    pkg, ctx = mm
    w = synth.uplink(80 + nt + mb, n_r, nt, mb, n_sub=7, n_sym=3, snr_db=14.0, hold=hold)
    g = _guesses(w, nt)
    out = ctx.build_detect(T(w["H"]), T(w["y"]), T(w["noise_var"]), mb, chan_index=T(w["chan_index"]), guess=T(g))
    torch.cuda.synchronize()
    for p in range(w["y"].shape[0]):
        c = int(w["chan_index"][p])
        b = oracle.build_detect32(w["H"][c], w["y"][p], w["noise_var"][p], mb, g_in=g[p].astype(np.int32))
        assert np.array_equal(out["g"][p].cpu().numpy(), g[p]), p
        assert np.array_equal(out["A_q"][p].cpu().numpy(), b["Aq"]), p
        assert np.array_equal(out["h_q"][p].cpu().numpy(), b["hq"]), p
        assert np.array_equal(out["h"][p].cpu().numpy(), b["h32"]), p
        assert int(out["sigma_exp"][p]) == b["sigma_exp"], p
    assert ctx.device_errors() == 0


@pytest.mark.parametrize("nt,mb,K", [(16, 4, 0), (8, 4, 3), (4, 6, 0), (32, 4, 0)])
def test_detect_around_given_guess_bit_exact(mm, nt, mb, K):
    pkg, ctx = mm
    w = synth.uplink(90 + nt, nt, nt, mb, n_sub=6, n_sym=4, snr_db=15.0)
    g = _guesses(w, 3 + nt)
    prm = pkg.Params.default(steps=120, early_exit=K)
    out = ctx.detect(T(w["H"]), T(w["y"]), T(w["noise_var"]), mb, prm, 41, chan_index=T(w["chan_index"]),
                     want_energy=True, want_guess=True, want_offset=True, guess=T(g))
    torch.cuda.synchronize()
    Lm = (1 << (mb // 2)) - 1
    for p in range(w["y"].shape[0]):
        c = int(w["chan_index"][p])
        b = oracle.build_detect32(w["H"][c], w["y"][p], w["noise_var"][p], mb, g_in=g[p].astype(np.int32))
        r = oracle.cac_solve(b["Aq"], b["hq"], b["g"], Lm, oparams(prm), 41, p)
        assert np.array_equal(out["guess"][p].cpu().numpy(), g[p]), p
        assert np.array_equal(out["offset"][p].cpu().numpy(), r["d"]), p
        assert int(out["energy"][p]) == r["E"], p
        assert np.array_equal(out["sym"][p].cpu().numpy(), oracle.decode_detect(nt, mb, b["g"], r["d"])), p


def test_given_guess_in_batch_and_server_equals_per_job(mm):
    pkg, ctx = mm
    prm = pkg.Params.default(steps=90)
    ws = [synth.uplink(95, 16, 16, 4, n_sub=10, n_sym=14, snr_db=16.0),
          synth.uplink(96, 8, 8, 2, n_sub=24, n_sym=14, snr_db=8.0, model="kron", hold="prb"),
          synth.uplink(97, 32, 32, 4, n_sub=3, n_sym=4, snr_db=18.0)]
    keep, jobs, outs, refs = [], [], [], []
    for i, w in enumerate(ws):
        t = [T(w[k]) for k in ("H", "y", "noise_var", "chan_index")] + [T(_guesses(w, 50 + i))]
        P, nt = w["y"].shape[0], w["n_t"]
        o = {"sym": torch.full((P, nt), 255, dtype=torch.uint8, device=DEV),
             "energy": torch.full((P,), 3, dtype=torch.int32, device=DEV)}
        r = {k: torch.empty_like(v) for k, v in o.items()}
        ctx.detect_jobs([ctx.detect_job(t[0], t[1], t[2], w["mod_bits"], 60 + i, r, t[3], guess=t[4])], prm)
        keep.append(t)
        outs.append(o)
        refs.append(r)
        jobs.append(ctx.detect_job(t[0], t[1], t[2], w["mod_bits"], 60 + i, o, t[3], guess=t[4]))
    with pkg.Batch(0, prm, jobs, keepalive=(keep, outs)) as b:
        b.run(use_graph=True)
        torch.cuda.synchronize()
    for o, r in zip(outs, refs):
        for k in o:
            assert torch.equal(o[k], r[k]), k
    for o in outs:
        for v in o.values():
            v.fill_(7)
    with pkg.Server(0, prm, scratch_bytes=64 << 20, n_lanes=2, max_n_t=32, max_n_r=32) as srv:
        tickets = [srv.submit(j) for j in jobs]
        for tk in tickets:
            srv.wait(tk, timeout_us=60_000_000)
    for o, r in zip(outs, refs):
        for k in o:
            assert torch.equal(o[k], r[k]), k


def test_guess_outside_the_alphabet_is_flagged(mm):
    pkg, ctx = mm
    w = synth.uplink(98, 8, 8, 4, n_sub=4, n_sym=2, snr_db=15.0)
    g = _guesses(w, 1)
    assert ctx.device_errors() == 0
    ctx.detect(T(w["H"]), T(w["y"]), T(w["noise_var"]), 4, pkg.Params.default(steps=20), 1,
               chan_index=T(w["chan_index"]), guess=T(g))
    assert ctx.device_errors() == 0
    bad = g.copy()
    bad[3, 5] = 2       # even: not a lattice point
    bad[6, 0] = 5       # beyond +-3 for 16-QAM
    ctx.detect(T(w["H"]), T(w["y"]), T(w["noise_var"]), 4, pkg.Params.default(steps=20), 1,
               chan_index=T(w["chan_index"]), guess=T(bad))
    assert ctx.device_errors() == 4


def test_guess_refusals(mm):
    pkg, ctx = mm
    w = synth.uplink(99, 8, 8, 4, n_sub=3, n_sym=2)
    g = T(_guesses(w, 2))
    with pytest.raises(pkg.MMGaPError) as e:  # the direct mapping anneals around its own reference
        ctx.detect(T(w["H"]), T(w["y"]), T(w["noise_var"]), 4, pkg.Params.default(), 1,
                   chan_index=T(w["chan_index"]), mapping=1, guess=g)
    assert e.value.status == 5
    o = {"sym": torch.empty((w["y"].shape[0], 8), dtype=torch.uint8, device=DEV)}
    job = ctx.detect_job(T(w["H"]), T(w["y"]), T(w["noise_var"]), 4, 1, o, T(w["chan_index"]), guess=g)
    import ctypes
    from paper_2510_01579_gb300 import binding
    cp = pkg.Params.default()._c()
    st = binding._lib.mmgap_detect_e(ctx._h, ctypes.byref(cp), ctypes.byref(job), 1, None, None, None,
                                     ctx._stream())
    assert st == 5  # MMGaP-E makes its own guesses
