"""Slot-scale parity in the launch configurations the benchmarks time.

* The mixed-size batched launch (16x16 16-QAM + 16x16 64-QAM + 8x8 QPSK, a
  full 100 MHz slot of each, 137,592 problems in one CUDA-graph launch):
  sampled problems of every class against the oracle, one by one.
* A full 16x16 16-QAM VPP slot (3276 channels, FP64 inverse) sampled against
  the oracle, and properties that hold at any size (perturbations in
  {-1, 0, 1}, energies <= 0, power equal to the transmit vector's norm).
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def oparams(prm):
    return oracle.Params(**{f: getattr(prm, f) for f in ("runs", "steps", "f_mvm", "dt", "p", "a", "zeta", "eps",
                                                         "sigma0", "x_max")})


def test_mixed_batched_slot_sampled():
    import paper_2510_01579_gb300 as pkg
    prm = pkg.Params.default()
    specs = [(16, 4, 16.0, 31), (16, 6, 24.0, 32), (8, 2, 10.0, 33)]
    with pkg.Context(0) as ctx:
        ws, jobs, outs, keep = [], [], [], []
        for n_t, mb, snr, seed in specs:
            w = synth.uplink(seed, n_t, n_t, mb, snr_db=snr)
            t = [T(w[k]) for k in ("H", "y", "noise_var", "chan_index")]
            o = {"sym": torch.empty((w["y"].shape[0], n_t), dtype=torch.uint8, device=DEV),
                 "energy": torch.empty(w["y"].shape[0], dtype=torch.int32, device=DEV),
                 "ndiv": torch.empty(w["y"].shape[0], dtype=torch.int32, device=DEV)}
            ws.append(w)
            outs.append(o)
            keep.append(t)
            jobs.append(ctx.detect_job(t[0], t[1], t[2], mb, seed, o, t[3]))
        with pkg.Batch(0, prm, jobs, keepalive=(keep, outs)) as b:
            b.run(use_graph=True)
            torch.cuda.synchronize()
    assert sum(w["y"].shape[0] for w in ws) == 3 * 3276 * 14
    for (n_t, mb, snr, seed), w, o in zip(specs, ws, outs):
        got = {k: v.cpu().numpy() for k, v in o.items()}
        P = w["y"].shape[0]
        for p in [0, 13, P // 3, P - 1] + list(np.random.default_rng(seed).integers(0, P, 4)):
            p = int(p)
            c = int(w["chan_index"][p])
            bld = oracle.build_detect32(w["H"][c], w["y"][p], w["noise_var"][p], mb)
            r = oracle.cac_solve(bld["Aq"], bld["hq"], bld["g"], (1 << (mb // 2)) - 1, oparams(prm), seed, p)
            sym = oracle.decode_detect(n_t, mb, bld["g"], r["d"])
            assert np.array_equal(got["sym"][p], sym), (n_t, mb, p)
            assert got["energy"][p] == r["E"] and got["ndiv"][p] == r["n_div"], (n_t, mb, p)
        assert np.all(got["energy"] <= 0)


def test_precode_full_slot_sampled():
    import paper_2510_01579_gb300 as pkg
    d = synth.downlink(4016, 16, 16, 4)
    prm = pkg.Params.default()
    with pkg.Context(0, workspace_bytes=512 << 20) as ctx:
        out = ctx.precode(T(d["H"]), T(d["u_sym"]), 4, prm, 5, chan_index=T(d["chan_index"]), want_energy=True,
                          want_ndiv=True)
        torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    P = d["u_sym"].shape[0]
    assert P == 3276
    for p in [0, 1, P // 2, P - 1] + list(np.random.default_rng(4).integers(0, P, 6)):
        p = int(p)
        Hc = d["H"][int(d["chan_index"][p])].astype(np.complex128)
        b = oracle.build_precode(Hc, d["u_sym"][p], 4)
        r = oracle.cac_solve(b["Aq"], b["hq"], None, 0, oparams(prm), 5, p)
        v, x, pw = oracle.precode_output(Hc, b["Q"], d["u_sym"][p], r["d"], 4)
        assert np.array_equal(got["v"][p], v), p
        assert np.array_equal(got["x"][p], x) and got["power"][p] == pw, p
        assert got["energy"][p] == r["E"] and got["ndiv"][p] == r["n_div"], p
    assert np.all(np.abs(got["v"]) <= 1) and np.all(got["energy"] <= 0)
    pw = np.sum(np.abs(got["x"].astype(np.complex128)) ** 2, axis=1)
    assert np.allclose(pw, got["power"], rtol=1e-4)
