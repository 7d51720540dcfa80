"""Direct (binary-weighted) spin mapping on the GPU against the oracle.

Builder (J_q, c_q, guess, FP32 J and c, normaliser), general-coupling solver
(spins, energy, winning anneal, divergence count) and end-to-end detection
(symbols, energies, guesses, offsets) must equal the oracle's FP32 mirror bit
for bit, for every compiled spin count N = 2 n_t log2(M)/2 in {8, 16, 24, 32,
48, 64, 96}.
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


@pytest.fixture(scope="module")
def mm():
    import paper_2510_01579_gb300 as pkg
    ctx = pkg.Context(0)
    yield pkg, ctx
    ctx.close()


def oparams(prm):
    return oracle.Params(**{f: getattr(prm, f) for f in ("runs", "steps", "f_mvm", "dt", "p", "a", "zeta", "eps",
                                                         "sigma0", "x_max")})


@pytest.mark.parametrize("n_t,mb,n_r,hold", [(4, 2, 4, "subcarrier"), (4, 6, 8, "problem"), (8, 4, 8, "prb"),
                                              (8, 6, 12, "problem"), (16, 2, 16, "problem"), (16, 4, 16, "subcarrier"),
                                              (16, 6, 20, "problem")])
def test_build_bit_exact(mm, n_t, mb, n_r, hold):
    pkg, ctx = mm
    w = synth.uplink(500 + n_t + mb, n_r, n_t, mb, n_sub=10, n_sym=2, snr_db=12.0, hold=hold)
    P = w["y"].shape[0]
    out = ctx.build_detect(T(w["H"]), T(w["y"]), T(w["noise_var"]), mb, chan_index=T(w["chan_index"]), mapping=1)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    for p in range(P):
        r = oracle.build_direct32(w["H"][w["chan_index"][p]], w["y"][p], w["noise_var"][p], mb)
        assert np.array_equal(got["A_q"][p], r["Jq"]), p
        assert np.array_equal(got["h_q"][p], r["cq"]), p
        assert np.array_equal(got["g"][p], r["g"]), p
        assert np.array_equal(got["G"][p], r["J32"]), p
        assert np.array_equal(got["h"][p], r["c32"]), p
        assert got["sigma_exp"][p] == r["sigma_exp"], p


@pytest.mark.parametrize("N,runs,steps,f", [(8, 32, 41, 2), (16, 64, 40, 1), (24, 32, 37, 3), (32, 32, 50, 2),
                                            (48, 64, 33, 2), (64, 32, 30, 2), (96, 64, 25, 1), (96, 32, 23, 2)])
def test_general_solver_bit_exact(mm, N, runs, steps, f):
    pkg, ctx = mm
    P = 10
    Jq, cq = synth.random_ising(700 + N + f, P, N)
    for p in range(P):
        np.fill_diagonal(Jq[p], 0)
    rng = np.random.default_rng(N)
    sref = np.where(rng.random((P, N)) < 0.5, 1, -1).astype(np.int8)
    prm = pkg.Params.default(runs=runs, steps=steps, f_mvm=f)
    for with_ref in (True, False):
        out = ctx.solve_general(T(Jq), T(cq), prm, 31, s_ref=T(sref) if with_ref else None)
        torch.cuda.synchronize()
        got = {k: v.cpu().numpy() for k, v in out.items()}
        for p in range(P):
            r = oracle.cac_solve_general(Jq[p], cq[p], sref[p] if with_ref else None, oparams(prm), 31, p)
            assert np.array_equal(got["s"][p], r["s"]), (p, with_ref)
            assert got["E"][p] == r["E"] and got["run"][p] == r["run"] and got["ndiv"][p] == r["n_div"], p


def test_general_solver_divergence_and_reference(mm):
    """dt = 3 diverges every anneal: the reference (or all +1 without one) comes back."""
    pkg, ctx = mm
    Jq, cq = synth.random_ising(5, 6, 32)
    for p in range(6):
        np.fill_diagonal(Jq[p], 0)
    sref = np.ones((6, 32), np.int8)
    sref[:, ::3] = -1
    prm = pkg.Params.default(runs=32, steps=40, dt=3.0)
    for ref in (sref, None):
        out = ctx.solve_general(T(Jq), T(cq), prm, 2, s_ref=None if ref is None else T(ref))
        torch.cuda.synchronize()
        assert (out["ndiv"] == 32).all() and (out["run"] == -1).all()
        want = ref if ref is not None else np.ones((6, 32), np.int8)
        assert np.array_equal(out["s"].cpu().numpy(), want)
        for p in range(6):
            assert int(out["E"][p]) == oracle.energy_direct(Jq[p], cq[p], want[p])


@pytest.mark.parametrize("n_t,mb,snr,n_sub,steps", [(8, 2, 10.0, 64, 200), (4, 4, 14.0, 40, 200),
                                                     (16, 4, 16.0, 6, 120), (16, 6, 22.0, 3, 60),
                                                     (8, 6, 20.0, 8, 100)])
def test_detect_bit_exact(mm, n_t, mb, snr, n_sub, steps):
    pkg, ctx = mm
    w = synth.uplink(900 + n_t + mb, n_t, n_t, mb, n_sub=n_sub, n_sym=1, snr_db=snr)
    P = w["y"].shape[0]
    prm = pkg.Params.default(steps=steps)
    out = ctx.detect(T(w["H"]), T(w["y"]), T(w["noise_var"]), mb, prm, 17, chan_index=T(w["chan_index"]),
                     want_energy=True, want_guess=True, want_offset=True, want_ndiv=True, mapping=1)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    for p in range(P):
        r = oracle.detect_direct(w["H"][w["chan_index"][p]], w["y"][p], w["noise_var"][p], mb, oparams(prm), 17, p)
        assert np.array_equal(got["sym"][p], r["sym"]), p
        assert got["energy"][p] == r["E"] and got["ndiv"][p] == r["n_div"], p
        assert np.array_equal(got["guess"][p], r["g"]), p
        x = oracle.direct_lattice(n_t, mb, r["s"])
        assert np.array_equal(got["offset"][p], (x - r["g"]) // 2), p


def test_detect_qpsk_near_ml_and_better_than_mmse(mm):
    """8x8 QPSK at 10 dB (16 spins): bit errors of the direct-mapping detector
    within 25 % of exhaustive ML and below MMSE."""
    pkg, ctx = mm
    w = synth.uplink(41, 8, 8, 2, n_sub=64, n_sym=1, snr_db=10.0)
    out = ctx.detect(T(w["H"]), T(w["y"]), T(w["noise_var"]), 2, pkg.Params.default(), 3,
                     chan_index=T(w["chan_index"]), want_guess=True, mapping=1)
    torch.cuda.synchronize()
    err = synth.bit_errors(out["sym"].cpu().numpy(), w["sym"], 2)
    g = out["guess"].cpu().numpy().astype(int)
    mmse = synth.bit_errors(((g[:, :8] + 1) // 2) * 2 + (g[:, 8:] + 1) // 2, w["sym"], 2)
    ml = 0
    for p in range(64):
        _, x = oracle.ml_exhaustive(w["H"][w["chan_index"][p]].astype(np.complex128),
                                    w["y"][p].astype(np.complex128), 2)
        ml += synth.bit_errors((((x[:8] + 1) // 2) * 2 + (x[8:] + 1) // 2)[None], w["sym"][p:p + 1], 2)
    assert err <= max(ml * 1.25, ml + 3) and err <= mmse


def test_direct_mapping_arguments(mm):
    pkg, ctx = mm
    w = synth.uplink(3, 2, 2, 4, n_sub=2, n_sym=1)
    with pytest.raises(pkg.MMGaPError) as e:  # n_t = 2 is not compiled for the direct form
        ctx.detect(T(w["H"]), T(w["y"]), T(w["noise_var"]), 4, pkg.Params.default(), 1,
                   chan_index=T(w["chan_index"]), mapping=1)
    assert e.value.status == 5
    w = synth.uplink(3, 16, 16, 6, n_sub=2, n_sym=1)
    with pytest.raises(pkg.MMGaPError) as e:  # 96 spins x 4 threads per anneal x 96 anneals > 256 threads
        ctx.detect(T(w["H"]), T(w["y"]), T(w["noise_var"]), 6, pkg.Params.default(runs=96), 1,
                   chan_index=T(w["chan_index"]), mapping=1)
    assert e.value.status == 5
    with pytest.raises(pkg.MMGaPError) as e:
        ctx.detect(T(w["H"]), T(w["y"]), T(w["noise_var"]), 6, pkg.Params.default(), 1,
                   chan_index=T(w["chan_index"]), mapping=2)
    assert e.value.status == 1
    with pytest.raises(pkg.MMGaPError) as e:
        ctx.solve_general(torch.zeros((1, 12, 12), dtype=torch.int16, device=DEV),
                          torch.zeros((1, 12), dtype=torch.int16, device=DEV), pkg.Params.default(), 1)
    assert e.value.status == 5
    out = {"sym": torch.empty((2, 16), dtype=torch.uint8, device=DEV)}
    job = ctx.detect_job(T(w["H"]), T(w["y"]), T(w["noise_var"]), 6, 1, out, T(w["chan_index"]), mapping=1)
    with pytest.raises(pkg.MMGaPError):
        pkg.Batch(0, pkg.Params.default(), [job])


def test_direct_chunked_workspace_is_deterministic(mm):
    """A workspace that holds a few problems per chunk gives the same bits as one chunk."""
    pkg, ctx = mm
    w = synth.uplink(77, 8, 8, 4, n_sub=6, n_sym=4, snr_db=14.0)
    prm = pkg.Params.default(steps=60)
    outs = []
    for ws in (24 * 1024, 0):
        with pkg.Context(0, workspace_bytes=ws) as c:
            o = c.detect(T(w["H"]), T(w["y"]), T(w["noise_var"]), 4, prm, 5, chan_index=T(w["chan_index"]),
                         want_energy=True, want_guess=True, want_offset=True, want_ndiv=True, mapping=1)
            torch.cuda.synchronize()
            outs.append({k: v.cpu().numpy() for k, v in o.items()})
    for k in outs[0]:
        assert np.array_equal(outs[0][k], outs[1][k]), k
    for p in (0, 11, 23):
        r = oracle.detect_direct(w["H"][w["chan_index"][p]], w["y"][p], w["noise_var"][p], 4, oparams(prm), 5, p)
        assert np.array_equal(outs[0]["sym"][p], r["sym"]) and outs[0]["energy"][p] == r["E"], p
