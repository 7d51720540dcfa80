"""32 users (the high-connectivity 32x32 scenario, n = 64 spins): delta-mapping
detection and the quantised solver through the C ABI, bit-exact against the
oracle, and the calls that refuse 32 users."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module")
def mm():
    import paper_2510_01579_gb300 as pkg
    ctx = pkg.Context(0)
    yield pkg, ctx
    ctx.close()


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def oparams(prm):
    return oracle.Params(**{f: getattr(prm, f) for f in ("runs", "steps", "f_mvm", "dt", "p", "a", "zeta", "eps",
                                                         "sigma0", "x_max")})


def _detect(ctx, w, prm, seed):
    out = ctx.detect(T(w["H"]), T(w["y"]), T(w["noise_var"]), w["mod_bits"], prm, seed,
                     chan_index=T(w["chan_index"]), want_energy=True, want_guess=True, want_offset=True,
                     want_ndiv=True)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("n_r,mb,runs,f_mvm,steps", [(32, 2, 32, 2, 150), (32, 4, 128, 1, 80), (48, 4, 64, 2, 100),
                                                     (32, 6, 96, 2, 60), (32, 4, 32, 3, 100), (64, 4, 64, 5, 77)])
def test_detect_32x32_bit_exact(mm, n_r, mb, runs, f_mvm, steps):
    """Shared channels (three symbols per subcarrier) go through the
    per-channel factorisation; noise variances of every other problem differ
    so half the problems factorise for themselves."""
    pkg, ctx = mm
    w = synth.uplink(3200 + n_r + mb, n_r, 32, mb, n_sub=4, n_sym=3, snr_db=16.0, hold="subcarrier")
    nv = w["noise_var"].copy()
    nv[1::2] *= np.float32(1.25)
    w = dict(w, noise_var=nv)
    prm = pkg.Params.default(runs=runs, f_mvm=f_mvm, steps=steps)
    got = _detect(ctx, w, prm, 21)
    ref = oracle.detect_batch(w["H"], w["y"], w["noise_var"], mb, oparams(prm), 21, w["chan_index"])
    assert np.array_equal(got["sym"], ref["sym"])
    assert np.array_equal(got["energy"], ref["E"])
    assert np.array_equal(got["ndiv"], ref["n_div"])
    assert np.array_equal(got["guess"], ref["g"].astype(np.int8))
    assert np.array_equal(got["offset"], ref["d"])


def test_detect_32x32_small_workspace_same_bits(mm):
    """A workspace that holds one problem but not the per-channel factors
    (so every problem factorises itself, in chunks) gives the same bits."""
    pkg, ctx = mm
    w = synth.uplink(3299, 32, 32, 4, n_sub=3, n_sym=4, snr_db=14.0, hold="subcarrier")
    prm = pkg.Params.default(steps=50)
    got = _detect(ctx, w, prm, 4)
    with pkg.Context(0, workspace_bytes=40 * 1024) as c2:
        got2 = _detect(c2, w, prm, 4)
    for k in got:
        assert np.array_equal(got[k], got2[k]), k


@pytest.mark.parametrize("runs,f_mvm", [(32, 2), (64, 1), (128, 2), (32, 4), (96, 3)])
def test_solve_ising_n64_bit_exact(mm, runs, f_mvm):
    """Random Appendix-style instances at n = 64: a stable step and one large
    enough that anneals diverge (the counts and the all-diverged result must
    agree too)."""
    pkg, ctx = mm
    A, h = synth.random_ising(640 + runs, 7, 64)
    for dt, steps in ((0.02, 120), (0.3, 40)):
        prm = pkg.Params.default(runs=runs, f_mvm=f_mvm, dt=dt, steps=steps)
        got = ctx.solve_ising(T(A), T(h), prm, seed=0xABCDEF)
        torch.cuda.synchronize()
        ref = oracle.solve_batch(A, h, None, 0, oparams(prm), 0xABCDEF)
        for k, rk in (("d", "d"), ("E", "E"), ("run", "run"), ("ndiv", "n_div")):
            assert np.array_equal(got[k].cpu().numpy(), ref[rk]), (dt, k)


def test_solve_ising_n64_with_guess_and_levels(mm):
    """The detection form (guess g, clipping to the QAM levels) at n = 64."""
    pkg, ctx = mm
    w = synth.uplink(3333, 32, 32, 4, n_sub=5, n_sym=1, snr_db=15.0, hold="problem")
    bs = [oracle.build_detect32(w["H"][p], w["y"][p], w["noise_var"][p], 4) for p in range(5)]
    Aq = np.stack([b["Aq"] for b in bs])
    hq = np.stack([b["hq"] for b in bs])
    g = np.stack([b["g"] for b in bs]).astype(np.int8)
    prm = pkg.Params.default(runs=64, steps=90)
    got = ctx.solve_ising(T(Aq), T(hq), prm, seed=5, g=T(g), level_max=3)
    torch.cuda.synchronize()
    ref = oracle.solve_batch(Aq, hq, g, 3, oparams(prm), 5)
    for k, rk in (("d", "d"), ("E", "E"), ("run", "run"), ("ndiv", "n_div")):
        assert np.array_equal(got[k].cpu().numpy(), ref[rk]), k


def test_32_users_refused_outside_the_delta_path(mm):
    pkg, ctx = mm
    w = synth.uplink(3400, 32, 32, 2, n_sub=2, n_sym=1, snr_db=10.0, hold="problem")
    H, y, nv = T(w["H"]), T(w["y"]), T(w["noise_var"])
    cases = [
        lambda: ctx.detect(H, y, nv, 2, pkg.Params.default(), 1, mapping=1),
        lambda: ctx.detect(H, y, nv, 2, pkg.Params.default(), 1, gram_precision=1),
        lambda: ctx.detect_e(H, y, nv, 2, pkg.Params.default(), 1),
        lambda: ctx.anneal_spins(T(np.zeros((1, 64, 64), np.int16)), T(np.zeros((1, 64), np.int16)),
                                 pkg.Params.default(), 1),
        lambda: ctx.set_solver_variant(32, 1),
    ]
    for i, c in enumerate(cases):
        with pytest.raises(pkg.MMGaPError) as e:
            c()
        assert e.value.status == 5, i


@pytest.mark.parametrize("runs", [64, 96, 128])
def test_cluster_split_small_calls_equal_large_calls(mm, runs):
    """A call whose problems' 32-anneal groups fit the SMs runs each problem as
    a cluster of runs/32 CTAs (combined through distributed shared memory);
    the same problems inside a larger call (one CTA each) give the same bits."""
    pkg, ctx = mm
    w = synth.uplink(3500 + runs, 32, 32, 4, n_sub=200, n_sym=1, snr_db=16.0, hold="problem")
    prm = pkg.Params.default(runs=runs, steps=60)
    big = _detect(ctx, w, prm, 8)  # 200 problems x runs/32 CTAs > the SM count: one CTA per problem
    small = _detect(ctx, dict(w, H=w["H"][:5], y=w["y"][:5], noise_var=w["noise_var"][:5],
                              chan_index=w["chan_index"][:5]), prm, 8)
    for k in big:
        assert np.array_equal(small[k], big[k][:5]), k


@pytest.mark.parametrize("n_r,mb,hold", [(32, 4, "subcarrier"), (64, 6, "problem"), (8, 2, "problem")])
def test_builder_32_users_bit_exact(mm, n_r, mb, hold):
    """Q14 couplings, field, guess, FP32 Gram and field and the normaliser of
    the 32-user builder equal the oracle's FP32 mirror (n_r = 8 < n_t: the
    regularised Gram of an under-determined system)."""
    pkg, ctx = mm
    w = synth.uplink(3600 + n_r + mb, n_r, 32, mb, n_sub=5, n_sym=2, snr_db=15.0, hold=hold)
    out = ctx.build_detect(T(w["H"]), T(w["y"]), T(w["noise_var"]), mb, chan_index=T(w["chan_index"]))
    torch.cuda.synchronize()
    for p in range(w["y"].shape[0]):
        c = int(w["chan_index"][p])
        b = oracle.build_detect32(w["H"][c], w["y"][p], w["noise_var"][p], mb)
        assert np.array_equal(out["A_q"][p].cpu().numpy(), b["Aq"]), p
        assert np.array_equal(out["h_q"][p].cpu().numpy(), b["hq"]), p
        assert np.array_equal(out["g"][p].cpu().numpy(), b["g"].astype(np.int8)), p
        assert np.array_equal(out["G"][p].cpu().numpy(), b["G32"]), p
        assert np.array_equal(out["h"][p].cpu().numpy(), b["h32"]), p
        assert int(out["sigma_exp"][p]) == b["sigma_exp"]


def test_32_users_degenerate_empty_and_bad_index(mm):
    """All-zero channel, a noise-free rank-deficient channel (the Cholesky
    pivot fails: guess from x_mmse = 0), an empty job, and an out-of-range
    channel index (flagged in the device error word)."""
    pkg, ctx = mm
    rng = np.random.default_rng(32)
    H = np.zeros((2, 32, 32), np.complex64)
    H[1] = (rng.standard_normal((32, 32)) + 1j * rng.standard_normal((32, 32))).astype(np.complex64)
    H[1][:, 31] = H[1][:, 30]
    y = (rng.standard_normal((2, 32)) + 1j * rng.standard_normal((2, 32))).astype(np.complex64)
    nv = np.zeros(2, np.float32)
    out = ctx.build_detect(T(H), T(y), T(nv), 4)
    prm = pkg.Params.default(steps=40)
    det = ctx.detect(T(H), T(y), T(nv), 4, prm, 6, want_energy=True)
    torch.cuda.synchronize()
    ref = oracle.detect_batch(H, y, nv, 4, oracle.Params(steps=40), 6, np.arange(2, dtype=np.int32))
    for p in range(2):
        b = oracle.build_detect32(H[p], y[p], nv[p], 4)
        assert np.array_equal(out["A_q"][p].cpu().numpy(), b["Aq"])
        assert np.array_equal(out["g"][p].cpu().numpy(), b["g"].astype(np.int8))
    assert not out["A_q"][0].any()
    assert np.array_equal(det["sym"].cpu().numpy(), ref["sym"])
    assert np.array_equal(det["energy"].cpu().numpy(), ref["E"])
    empty = ctx.detect(T(H), T(y[:0]), T(nv[:0]), 4, prm, 1)
    assert empty["sym"].shape == (0, 32)
    ctx.device_errors(clear=True)
    w = synth.uplink(3700, 32, 32, 2, n_sub=3, n_sym=1)
    ctx.detect(T(w["H"]), T(w["y"]), T(w["noise_var"]), 2, prm, 1, chan_index=T(np.array([0, 9, 1], np.int32)))
    torch.cuda.synchronize()
    assert ctx.device_errors(clear=True) & 1
