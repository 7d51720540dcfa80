"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Integer results (guesses, Q14 couplings, offsets, energies, winning anneal,
divergence counts, symbols, perturbations) must be identical; FP32 Gram and
field must equal the oracle's FP32 mirror bit for bit and the FP64 truth
within 1e-5 normwise.
"""
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


def oracle_detect_one(w, p, prm, seed):
    """Oracle pipeline for problem p of an uplink workload (FP32 mirror)."""
    c = int(w["chan_index"][p])
    n_t, mb = w["n_t"], w["mod_bits"]
    b = oracle.build_detect32(w["H"][c], w["y"][p], w["noise_var"][p], mb)
    r = oracle.cac_solve(b["Aq"], b["hq"], b["g"], (1 << (mb // 2)) - 1, oparams(prm), seed, p)
    sym = oracle.decode_detect(n_t, mb, b["g"], r["d"])
    return dict(sym=sym, E=r["E"], g=b["g"], d=r["d"], ndiv=r["n_div"], run=r["run"])


# ------------------------------------------------------------------ solver
@pytest.mark.parametrize("nt,runs,f_mvm,steps", [(1, 32, 2, 200), (2, 64, 2, 150), (3, 32, 3, 100),
                                                  (4, 32, 2, 200), (8, 32, 2, 200), (8, 128, 1, 64),
                                                  (16, 32, 2, 200), (16, 96, 5, 37)])
def test_solver_bit_exact(mm, nt, runs, f_mvm, steps):
    pkg, ctx = mm
    w = synth.uplink(300 + nt, nt + 2, nt, 4, n_sub=11, n_sym=1, snr_db=12.0, hold="problem")
    bs = [oracle.build_detect32(w["H"][p], w["y"][p], w["noise_var"][p], 4) for p in range(11)]
    Aq = np.stack([b["Aq"] for b in bs])
    hq = np.stack([b["hq"] for b in bs])
    g = np.stack([b["g"] for b in bs]).astype(np.int8)
    prm = pkg.Params.default(runs=runs, f_mvm=f_mvm, steps=steps)
    got = ctx.solve_ising(T(Aq), T(hq), prm, seed=0x1234_5678_9ABC, g=T(g), level_max=3)
    torch.cuda.synchronize()
    ref = oracle.solve_batch(Aq, hq, g, 3, oparams(prm), 0x1234_5678_9ABC)
    assert np.array_equal(got["d"].cpu().numpy(), ref["d"])
    assert np.array_equal(got["E"].cpu().numpy(), ref["E"])
    assert np.array_equal(got["run"].cpu().numpy(), ref["run"])
    assert np.array_equal(got["ndiv"].cpu().numpy(), ref["n_div"])


def test_solver_random_instances_and_divergence(mm):
    """Appendix-style random Ising instances without clipping, including a
    step size large enough to make anneals diverge (counts must agree)."""
    pkg, ctx = mm
    A, h = synth.random_ising(7, 9, 16)
    for dt in (0.02, 0.3):
        prm = pkg.Params.default(dt=dt, steps=120)
        got = ctx.solve_ising(T(A), T(h), prm, seed=99)
        torch.cuda.synchronize()
        ref = oracle.solve_batch(A, h, None, 0, oparams(prm), 99)
        for k, rk in (("d", "d"), ("E", "E"), ("run", "run"), ("ndiv", "n_div")):
            assert np.array_equal(got[k].cpu().numpy(), ref[rk]), (dt, k)
    assert ref["n_div"].sum() > 0  # the large step really diverges


def test_solver_zero_steps(mm):
    """steps = 0: spins are the signs of the Philox initial amplitudes."""
    pkg, ctx = mm
    A, h = synth.random_ising(8, 5, 8)
    prm = pkg.Params.default(steps=0)
    got = ctx.solve_ising(T(A), T(h), prm, seed=3)
    torch.cuda.synchronize()
    ref = oracle.solve_batch(A, h, None, 0, oparams(prm), 3)
    assert np.array_equal(got["d"].cpu().numpy(), ref["d"])
    assert np.array_equal(got["E"].cpu().numpy(), ref["E"])


# ----------------------------------------------------------------- builder
@pytest.mark.parametrize("n_r,nt,mb,hold", [(8, 8, 4, "problem"), (16, 16, 4, "subcarrier"), (16, 16, 6, "problem"),
                                            (12, 8, 2, "prb"), (4, 8, 4, "problem"), (64, 16, 6, "problem"),
                                            (1, 1, 2, "problem"), (5, 3, 4, "problem")])
def test_builder_bit_exact(mm, n_r, nt, mb, hold):
    pkg, ctx = mm
    w = synth.uplink(400 + n_r + nt, n_r, nt, mb, n_sub=13, n_sym=3, snr_db=14.0, hold=hold)
    out = ctx.build_detect(T(w["H"]), T(w["y"]), T(w["noise_var"]), mb, chan_index=T(w["chan_index"]))
    torch.cuda.synchronize()
    P = w["y"].shape[0]
    n = 2 * nt
    k = oracle.qam_kappa(mb)
    for p in range(P):
        c = int(w["chan_index"][p])
        b = oracle.build_detect32(w["H"][c], w["y"][p], w["noise_var"][p], mb)
        assert np.array_equal(out["A_q"][p].cpu().numpy(), b["Aq"]), p
        assert np.array_equal(out["h_q"][p].cpu().numpy(), b["hq"]), p
        assert np.array_equal(out["g"][p].cpu().numpy(), b["g"].astype(np.int8)), p
        assert np.array_equal(out["G"][p].cpu().numpy(), b["G32"]), p
        assert np.array_equal(out["h"][p].cpu().numpy(), b["h32"]), p
        assert int(out["sigma_exp"][p]) == b["sigma_exp"]
        # FP64 truth within 1e-5 normwise
        b64 = oracle.build_detect64(w["H"][c].astype(np.complex128), w["y"][p].astype(np.complex128),
                                    float(w["noise_var"][p]), mb, g_in=b["g"])
        Hs = k * w["H"][c].astype(np.complex128)
        Hr = np.abs(np.block([[Hs.real, -Hs.imag], [Hs.imag, Hs.real]]))
        assert np.all(np.abs(out["G"][p].cpu().numpy() - b64["G"]) <= 1e-5 * (Hr.T @ Hr))
        yr = np.concatenate([w["y"][p].real, w["y"][p].imag]).astype(np.float64)
        zb = np.abs(yr) + Hr @ np.abs(b["g"])
        assert np.all(np.abs(out["h"][p].cpu().numpy() - b64["h"]) <= 1e-5 * (Hr.T @ zb))
    assert out["A_q"].shape == (P, n, n)


def test_builder_degenerate_inputs(mm):
    """All-zero channel (sigma = 1, zero couplings), noise-free rank-deficient
    channel (Cholesky pivot fails -> guess from x_mmse = 0)."""
    pkg, ctx = mm
    H = np.zeros((2, 4, 4), np.complex64)
    rng = np.random.default_rng(1)
    H[1] = (rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))).astype(np.complex64)
    H[1][:, 3] = H[1][:, 2]  # rank deficient
    y = (rng.standard_normal((2, 4)) + 1j * rng.standard_normal((2, 4))).astype(np.complex64)
    nv = np.zeros(2, np.float32)
    out = ctx.build_detect(T(H), T(y), T(nv), 4)
    torch.cuda.synchronize()
    for p in range(2):
        b = oracle.build_detect32(H[p], y[p], nv[p], 4)
        assert np.array_equal(out["A_q"][p].cpu().numpy(), b["Aq"])
        assert np.array_equal(out["h_q"][p].cpu().numpy(), b["hq"])
        assert np.array_equal(out["g"][p].cpu().numpy(), b["g"].astype(np.int8))
    assert not out["A_q"][0].any()


# --------------------------------------------------------------- end to end
def _detect(ctx, w, prm, seed, **kw):
    out = ctx.detect(T(w["H"]), T(w["y"]), T(w["noise_var"]), w["mod_bits"], prm, seed,
                     chan_index=T(w["chan_index"]), want_energy=True, want_guess=True, want_offset=True,
                     want_ndiv=True, **kw)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_detect_small_config_bit_exact_and_ml(mm):
    """8x8 QPSK, 64 problems, i.i.d. CN(0,1), 10 dB, 32 runs x 200 steps:
    bit-exact against the oracle; the oracle's exhaustive 4^8 ML search shows
    how often the result is the ML solution."""
    pkg, ctx = mm
    w = synth.uplink(1, 8, 8, 2, n_sub=64, n_sym=1, snr_db=10.0, hold="problem")
    prm = pkg.Params.default(runs=32, steps=200)
    got = _detect(ctx, w, prm, 11)
    ref = oracle.detect_batch(w["H"], w["y"], w["noise_var"], 2, oparams(prm), 11, w["chan_index"])
    assert np.array_equal(got["sym"], ref["sym"])
    assert np.array_equal(got["energy"], ref["E"])
    assert np.array_equal(got["ndiv"], ref["n_div"])
    assert np.array_equal(got["guess"], ref["g"].astype(np.int8))
    assert np.array_equal(got["offset"], ref["d"])
    hits = 0
    for p in range(64):
        ml, _ = oracle.ml_exhaustive(w["H"][p].astype(np.complex128), w["y"][p].astype(np.complex128), 2)
        xh = synth.symbols_to_complex(got["sym"][p], 2)
        obj = np.linalg.norm(w["y"][p].astype(np.complex128) - w["H"][p].astype(np.complex128) @ xh) ** 2
        hits += obj <= ml * (1 + 1e-6) + 1e-9
    assert hits >= 60


def test_qpsk_ber_ordering_over_snr(mm):
    """8x8 QPSK, 96 problems per SNR (i.i.d. CN(0,1)), 32 x 200 anneals: MMGaP
    never has a larger ML objective than the MMSE guess (the selection energy
    is exact up to the couplings' Q14 rounding), its bit errors stay close to
    exhaustive 4^8 ML's at every SNR (QPSK: the delta neighbourhood covers the
    alphabet) and below MMSE's wherever MMSE makes errors."""
    pkg, ctx = mm
    prm = pkg.Params.default()
    for snr in (0.0, 5.0, 10.0, 15.0):
        w = synth.uplink(int(30 + snr), 8, 8, 2, n_sub=96, n_sym=1, snr_db=snr, hold="problem")
        got = _detect(ctx, w, prm, 13)
        g = got["guess"].astype(int)
        mmse = ((g[:, :8] + 1) // 2) * 2 + (g[:, 8:] + 1) // 2
        ml = np.zeros_like(w["sym"])
        for p in range(96):
            H, y = w["H"][p].astype(np.complex128), w["y"][p].astype(np.complex128)
            _, x = oracle.ml_exhaustive(H, y, 2)
            ml[p] = ((x[:8] + 1) // 2) * 2 + (x[8:] + 1) // 2
            obj = lambda s: np.linalg.norm(y - H @ synth.symbols_to_complex(s, 2)) ** 2
            # (up to the Q14 rounding of the energy that decides the selection)
            assert obj(got["sym"][p]) <= obj(mmse[p]) * (1 + 1e-3) + 1e-3, (snr, p)
        e_ml, e_mm, e_mmse = (synth.bit_errors(s, w["sym"], 2) for s in (ml, got["sym"], mmse))
        assert e_mm <= 1.5 * e_ml + 4, (snr, e_ml, e_mm)
        assert e_mm < e_mmse or e_mmse == 0, (snr, e_mm, e_mmse)


def test_detect_prb_kronecker_bit_exact(mm):
    """8x8 16-QAM, Kronecker rho = 0.5, channel held per PRB (12 subcarriers x
    14 symbols), an SNR sweep across problems."""
    pkg, ctx = mm
    snr = np.repeat(np.arange(0, 35, 5.0), 6)[:36 * 1]
    w = synth.uplink(2, 8, 8, 4, n_sub=36, n_sym=1, snr_db=snr[:36], model="kron", hold="prb")
    prm = pkg.Params.default()
    got = _detect(ctx, w, prm, 5)
    ref = oracle.detect_batch(w["H"], w["y"], w["noise_var"], 4, oparams(prm), 5, w["chan_index"])
    assert np.array_equal(got["sym"], ref["sym"])
    assert np.array_equal(got["energy"], ref["E"])


def test_detect_chunked_workspace_is_deterministic(mm):
    """A workspace that forces many chunks gives the same bits as one chunk."""
    pkg, _ = mm
    w = synth.uplink(3, 8, 8, 4, n_sub=10, n_sym=7, snr_db=12.0)
    prm = pkg.Params.default(steps=80)
    with pkg.Context(0, workspace_bytes=8 * 1024) as small, pkg.Context(0) as big:
        a = _detect(small, w, prm, 21)
        b = _detect(big, w, prm, 21)
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    ref = oracle.detect_batch(w["H"], w["y"], w["noise_var"], 4, oparams(prm), 21, w["chan_index"])
    assert np.array_equal(a["sym"], ref["sym"])


@pytest.mark.parametrize("n_t,hold", [(16, "subcarrier"), (8, "prb")])
def test_detect_per_channel_factorisation(mm, n_t, hold):
    """Channels shared by several problems are factorised once; problems whose
    noise variance differs from their channel's first problem factorise for
    themselves.  With half the noise variances changed, every problem still
    equals the oracle (which factorises per problem), and a workspace too small
    for the per-channel factors (so no sharing at all) gives the same bits."""
    pkg, ctx = mm
    w = synth.uplink(660 + n_t, n_t, n_t, 4, n_sub=24, n_sym=14, snr_db=14.0, hold=hold)
    nv = w["noise_var"].copy()
    nv[1::2] *= np.float32(1.5)
    w = dict(w, noise_var=nv)
    prm = pkg.Params.default(steps=60)
    got = _detect(ctx, w, prm, 9)
    small = 3 * 1024 if n_t == 8 else 40 * 1024  # holds a problem but not the per-channel factors
    with pkg.Context(0, workspace_bytes=small) as c2:
        got2 = _detect(c2, w, prm, 9)
    for k in got:
        assert np.array_equal(got[k], got2[k]), k
    ref = oracle.detect_batch(w["H"], w["y"], w["noise_var"], 4, oparams(prm), 9, w["chan_index"])
    assert np.array_equal(got["sym"], ref["sym"]) and np.array_equal(got["energy"], ref["E"])
    assert np.array_equal(got["guess"], ref["g"].astype(np.int8))


def test_detect_mixed_jobs_one_call(mm):
    """Jobs of different sizes in one call equal their separate calls."""
    pkg, ctx = mm
    prm = pkg.Params.default(steps=60)
    ws = [synth.uplink(10, 16, 16, 6, n_sub=5, n_sym=2), synth.uplink(11, 8, 8, 2, n_sub=7, n_sym=2),
          synth.uplink(12, 4, 4, 4, n_sub=3, n_sym=2)]
    tens, outs, jobs = [], [], []
    for i, w in enumerate(ws):
        t = dict(H=T(w["H"]), y=T(w["y"]), nv=T(w["noise_var"]), ci=T(w["chan_index"]))
        o = {"sym": torch.empty((w["y"].shape[0], w["n_t"]), dtype=torch.uint8, device=DEV),
             "energy": torch.empty(w["y"].shape[0], dtype=torch.int32, device=DEV)}
        tens.append(t)
        outs.append(o)
        jobs.append(ctx.detect_job(t["H"], t["y"], t["nv"], w["mod_bits"], 100 + i, o, t["ci"]))
    ctx.detect_jobs(jobs, prm)
    torch.cuda.synchronize()
    for i, w in enumerate(ws):
        alone = _detect(ctx, w, prm, 100 + i)
        assert np.array_equal(outs[i]["sym"].cpu().numpy(), alone["sym"])
        assert np.array_equal(outs[i]["energy"].cpu().numpy(), alone["energy"])


def test_detect_sampled_full_slot_16x16(mm):
    """Full 100 MHz slot of 16x16 16-QAM (3276 x 14 problems, i.i.d. Rayleigh,
    H per subcarrier) in the launch configuration the benchmark times;
    sampled problems checked one by one against the oracle."""
    pkg, ctx = mm
    w = synth.uplink(2025, 16, 16, 4, snr_db=16.0)
    prm = pkg.Params.default()
    with pkg.Context(0, workspace_bytes=512 << 20) as big:
        got = _detect(big, w, prm, 77)
    P = w["y"].shape[0]
    assert P == 3276 * 14
    idx = [0, 1, 13, 14, P // 2, P - 15, P - 1] + list(np.random.default_rng(5).integers(0, P, 9))
    for p in idx:
        r = oracle_detect_one(w, int(p), prm, 77)
        assert np.array_equal(got["sym"][p], r["sym"]), p
        assert got["energy"][p] == r["E"], p
        assert got["ndiv"][p] == r["ndiv"], p
    # properties that hold at any size
    assert np.all(got["energy"] <= 0)
    assert np.all(np.abs(got["offset"]) <= 1)
    L = 3
    lat = got["guess"].astype(int) + 2 * got["offset"].astype(int)
    assert np.all(np.abs(lat) <= L) and np.all(lat % 2 != 0)


def test_detect_sampled_full_slot_8x8_prb(mm):
    """100 MHz slot of 8x8 16-QAM, Kronecker rho = 0.5, H per PRB."""
    pkg, ctx = mm
    w = synth.uplink(2026, 8, 8, 4, snr_db=15.0, model="kron", hold="prb")
    prm = pkg.Params.default()
    got = _detect(ctx, w, prm, 78)
    P = w["y"].shape[0]
    for p in [0, 167, 168, P - 1] + list(np.random.default_rng(6).integers(0, P, 8)):
        r = oracle_detect_one(w, int(p), prm, 78)
        assert np.array_equal(got["sym"][p], r["sym"]), p
        assert got["energy"][p] == r["E"], p


def test_mmgap_lowers_ber_against_mmse(mm):
    """Behaviour at slot scale: MMGaP BER < MMSE BER at 15 dB (16x16 16-QAM)."""
    pkg, ctx = mm
    w = synth.uplink(31, 16, 16, 4, n_sub=256, n_sym=2, snr_db=15.0)
    got = _detect(ctx, w, pkg.Params.default(), 1)
    side = 4
    g = got["guess"].astype(int)
    mmse_sym = ((g[:, :16] + 3) // 2) * side + (g[:, 16:] + 3) // 2
    assert synth.bit_errors(got["sym"], w["sym"], 4) < 0.6 * synth.bit_errors(mmse_sym, w["sym"], 4)


# ------------------------------------------------------------------- precode
@pytest.mark.parametrize("nu,nt,mb", [(2, 2, 4), (8, 8, 4), (16, 16, 4), (4, 8, 2), (3, 3, 6)])
def test_precode_bit_exact(mm, nu, nt, mb):
    pkg, ctx = mm
    d = synth.downlink(500 + nu, nu, nt, mb, n_sub=9, n_sym=2)
    prm = pkg.Params.default(steps=120)
    out = ctx.precode(T(d["H"]), T(d["u_sym"]), mb, prm, 13, chan_index=T(d["chan_index"]), want_energy=True,
                      want_ndiv=True)
    torch.cuda.synchronize()
    ref = oracle.precode_batch(d["H"], d["u_sym"], mb, oparams(prm), 13, d["chan_index"])
    assert np.array_equal(out["v"].cpu().numpy(), ref["v"])
    assert np.array_equal(out["energy"].cpu().numpy(), ref["E"])
    assert np.array_equal(out["ndiv"].cpu().numpy(), ref["n_div"])
    assert np.array_equal(out["x"].cpu().numpy(), ref["x"])
    assert np.array_equal(out["power"].cpu().numpy(), ref["power"])
    # in aggregate VPP needs less power than zero forcing (v = 0 is the fallback)
    zf = np.array([np.linalg.norm(np.linalg.pinv(d["H"][c].astype(np.complex128)) @
                                  ((2 * (d["u_sym"][p].astype(int) // (1 << mb // 2)) - ((1 << mb // 2) - 1)) +
                                   1j * (2 * (d["u_sym"][p].astype(int) % (1 << mb // 2)) - ((1 << mb // 2) - 1))))
                   ** 2 for p, c in enumerate(d["chan_index"])])
    assert out["power"].cpu().numpy().sum() <= zf.sum()


# -------------------------------------------------------------- edge cases
def test_empty_and_invalid_arguments(mm):
    pkg, ctx = mm
    prm = pkg.Params.default()
    w = synth.uplink(1, 4, 4, 2, n_sub=0, n_sym=1)
    H = torch.zeros((1, 4, 4), dtype=torch.complex64, device=DEV)
    out = ctx.detect(H, T(w["y"].reshape(0, 4)), T(np.zeros(0, np.float32)), 2, prm, 1)
    assert out["sym"].shape == (0, 4)
    with pytest.raises(pkg.MMGaPError) as e:
        ctx.detect(H, torch.zeros((1, 4), dtype=torch.complex64, device=DEV),
                   torch.zeros(1, dtype=torch.float32, device=DEV), 2, pkg.Params.default(runs=48), 1)
    assert e.value.status == 5
    with pytest.raises(pkg.MMGaPError) as e:
        ctx.detect(H, torch.zeros((1, 4), dtype=torch.complex64, device=DEV),
                   torch.zeros(1, dtype=torch.float32, device=DEV), 3, prm, 1)
    assert e.value.status == 5
    with pytest.raises(pkg.MMGaPError) as e:
        ctx.detect(H, torch.zeros((1, 4), dtype=torch.complex64, device=DEV),
                   torch.zeros(1, dtype=torch.float32, device=DEV), 2, pkg.Params.default(dt=-1.0), 1)
    assert e.value.status == 1
    with pytest.raises(pkg.MMGaPError) as e:
        Hb = torch.zeros((1, 4, 5), dtype=torch.complex64, device=DEV)
        ctx.detect(Hb, torch.zeros((1, 4), dtype=torch.complex64, device=DEV),
                   torch.zeros(1, dtype=torch.float32, device=DEV), 2, prm, 1)
    assert e.value.status == 5


def test_bad_channel_index_is_flagged(mm):
    pkg, ctx = mm
    ctx.device_errors(clear=True)
    w = synth.uplink(4, 4, 4, 2, n_sub=3, n_sym=1)
    ci = np.array([0, 7, 1], np.int32)
    out = ctx.detect(T(w["H"]), T(w["y"]), T(w["noise_var"]), 2, pkg.Params.default(steps=10), 1,
                     chan_index=T(ci))
    torch.cuda.synchronize()
    assert ctx.device_errors(clear=True) & 1
    assert ctx.device_errors(clear=True) == 0
    assert out["sym"].shape == (3, 4)


# ---------------------------------------------------------- solver shapes
@pytest.mark.parametrize("nt", [4, 8, 16])
@pytest.mark.parametrize("variant", [1, 2, 3, 4, 6, 9, 10])
@pytest.mark.parametrize("f_mvm,steps,runs", [(2, 200, 32), (1, 41, 64), (2, 77, 96), (2, 60, 128)])
def test_solver_shapes_bit_exact(mm, nt, variant, f_mvm, steps, runs):
    """Every launch shape gives the oracle's bits (ragged step counts too); a
    shape not compiled for the size (4 or 8 threads per anneal with too few
    rows per thread) resolves to one that is."""
    pkg, ctx = mm
    w = synth.uplink(600 + nt, nt, nt, 4, n_sub=7, n_sym=1, snr_db=13.0, hold="problem")
    bs = [oracle.build_detect32(w["H"][p], w["y"][p], w["noise_var"][p], 4) for p in range(7)]
    Aq = np.stack([b["Aq"] for b in bs])
    hq = np.stack([b["hq"] for b in bs])
    g = np.stack([b["g"] for b in bs]).astype(np.int8)
    prm = pkg.Params.default(runs=runs, f_mvm=f_mvm, steps=steps)
    ctx.set_solver_variant(nt, variant)
    try:
        compiled = not ((variant == 9 and nt < 8) or (variant == 10 and nt < 16))
        want = variant if compiled else {(9, 4): 4, (10, 4): 4, (10, 8): 9}[(variant, nt)]
        assert ctx.solver_variant(nt, f_mvm) == want
        got = ctx.solve_ising(T(Aq), T(hq), prm, seed=4242, g=T(g), level_max=3)
        torch.cuda.synchronize()
    finally:
        ctx.set_solver_variant(nt, 0)
    ref = oracle.solve_batch(Aq, hq, g, 3, oparams(prm), 4242)
    assert np.array_equal(got["d"].cpu().numpy(), ref["d"])
    assert np.array_equal(got["E"].cpu().numpy(), ref["E"])
    assert np.array_equal(got["run"].cpu().numpy(), ref["run"])
    assert np.array_equal(got["ndiv"].cpu().numpy(), ref["n_div"])


def _cluster_sizes():
    """Call sizes at the edges of the latency shapes' clusters on this device:
    a cluster of 4 CTAs per problem up to n_sm / 4 problems, of 2 up to
    n_sm / 2, none above."""
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    return [1, n_sm // 4, n_sm // 4 + 1, n_sm // 2, n_sm // 2 + 1]


@pytest.mark.parametrize("nt,runs", [(16, 32), (16, 96), (8, 32), (8, 64)])
def test_latency_clusters_are_bit_identical(mm, nt, runs):
    """The latency shapes (8 threads per anneal for 16 users, 4 for 8) run a
    small call's problems as clusters of 4 or 2 CTAs; at every cluster size
    every output of every problem equals the throughput shape's, and sampled
    problems equal the oracle's."""
    pkg, ctx = mm
    prm = pkg.Params.default(runs=runs, steps=50)
    for P in _cluster_sizes():
        w = synth.uplink(690 + nt + P, nt, nt, 4, n_sub=P, n_sym=1, snr_db=14.0)
        ctx.set_solver_variant(nt, 10 if nt == 16 else 9)
        try:
            lat = _detect(ctx, w, prm, 5)
            ctx.set_solver_variant(nt, 6 if nt == 16 else 3)
            thr = _detect(ctx, w, prm, 5)
        finally:
            ctx.set_solver_variant(nt, 0)
        for k in ("sym", "energy", "offset", "ndiv", "guess"):
            assert np.array_equal(lat[k], thr[k]), (P, k)
        for p in sorted({0, P - 1}):
            c = int(w["chan_index"][p])
            bld = oracle.build_detect32(w["H"][c], w["y"][p], w["noise_var"][p], 4)
            r = oracle.cac_solve(bld["Aq"], bld["hq"], bld["g"], 3, oparams(prm), 5, p)
            assert lat["energy"][p] == r["E"] and lat["ndiv"][p] == r["n_div"], (P, p)


@pytest.mark.parametrize("nt,P", [(16, 5), (16, 200), (16, 400), (8, 5), (8, 200), (8, 400)])
def test_default_shape_by_call_size_is_bit_identical(mm, nt, P):
    """The default shape depends on the call's size (latency shapes when SMs
    would idle); every choice gives the bits of the throughput shape and,
    on sampled problems, the oracle's."""
    pkg, ctx = mm
    w = synth.uplink(650 + nt + P, nt, nt, 4, n_sub=P, n_sym=1, snr_db=14.0)
    prm = pkg.Params.default(steps=60)
    ctx.set_solver_variant(nt, 0)
    auto = _detect(ctx, w, prm, 21)
    ctx.set_solver_variant(nt, 6 if nt == 16 else 3)
    try:
        fixed = _detect(ctx, w, prm, 21)
    finally:
        ctx.set_solver_variant(nt, 0)
    assert np.array_equal(auto["sym"], fixed["sym"]) and np.array_equal(auto["energy"], fixed["energy"])
    for p in (0, P // 2, P - 1):
        c = int(w["chan_index"][p])
        bld = oracle.build_detect32(w["H"][c], w["y"][p], w["noise_var"][p], 4)
        r = oracle.cac_solve(bld["Aq"], bld["hq"], bld["g"], 3, oparams(prm), 21, p)
        assert np.array_equal(auto["sym"][p], oracle.decode_detect(nt, 4, bld["g"], r["d"])), p
        assert auto["energy"][p] == r["E"], p


def test_autotuner_picks_a_compiled_shape(mm):
    pkg, _ = mm
    with pkg.Context(0) as ctx:
        v, ms = ctx.autotune(pkg.Params.default(steps=40), 16, 2048)
        assert v in ms and all(t > 0 for t in ms.values()) and set(ms) == {1, 2, 3, 4, 6, 9, 10}
        assert ms[v] == min(ms.values())
        v4, ms4 = ctx.autotune(pkg.Params.default(steps=40), 3, 512)
        assert v4 == 1 and set(ms4) == {1}
        w = synth.uplink(9, 16, 16, 4, n_sub=4, n_sym=2)
        prm = pkg.Params.default(steps=50)
        got = _detect(ctx, w, prm, 3)
    ref = oracle.detect_batch(w["H"], w["y"], w["noise_var"], 4, oparams(prm), 3, w["chan_index"])
    assert np.array_equal(got["sym"], ref["sym"]) and np.array_equal(got["energy"], ref["E"])


# ------------------------------------------------------------- MMGaP-E
@pytest.mark.parametrize("n_r,nt,mb,stages,hold", [(8, 8, 6, 1, "problem"), (16, 16, 6, 2, "subcarrier"),
                                                   (4, 4, 2, 2, "prb"), (12, 8, 4, 3, "problem"),
                                                   (3, 3, 4, 1, "problem")])
def test_detect_e_bit_exact(mm, n_r, nt, mb, stages, hold):
    pkg, ctx = mm
    w = synth.uplink(700 + nt + stages, n_r, nt, mb, n_sub=9, n_sym=2, snr_db=20.0, hold=hold)
    prm = pkg.Params.default(steps=70)
    out = ctx.detect_e(T(w["H"]), T(w["y"]), T(w["noise_var"]), mb, prm, 31, stages=stages,
                       chan_index=T(w["chan_index"]), want_candidates=True)
    torch.cuda.synchronize()
    cands = out["candidates"].cpu().numpy()
    for p in range(w["y"].shape[0]):
        c = int(w["chan_index"][p])
        r = oracle.detect_e(w["H"][c], w["y"][p], w["noise_var"][p], mb, stages, oparams(prm), 31, p)
        assert np.array_equal(cands[:, p, :], r["candidates"].astype(np.int8)), p
        assert int(out["best"][p]) == r["best"]
        assert float(out["obj"][p]) == np.float32(r["obj"])
        assert np.array_equal(out["sym"][p].cpu().numpy(), r["sym"])


# ------------------------------------------------------- Appendix A study
def test_anneal_spins_bit_exact(mm):
    """Every anneal's final sign pattern and divergence flag equal the oracle's
    final states (random Appendix-style instances, a stable and a diverging dt)."""
    pkg, ctx = mm
    A, h = synth.random_ising(17, 6, 16)
    for dt, steps in ((0.02, 128), (0.3, 60)):
        prm = pkg.Params.default(dt=dt, steps=steps, f_mvm=2)
        got = ctx.anneal_spins(T(A), T(h), prm, seed=77)
        torch.cuda.synchronize()
        got = got.cpu().numpy().view(np.uint64)
        for p in range(6):
            r = oracle.cac_solve(A[p], h[p], None, 0, oparams(prm), 77, p, want_states=True)
            for run in range(prm.runs):
                x = r["x_final"][run]
                w0 = sum(1 << q for q in range(min(64, len(x))) if x[q] >= 0)
                w1 = sum(1 << (q - 64) for q in range(64, len(x)) if x[q] >= 0)
                if r["E_runs"][run] == 2 ** 31 - 1:
                    w1 |= 1 << 63
                assert int(got[p, run, 0]) == w0 and int(got[p, run, 1]) == w1, (dt, p, run)
