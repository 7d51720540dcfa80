"""Pins of the oracle's direct (binary-weighted) spin mapping.

The mapping writes each real dimension of a lattice symbol as x = sum_b 2^b s_b
over B = log2(M)/2 spins.  Its Ising form (J, c, constant) is pinned to the
ML objective it encodes (every spin state, FP64), to exhaustive ML (its ground
state), and its FP32 mirror to the FP64 truth; the general-coupling anneal is
pinned to the dense field and to brute-force ground states of small problems.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth


def _problem(seed, n_r, n_t, snr_db=None):
    rng = np.random.default_rng(seed)
    H = (rng.standard_normal((n_r, n_t)) + 1j * rng.standard_normal((n_r, n_t))) / np.sqrt(2)
    y = rng.standard_normal(n_r) + 1j * rng.standard_normal(n_r)
    return H, y


@pytest.mark.parametrize("n_t,mb,n_r", [(1, 2, 2), (2, 2, 3), (1, 4, 2), (2, 4, 2), (1, 6, 3), (2, 6, 3),
                                         (3, 2, 4)])
def test_energy_identity_over_every_spin_state(n_t, mb, n_r):
    """||y - kappa H T s||^2 = -s^T J s - 2 c^T s + const for all 2^N states."""
    H, y = _problem(n_t * 10 + mb, n_r, n_t)
    d = oracle.build_direct64(H, y, mb)
    N = len(d["c"])
    assert N == 2 * n_t * (mb // 2)
    assert np.all(np.diag(d["J"]) == 0) and np.array_equal(d["J"], d["J"].T)
    kap = oracle.qam_kappa(mb)
    for bits in itertools.product([-1, 1], repeat=N):
        s = np.array(bits, np.int8)
        x = oracle.direct_lattice(n_t, mb, s)
        lhs = np.linalg.norm(y - kap * H @ (x[:n_t] + 1j * x[n_t:])) ** 2
        rhs = -s @ d["J"] @ s - 2 * d["c"] @ s + d["const"]
        assert abs(lhs - rhs) <= 1e-12 * max(1.0, lhs)


@pytest.mark.parametrize("mb", [2, 4, 6])
def test_binary_weights_enumerate_the_alphabet(mb):
    """x = sum 2^b s_b is a bijection from {-1,1}^B onto {+-1, +-3, ..., +-(2^B - 1)}."""
    B = mb // 2
    L = (1 << B) - 1
    seen = set()
    for bits in itertools.product([-1, 1], repeat=B):
        s = np.array(bits * 2, np.int8)  # one user: re and im dimensions
        x = oracle.direct_lattice(1, mb, s)
        assert x[0] == x[1] and -L <= x[0] <= L and x[0] % 2 != 0
        seen.add(int(x[0]))
        assert np.array_equal(oracle.direct_spins(1, mb, x), s)
    assert seen == set(range(-L, L + 1, 2))


@pytest.mark.parametrize("n_t,mb", [(2, 2), (2, 4), (1, 6), (3, 2)])
def test_ground_state_is_the_ml_solution(n_t, mb):
    H, y = _problem(77 + n_t + mb, 3, n_t)
    d = oracle.build_direct64(H, y, mb)
    N = len(d["c"])
    best, sbest = None, None
    for bits in itertools.product([-1, 1], repeat=N):
        s = np.array(bits, np.int8)
        e = -s @ d["J"] @ s - 2 * d["c"] @ s
        if best is None or e < best:
            best, sbest = e, s
    obj, xml = oracle.ml_exhaustive(H, y, mb)
    assert np.array_equal(oracle.direct_lattice(n_t, mb, sbest), xml)
    assert abs(best + d["const"] - obj) <= 1e-10 * max(1.0, obj)


@pytest.mark.parametrize("n_t,mb,n_r", [(4, 2, 4), (8, 4, 8), (16, 4, 16), (16, 6, 16), (4, 6, 8)])
def test_fp32_mirror_against_fp64(n_t, mb, n_r):
    w = synth.uplink(300 + n_t + mb, n_r, n_t, mb, n_sub=4, n_sym=1, snr_db=12.0)
    for p in range(4):
        H, y = w["H"][w["chan_index"][p]], w["y"][p]
        f32 = oracle.build_direct32(H, y, w["noise_var"][p], mb)
        f64 = oracle.build_direct64(H.astype(np.complex128), y.astype(np.complex128), mb)
        N = len(f64["c"])
        B = mb // 2
        # normwise: |dJ_ij| <= 1e-5 2^(b_i + b_j) sum_k |Hs_ki| |Hs_kj| (real form)
        kap = oracle.qam_kappa(mb)
        Hr = np.block([[H.real, -H.imag], [H.imag, H.real]]).astype(np.float64) * kap
        absG = np.abs(Hr).T @ np.abs(Hr)
        w2 = 2.0 ** (np.arange(N) % B)
        scale = np.outer(w2, w2) * absG[np.ix_(np.arange(N) // B, np.arange(N) // B)]
        assert np.all(np.abs(f32["J32"] - f64["J"]) <= 1e-5 * scale + 1e-30)
        yr = np.concatenate([y.real, y.imag]).astype(np.float64)
        cscale = w2 * (np.abs(Hr).T @ np.abs(yr))[np.arange(N) // B]
        assert np.all(np.abs(f32["c32"] - f64["c"]) <= 1e-5 * cscale)
        # codes: exact Q14 of the FP32 values, zero diagonal, symmetric
        s = 2.0 ** (14 - f32["sigma_exp"])
        assert np.array_equal(f32["Jq"], np.rint(f32["J32"].astype(np.float64) * s).astype(np.int16))
        assert np.all(np.diag(f32["Jq"]) == 0) and np.array_equal(f32["Jq"], f32["Jq"].T)
        assert np.abs(f32["Jq"]).max() <= 1 << 14 and np.abs(f32["cq"]).max() <= 1 << 14
        # the guess is the delta build's MMSE guess
        assert np.array_equal(f32["g"], oracle.build_detect32(H, y, w["noise_var"][p], mb)["g"])


def test_general_field_is_the_dense_product():
    rng = np.random.default_rng(5)
    for N in (8, 24, 64, 96):
        J = rng.uniform(-1, 1, (N, N)).astype(np.float32)
        J = np.triu(J, 1) + np.triu(J, 1).T
        c = rng.uniform(-1, 1, N).astype(np.float32)
        x = rng.uniform(-2, 2, N + 1).astype(np.float32)
        mu = oracle.general_field(J, c, x).astype(np.float64)
        Jd, cd, xd = J.astype(np.float64), c.astype(np.float64), x.astype(np.float64)
        ref = np.concatenate([Jd @ xd[:N] + cd * xd[N], [cd @ xd[:N]]])
        bound = (N + 1) * 2.0 ** -23 * np.concatenate([np.abs(Jd) @ np.abs(xd[:N]) + np.abs(cd * xd[N]),
                                                       [np.abs(cd) @ np.abs(xd[:N])]])
        assert np.all(np.abs(mu - ref) <= bound)


@pytest.mark.parametrize("N,f,steps", [(8, 1, 40), (16, 2, 40), (24, 3, 40), (64, 2, 40), (96, 1, 30)])
def test_general_trajectory_matches_fp64_euler(N, f, steps):
    """Short anneals of the general solver equal a forward-Euler integration of
    Eqs. 10-11 in FP64 written here: the N + 1 amplitudes coupled by
    [[J, c], [c^T, 0]] (J = J_q 2^-14 with zero diagonal, the field c reaching
    the spins through the auxiliary spin), the field frozen for f_mvm steps,
    from the same Philox amplitudes, to 5e-3 relative.  The FP32 rounding the
    horizon accumulates stays below 8e-4 (96 spins); a flipped c or a halved J
    miss by more than 5."""
    Jq, cq = synth.random_ising(800 + N, 1, N)
    Jq, cq = Jq[0].copy(), cq[0]
    np.fill_diagonal(Jq, 0)
    prm = oracle.Params(runs=3, steps=steps, f_mvm=f)
    r = oracle.cac_solve_general(Jq, cq, None, prm, 9, 4, want_states=True)
    K = np.zeros((N + 1, N + 1))
    K[:N, :N] = Jq * 2.0 ** -14
    K[:N, N] = K[N, :N] = cq * 2.0 ** -14
    xs = oracle.cac_consts(prm).xs
    dt, p, a, zeta, eps = prm.dt, prm.p, prm.a, prm.zeta, prm.eps
    for run in range(3):
        x = np.array([float(oracle.initial_x(9, 4, run, k, xs)) for k in range(N + 1)])
        e = np.ones(N + 1)
        for t in range(steps):
            if t % f == 0:
                mu = K @ x
            x, e = x + dt * ((p - 1) * x - x ** 3 + eps * e * mu), e + dt * (-zeta * (x ** 2 - a) * e)
        got = r["x_final"][run].astype(np.float64)
        assert np.all(np.abs(got - x) <= 5e-3 * (np.abs(x) + 1e-3)), run


def test_general_anneal_finds_small_ground_states():
    """Random small problems (N = 6): 64 anneals reach the brute-force minimum
    of the exact quantised energy, and the reported energy is that of the
    reported spins."""
    prm = oracle.Params(runs=64, steps=200)
    hits = 0
    for seed in range(12):
        Jq, cq = synth.random_ising(seed, 1, 6)
        Jq, cq = Jq[0].copy(), cq[0]
        np.fill_diagonal(Jq, 0)
        r = oracle.cac_solve_general(Jq, cq, None, prm, 3, seed)
        assert r["E"] == oracle.energy_direct(Jq, cq, r["s"])
        emin = min(oracle.energy_direct(Jq, cq, np.array(b, np.int8)) for b in itertools.product([-1, 1], repeat=6))
        assert r["E"] >= emin
        hits += r["E"] == emin
    assert hits >= 11


def test_reference_candidate_wins_ties_and_diverged_anneals_are_skipped():
    Jq, cq = synth.random_ising(9, 1, 8)
    Jq, cq = Jq[0].copy(), cq[0]
    np.fill_diagonal(Jq, 0)
    ground = min((oracle.energy_direct(Jq, cq, np.array(b, np.int8)), b) for b in itertools.product([-1, 1], repeat=8))
    sref = np.array(ground[1], np.int8)
    r = oracle.cac_solve_general(Jq, cq, sref, oracle.Params(runs=32, steps=150), 1, 0, want_energies=True)
    assert r["run"] == -1 and r["E"] == ground[0] and np.array_equal(r["s"], sref)
    # a step size that diverges every anneal: the reference comes back
    bad = oracle.cac_solve_general(Jq, cq, sref, oracle.Params(runs=8, steps=60, dt=3.0), 1, 0, want_energies=True)
    assert bad["n_div"] == 8 and bad["run"] == -1 and np.all(bad["E_runs"] == np.iinfo(np.int32).max)


def test_direct_detection_matches_ml_at_high_snr():
    """8x8 QPSK (16 spins) at 20 dB: the direct-mapping detector returns the
    exhaustive ML symbols on every problem of the sample."""
    w = synth.uplink(11, 8, 8, 2, n_sub=16, n_sym=1, snr_db=20.0)
    prm = oracle.Params(runs=32, steps=200)
    for p in range(16):
        H, y = w["H"][w["chan_index"][p]], w["y"][p]
        r = oracle.detect_direct(H, y, w["noise_var"][p], 2, prm, 5, p)
        _, xml = oracle.ml_exhaustive(H.astype(np.complex128), y.astype(np.complex128), 2)
        side = 2
        ml_sym = ((xml[:8] + 1) // 2) * side + (xml[8:] + 1) // 2
        assert np.array_equal(r["sym"], ml_sym.astype(np.uint8)), p


@pytest.mark.parametrize("n_t,mb", [(2, 2), (2, 4), (1, 6), (3, 4)])
def test_integer_energy_tracks_the_ml_objective(n_t, mb):
    """E(s) = -s^T Jq s - 2 cq^T s equals (||y - kappa H T s||^2 - const) 2^(14 - e)
    up to the code roundings: |error| <= (N^2 - N) / 2 + N (each code off by <= 1/2)."""
    w = synth.uplink(60 + n_t + mb, 3, n_t, mb, n_sub=2, n_sym=1, snr_db=10.0)
    for p in range(2):
        H, y = w["H"][w["chan_index"][p]], w["y"][p]
        f32 = oracle.build_direct32(H, y, w["noise_var"][p], mb)
        f64 = oracle.build_direct64(H.astype(np.complex128), y.astype(np.complex128), mb)
        N = len(f32["cq"])
        kap = oracle.qam_kappa(mb)
        scale = 2.0 ** (14 - f32["sigma_exp"])
        rng = np.random.default_rng(p)
        for _ in range(64):
            s = np.where(rng.random(N) < 0.5, 1, -1).astype(np.int8)
            x = oracle.direct_lattice(n_t, mb, s)
            obj = np.linalg.norm(y.astype(np.complex128) - kap * H.astype(np.complex128) @ (x[:n_t] + 1j * x[n_t:])) ** 2
            e = oracle.energy_direct(f32["Jq"], f32["cq"], s)
            # FP32 J, c differ from FP64 by <= 1e-5 normwise; allow that on top of the roundings
            slack = (N * N - N) / 2 + N + 1e-4 * scale * (np.abs(f64["J"]).sum() + 2 * np.abs(f64["c"]).sum())
            assert abs(e - (obj - f64["const"]) * scale) <= slack
