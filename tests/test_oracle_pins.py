"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test ties an oracle function to something other than itself: published
known-answer vectors, closed forms, textbook/library routines, identities
checked over every state of a tiny problem, or brute force.  The intent is
that a dropped term, a wrong sign, index or transposed operand anywhere in the
oracle fails at least one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle as o
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_problem(rng, n_r, n_t, mod_bits, noise_var):
    H = synth.channels(rng, 1, n_r, n_t)[0]
    x = synth.symbols_to_complex(rng.integers(0, 1 << mod_bits, n_t), mod_bits)
    y = H @ x + np.sqrt(noise_var / 2) * (rng.standard_normal(n_r) + 1j * rng.standard_normal(n_r))
    return H, y


# --------------------------------------------------------------------- Philox
def test_philox_known_answers():
    """Philox4x32-10 against the published known-answer vectors (Salmon et al.)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        out = o.philox4x32_10(v[0:4], v[4:6])
        assert [int(w) for w in out] == v[6:10]


def test_initial_amplitudes_uniform():
    """x0 = sigma0 * U[-1, 1): mean 0, variance sigma0^2/3 (closed form), range."""
    xs = np.float32(0.25 * 2.0 ** -23)
    vals = np.array([o.initial_x(5, p, r, k, xs) for p in range(4) for r in range(32) for k in range(33)])
    assert vals.min() >= -0.25 and vals.max() < 0.25
    assert abs(vals.mean()) < 0.02
    assert abs(vals.var() - 0.25 ** 2 / 3) < 0.004


# ------------------------------------------------------------- constellation
@pytest.mark.parametrize("mod_bits,kappa2", [(2, 1 / 2), (4, 1 / 10), (6, 1 / 42)])
def test_qam_unit_energy(mod_bits, kappa2):
    """kappa normalises the square QAM alphabet to E|x|^2 = 1 (Sec. 2.1)."""
    k = o.qam_kappa(mod_bits)
    assert math.isclose(k * k, kappa2, rel_tol=1e-15)
    sym = np.arange(1 << mod_bits)
    x = synth.symbols_to_complex(sym, mod_bits)
    assert math.isclose(np.mean(np.abs(x) ** 2), 1.0, rel_tol=1e-12)


def test_decode_roundtrip():
    """decode(g = transmitted lattice point, d = 0) recovers the symbol index."""
    rng = np.random.default_rng(3)
    for mod_bits in (2, 4, 6):
        side = 1 << (mod_bits // 2)
        sym = rng.integers(0, 1 << mod_bits, 8)
        g = np.concatenate([2 * (sym // side) - (side - 1), 2 * (sym % side) - (side - 1)]).astype(np.int32)
        assert np.array_equal(o.decode_detect(8, mod_bits, g, np.zeros(16, np.int8)), sym)
        # an offset d moves the lattice point by 2d
        d = np.zeros(16, np.int8)
        d[0] = 1 if g[0] < side - 1 else -1
        out = o.decode_detect(8, mod_bits, g, d)
        assert out[0] == sym[0] + d[0] * side and np.array_equal(out[1:], sym[1:])


# ------------------------------------------------------ delta-Ising mapping
@pytest.mark.parametrize("n_t,n_r,mod_bits", [(1, 1, 2), (1, 2, 4), (2, 2, 4), (2, 3, 6), (3, 3, 4), (3, 4, 2)])
def test_energy_identity_every_state(n_t, n_r, mod_bits):
    """||y - Hs(g + s_a(s1+s2))||^2 = -s^T J s + ||z||^2 + 2 tr G for every spin
    state (Eq. 9 with the Fig. 5 block structure), the objective computed
    directly from Eq. 2 with numpy."""
    rng = np.random.default_rng(100 + 10 * n_t + mod_bits)
    H, y = _rand_problem(rng, n_r, n_t, mod_bits, 0.2)
    b = o.build_detect64(H, y, 0.2, mod_bits)
    J = o.dense_J(b["G"], b["h"])
    n = 2 * n_t
    N = 2 * n + 1
    assert np.allclose(J, J.T) and np.all(np.diag(J) == 0)
    k = o.qam_kappa(mod_bits)
    const = b["znorm2"] + 2 * np.trace(b["G"])
    for bits in itertools.product([-1, 1], repeat=N):
        s = np.array(bits, np.int8)
        xl = b["g"] + s[2 * n] * (s[:n].astype(int) + s[n:2 * n])
        xc = xl[:n_t] + 1j * xl[n_t:]
        lhs = np.linalg.norm(y - k * H @ xc) ** 2
        rhs = o.ising_energy(J, s) + const
        assert abs(lhs - rhs) <= 1e-10 * max(1.0, lhs)


def test_mmse_matches_linear_solve():
    """x_mmse = (H^H H + rho I)^-1 H^H y (Eq. 3, rho = noise/signal power)."""
    rng = np.random.default_rng(5)
    for (n_r, n_t, mb, nv) in [(8, 8, 4, 0.05), (16, 16, 4, 0.02), (12, 8, 6, 0.01), (4, 4, 2, 0.3)]:
        H, y = _rand_problem(rng, n_r, n_t, mb, nv)
        b = o.build_detect64(H, y, nv, mb)
        ref = np.linalg.solve(H.conj().T @ H + nv * np.eye(n_t), H.conj().T @ y) / o.qam_kappa(mb)
        got = b["x_mmse"][:n_t] + 1j * b["x_mmse"][n_t:]
        assert np.allclose(got, ref, rtol=1e-10, atol=1e-10)


def test_guess_is_nearest_alphabet_point():
    """g is the alphabet point nearest to x_mmse per real dimension (ties upward)."""
    rng = np.random.default_rng(6)
    for mb in (2, 4, 6):
        L = (1 << (mb // 2)) - 1
        levels = np.arange(-L, L + 1, 2)
        for _ in range(20):
            H, y = _rand_problem(rng, 6, 6, mb, 1.0)
            b = o.build_detect64(H, y, 1.0, mb)
            for x, g in zip(b["x_mmse"], b["g"]):
                dist = np.abs(levels - x)
                best = levels[dist == dist.min()].max()
                assert g == best


@pytest.mark.parametrize("n_t,mod_bits", [(1, 4), (2, 2), (2, 4), (3, 2)])
def test_exhaustive_ml_matches_bruteforce(n_t, mod_bits):
    """Exhaustive ML of Eq. 2 against a numpy enumeration of Omega^{n_t}."""
    rng = np.random.default_rng(7 + n_t)
    H, y = _rand_problem(rng, n_t + 1, n_t, mod_bits, 0.5)
    best, x = o.ml_exhaustive(H, y, mod_bits)
    pts = synth.symbols_to_complex(np.arange(1 << mod_bits), mod_bits)
    ref = min(np.linalg.norm(y - H @ np.array(c)) ** 2 for c in itertools.product(pts, repeat=n_t))
    assert math.isclose(best, ref, rel_tol=1e-12)
    xc = x[:n_t] + 1j * x[n_t:]
    assert math.isclose(np.linalg.norm(y - o.qam_kappa(mod_bits) * H @ xc) ** 2, ref, rel_tol=1e-12)


@pytest.mark.parametrize("n_t", [1, 2, 3])
def test_qpsk_ising_ground_state_is_ml(n_t):
    """For QPSK the delta neighbourhood spans the alphabet, so the in-alphabet
    Ising ground state decodes to the exhaustive ML solution."""
    rng = np.random.default_rng(11 + n_t)
    for _ in range(5):
        H, y = _rand_problem(rng, n_t + 1, n_t, 2, 0.8)
        b = o.build_detect64(H, y, 0.8, 2)
        J = o.dense_J(b["G"], b["h"])
        _, s = o.ising_bruteforce(J, b["g"], 1)
        n = 2 * n_t
        xl = b["g"] + s[2 * n] * (s[:n].astype(int) + s[n:2 * n])
        ml, _ = o.ml_exhaustive(H, y, 2)
        assert math.isclose(o.ml_objective(H, y, xl.astype(np.int32), 2), ml, rel_tol=1e-12)


# ----------------------------------------------------- FP32 mirror vs truth
def _build_pair(rng, n_r, n_t, mb, nv):
    H, y = _rand_problem(rng, n_r, n_t, mb, nv)
    H32 = H.astype(np.complex64)
    y32 = y.astype(np.complex64)
    b32 = o.build_detect32(H32, y32, np.float32(nv), mb)
    b64 = o.build_detect64(H32.astype(np.complex128), y32.astype(np.complex128), float(np.float32(nv)), mb,
                           g_in=b32["g"])
    return H32, y32, b32, b64


@pytest.mark.parametrize("n_r,n_t,mb", [(8, 8, 4), (16, 16, 4), (16, 16, 6), (12, 8, 2), (4, 4, 6), (32, 32, 4),
                                        (48, 32, 2)])
def test_fp32_build_within_error_bound(n_r, n_t, mb):
    """FP32 Gram and field agree with FP64 within 1e-5 normwise:
    |dG_ij| <= 1e-5 sum_k |Hs_ki||Hs_kj| and |dh_i| <= 1e-5 sum_k |Hs_ki| (|z_k| + sum_j |Hs_kj g_j|)."""
    rng = np.random.default_rng(20 + n_t + mb)
    k = o.qam_kappa(mb)
    for _ in range(10):
        H32, y32, b32, b64 = _build_pair(rng, n_r, n_t, mb, 0.05)
        Hs = k * H32.astype(np.complex128)
        Hr = np.block([[Hs.real, -Hs.imag], [Hs.imag, Hs.real]])
        absG = np.abs(Hr).T @ np.abs(Hr)
        assert np.all(np.abs(b32["G32"] - b64["G"]) <= 1e-5 * absG)
        g = b32["g"]
        yr = np.concatenate([y32.real, y32.imag]).astype(np.float64)
        zbound = np.abs(yr) + np.abs(Hr) @ np.abs(g)
        assert np.all(np.abs(b32["h32"] - b64["h"]) <= 1e-5 * (np.abs(Hr).T @ zbound))


def test_fp32_quantised_codes_differ_only_near_midpoints():
    """Quantised codes of the FP32 build equal the FP64 ones except where the
    FP64 scaled value lies within the FP32 error bound of a rounding midpoint."""
    rng = np.random.default_rng(31)
    mismatches = 0
    for _ in range(40):
        H32, y32, b32, b64 = _build_pair(rng, 16, 16, 4, 0.03)
        se, Aq64, hq64 = o.quantise64(b64["G"], b64["h"])
        if se != b32["sigma_exp"]:
            mx = max(np.abs(b64["G"]).max(), np.abs(b64["h"]).max())
            assert abs(mx / 2.0 ** round(math.log2(mx)) - 1) < 1e-5
            continue
        s = 2.0 ** (14 - se)
        for got, ref, val in ((b32["Aq"], Aq64, -b64["G"] * s), (b32["hq"], hq64, b64["h"] * s)):
            bad = got.astype(np.int64) != ref
            mismatches += int(bad.sum())
            if bad.any():
                frac = np.abs(val[bad] - np.floor(val[bad]) - 0.5)
                assert np.all(frac <= 1e-5 * 2 ** 14 * 4), frac
                assert np.all(np.abs(got[bad].astype(np.int64) - ref[bad]) == 1)
    assert mismatches < 0.05 * 40 * (32 * 32 + 32)


# ---------------------------------------------------------------- dynamics
def test_coupling_field_matches_dense_J():
    """The half-size decomposition of Fig. 5 (one n x n MVM, two element-wise
    products, two scalings, one dot product) equals the dense (2n+1)^2 J x."""
    rng = np.random.default_rng(41)
    for n in (2, 8, 16, 32):
        A = rng.integers(-2 ** 14, 2 ** 14 + 1, (n, n))
        A = np.triu(A) + np.triu(A, 1).T
        Af = (A * 2.0 ** -14 * 0.01).astype(np.float32)
        hf = (rng.integers(-2 ** 14, 2 ** 14 + 1, n) * 2.0 ** -14 * 0.01).astype(np.float32)
        x = rng.uniform(-2, 2, 2 * n + 1).astype(np.float32)
        mu = o.coupling_field(Af, hf, x)
        J = o.dense_J(-Af.astype(np.float64), hf.astype(np.float64))
        ref = J @ x.astype(np.float64)
        bound = (n + 4) * 2.0 ** -24 * (np.abs(J) @ np.abs(x.astype(np.float64))) * 2
        assert np.all(np.abs(mu - ref) <= bound + 1e-30)


def test_euler_step_matches_eqs_10_11():
    """One step equals x + dt[(p-1)x - x^3 + eps e (Jx)] and e + dt[-zeta(x^2-a)e]
    evaluated directly in FP64 (Eqs. 10-11, forward Euler)."""
    rng = np.random.default_rng(43)
    prm = o.Params(dt=0.02, p=1.2, a=0.8, zeta=3.0, eps=0.7)
    c = o.cac_consts(prm)
    for _ in range(200):
        x = np.float32(rng.uniform(-2, 2))
        e = np.float32(rng.uniform(0.1, 5))
        jx = rng.uniform(-8, 8)
        mu = np.float32(np.float32(jx) * np.float32(c.ce))
        x1, e1 = o.euler_spin(x, e, mu, c)
        xd, ed = float(x), float(e)
        xr = xd + 0.02 * ((1.2 - 1) * xd - xd ** 3 + 0.7 * ed * float(np.float32(jx)))
        er = ed + 0.02 * (-3.0 * (xd ** 2 - 0.8) * ed)
        assert abs(x1 - xr) <= 1e-6 * (abs(xd) + abs(xd) ** 3 + 0.1 * ed * abs(jx) + 1e-3)
        assert abs(e1 - er) <= 1e-6 * ed * (1 + xd * xd)


@pytest.mark.parametrize("p", [0.5, 1.2, 2.0])
def test_decoupled_dynamics_closed_form(p):
    """With eps = 0 each amplitude follows dx/dt = (p-1)x - x^3 (Bernoulli; exact
    solution x^2 = c w0 e^{2ct} / (c + w0 (e^{2ct} - 1)), c = p-1) and
    ln e(T) = -zeta (int x^2 dt - a T) with int x^2 dt = ln((c + w0(e^{2cT}-1))/c) / 2.
    The Euler iterate must match to O(dt)."""
    n = 4
    prm = o.Params(steps=200, dt=0.02, p=p, a=1.0, zeta=0.5, eps=0.0)
    Af = np.zeros((n, n), np.float32)
    hf = np.zeros(n, np.float32)
    x0 = np.linspace(-0.4, 0.45, 2 * n + 1).astype(np.float32)
    x0[np.abs(x0) < 0.05] = 0.07
    x, e = o.anneal(Af, hf, prm, x0, np.ones(2 * n + 1, np.float32))
    T = prm.steps * prm.dt
    c = p - 1.0
    w0 = x0.astype(np.float64) ** 2
    w = c * w0 * np.exp(2 * c * T) / (c + w0 * (np.exp(2 * c * T) - 1))
    assert np.allclose(np.abs(x), np.sqrt(w), rtol=2e-2)
    assert np.all(np.sign(x) == np.sign(x0))
    intw = 0.5 * np.log((c + w0 * (np.exp(2 * c * T) - 1)) / c)
    assert np.allclose(np.log(e), -0.5 * (intw - 1.0 * T), rtol=3e-2, atol=3e-2)


@pytest.mark.parametrize("n,f,steps", [(4, 1, 40), (8, 2, 40), (16, 3, 41), (32, 2, 40), (32, 1, 60), (64, 2, 40),
                                         (64, 3, 31)])
def test_coupled_trajectory_matches_fp64_euler(n, f, steps):
    """Short coupled anneals: the oracle's FP32 amplitudes after S steps equal a
    forward-Euler integration of Eqs. 10-11 in FP64 written here from the
    paper's definitions -- J from the block structure of Eq. 9 / Fig. 5 (the
    two halves coupled by A, each half's self-coupling with a zero diagonal,
    the auxiliary spin coupled by b = h), the field J x frozen for f_mvm steps
    (Sec. 3.2.1), x and e updated together from the old values -- from the same
    Philox amplitudes, to 5e-4 relative.  The FP32 rounding the horizon
    accumulates stays below 4e-5; a kept diagonal, a flipped b, a field
    refreshed one step late or e updated from the new x each miss by > 0.08."""
    rng = np.random.default_rng(70 + n + f)
    A = rng.integers(-2 ** 14, 2 ** 14 + 1, (n, n))
    A = np.triu(A) + np.triu(A, 1).T
    h = rng.integers(-2 ** 14, 2 ** 14 + 1, n)
    prm = o.Params(runs=3, steps=steps, f_mvm=f)
    r = o.cac_solve(A.astype(np.int16), h.astype(np.int16), None, 0, prm, 11, 5, want_states=True)
    Ad, hd = A * 2.0 ** -14, h * 2.0 ** -14
    At = Ad - np.diag(np.diag(Ad))
    J = np.block([[At, Ad, hd[:, None]], [Ad, At, hd[:, None]], [hd[None, :], hd[None, :], np.zeros((1, 1))]])
    xs = o.cac_consts(prm).xs
    dt, p, a, zeta, eps = prm.dt, prm.p, prm.a, prm.zeta, prm.eps
    for run in range(3):
        x = np.array([float(o.initial_x(11, 5, run, k, xs)) for k in range(2 * n + 1)])
        e = np.ones(2 * n + 1)
        for t in range(steps):
            if t % f == 0:
                mu = J @ x
            x, e = x + dt * ((p - 1) * x - x ** 3 + eps * e * mu), e + dt * (-zeta * (x ** 2 - a) * e)
        got = r["x_final"][run].astype(np.float64)
        assert np.all(np.abs(got - x) <= 5e-4 * (np.abs(x) + 1e-3)), run


# ------------------------------------------------------ energy and selection
def test_integer_energy_matches_ml_objective():
    """E(d) = d^T G_q d - h_q^T d equals (||z - 2 Hs d||^2 - ||z||^2) 2^14 / (4 sigma)
    up to the code roundings (<= 1/2 each), the objective taken from Eq. 2."""
    rng = np.random.default_rng(51)
    for (n_t, mb) in [(2, 4), (4, 4), (8, 6), (8, 2), (32, 4)]:
        H, y = _rand_problem(rng, n_t, n_t, mb, 0.1)
        b = o.build_detect64(H, y, 0.1, mb)
        se, Aq, hq = o.quantise64(b["G"], b["h"])
        k = o.qam_kappa(mb)
        n = 2 * n_t
        for _ in range(30):
            d = rng.integers(-1, 2, n).astype(np.int8)
            E = o.energy_q(Aq.astype(np.int16), hq.astype(np.int16), d)
            xl = b["g"] + 2 * d.astype(int)
            obj = np.linalg.norm(y - k * H @ (xl[:n_t] + 1j * xl[n_t:])) ** 2
            ref = (obj - b["znorm2"]) * 2.0 ** 14 / (4 * 2.0 ** se)
            bound = 0.5 * (np.abs(d).sum() ** 2 + np.abs(d).sum()) + 1e-6
            assert abs(E - ref) <= bound


def _final_e(b, prm, seed, problem, run):
    """Error variables of one anneal at its end, from the plain integrator."""
    c = o.cac_consts(prm)
    n = len(b["hq"])
    Af = (b["Aq"].astype(np.float32) * np.float32(2.0 ** -14)).astype(np.float32) * np.float32(c.ce)
    hf = (b["hq"].astype(np.float32) * np.float32(2.0 ** -14)).astype(np.float32) * np.float32(c.ce)
    x0 = np.array([o.initial_x(seed, problem, run, k, c.xs) for k in range(2 * n + 1)], np.float32)
    x, e = o.anneal(Af.astype(np.float32), hf.astype(np.float32), prm, x0, np.ones(2 * n + 1, np.float32))
    return e


def test_solver_counts_a_nonpositive_error_variable_as_diverged():
    """An anneal whose error variable ends <= 0 (finite amplitudes) is not a
    candidate: E_runs marks it, the divergence count includes it, and the
    selection falls back as for |x| > x_max.  p = 4 drives x^2 towards 3, where
    1 + dt zeta (a - x^2) < 0 (a = 0.01, zeta = 25) flips the sign of e every
    step while |e| decays."""
    rng = np.random.default_rng(62)
    prm = o.Params(runs=32, steps=61, p=4.0, a=0.01, zeta=25.0)
    seen = 0
    for _ in range(4):
        H32, y32, b32, _ = _build_pair(rng, 4, 4, 4, 0.05)
        r = o.cac_solve(b32["Aq"], b32["hq"], b32["g"], 3, prm, 5, 2, want_states=True)
        for run in range(prm.runs):
            e = _final_e(b32, prm, 5, 2, run)
            x = r["x_final"][run]
            assert np.all(np.isfinite(x)) and np.all(np.abs(x) <= prm.x_max)
            bad = not np.all(e > 0)
            seen += bad
            assert (r["E_runs"][run] == 2 ** 31 - 1) == bad
        assert r["n_div"] == sum(not np.all(_final_e(b32, prm, 5, 2, q) > 0) for q in range(prm.runs))
    assert seen > 0


def test_solver_selection_rules():
    """Spins -> offset (d = s_a(s1+s2)/2, clipped), MMSE fallback (E > 0 or
    diverged -> guess) and arg-min over (E, run) of Sec. 3.2."""
    rng = np.random.default_rng(61)
    prm = o.Params(runs=32, steps=60)
    for _ in range(6):
        H32, y32, b32, _ = _build_pair(rng, 8, 8, 4, 0.05)
        r = o.cac_solve(b32["Aq"], b32["hq"], b32["g"], 3, prm, 9, 4, want_states=True)
        n = 16
        cands = []
        for run in range(prm.runs):
            x = r["x_final"][run]
            s = np.where(x >= 0, 1, -1)
            d = s[2 * n] * (s[:n] + s[n:2 * n]) // 2
            xl = b32["g"] + 2 * d
            d[np.abs(xl) > 3] = 0
            valid = np.all(np.abs(x) <= prm.x_max) and np.all(_final_e(b32, prm, 9, 4, run) > 0)
            E = o.energy_q(b32["Aq"], b32["hq"], d.astype(np.int8)) if valid else None
            assert r["E_runs"][run] == (E if valid else 2 ** 31 - 1)
            cands.append((E, run, d) if (valid and E <= 0) else (0, run, np.zeros(n, int)))
        E, run, d = min(cands, key=lambda t: (t[0], t[1]))
        assert r["E"] == E and r["run"] == run and np.array_equal(r["d"], d)
        assert r["E"] <= 0


def test_cac_reaches_ml_on_small_qpsk():
    """Behaviour: on 4x4 QPSK at 10 dB the anneals recover the exhaustive-ML
    solution for nearly every problem (the delta neighbourhood covers QPSK)."""
    w = synth.uplink(71, 4, 4, 2, n_sub=40, n_sym=1, snr_db=10.0, hold="problem")
    r = o.detect_batch(w["H"], w["y"], w["noise_var"], 2, o.Params(runs=32, steps=200), 5, w["chan_index"])
    hits = 0
    for p in range(40):
        ml, _ = o.ml_exhaustive(w["H"][p].astype(np.complex128), w["y"][p].astype(np.complex128), 2)
        xh = synth.symbols_to_complex(r["sym"][p], 2)
        obj = np.linalg.norm(w["y"][p].astype(np.complex128) - w["H"][p].astype(np.complex128) @ xh) ** 2
        hits += obj <= ml * (1 + 1e-6) + 1e-9
    assert hits >= 38


def test_mmgap_improves_on_mmse():
    """Behaviour (Sec. 5.2): the solver's result never has a worse ML objective
    than the MMSE guess beyond quantisation, and lowers the BER at 15 dB."""
    w = synth.uplink(72, 8, 8, 4, n_sub=48, n_sym=1, snr_db=15.0, hold="problem")
    r = o.detect_batch(w["H"], w["y"], w["noise_var"], 4, o.Params(), 5, w["chan_index"])
    mm = np.zeros_like(w["sym"])
    for p in range(48):
        b = o.build_detect32(w["H"][p], w["y"][p], w["noise_var"][p], 4)
        mm[p] = o.decode_detect(8, 4, b["g"], np.zeros(16, np.int8))
        obj = lambda s: np.linalg.norm(w["y"][p] - w["H"][p] @ synth.symbols_to_complex(s, 4)) ** 2
        assert obj(r["sym"][p]) <= obj(mm[p]) * (1 + 1e-3) + 1e-3
    assert synth.bit_errors(r["sym"], w["sym"], 4) < synth.bit_errors(mm, w["sym"], 4)


def test_appendix_no_divergence_at_small_dt():
    """Appendix A: with dt <= 0.02 the integration essentially never diverges
    (P_diverge ~ 0) on random Ising instances."""
    A, h = synth.random_ising(81, 24, 8)
    for dt, steps in ((0.01, 400), (0.02, 200)):
        prm = o.Params(runs=8, steps=steps, dt=dt)
        div = sum(o.cac_solve(A[i], h[i], None, 0, prm, 3, i)["n_div"] for i in range(24))
        assert div / (24 * 8) < 0.01


# ---------------------------------------------------------------------- VPP
def test_vpp_inverse_matches_linalg():
    """Q = (H H^H)^-1 (Eq. 5) against numpy's inverse and its residual."""
    rng = np.random.default_rng(91)
    for (n_u, n_t) in [(2, 2), (8, 8), (16, 16), (4, 8)]:
        H = synth.channels(rng, 1, n_u, n_t)[0].astype(np.complex64).astype(np.complex128)
        Q = o.vpp_inverse64(H)
        K = H @ H.conj().T
        assert np.allclose(Q, np.linalg.inv(K), rtol=1e-9, atol=1e-9 * np.abs(Q).max())
        assert np.abs(K @ Q - np.eye(n_u)).max() < 1e-9 * np.linalg.cond(K)
        assert np.array_equal(Q, Q.conj().T)


def test_vpp_mapping_energy_and_output():
    """Sec. 3.3: E(d) tracks ||W(u + tau d)||^2 - ||W u||^2 (W = H^H (H H^H)^-1,
    Eq. 5); the precoder output is W(u + tau v) with power ||.||^2."""
    rng = np.random.default_rng(92)
    for (n_u, mb) in [(2, 4), (4, 2), (8, 4)]:
        H = synth.channels(rng, 1, n_u, n_u)[0].astype(np.complex64).astype(np.complex128)
        u = rng.integers(0, 1 << mb, n_u).astype(np.uint8)
        b = o.build_precode(H, u, mb)
        W = H.conj().T @ np.linalg.inv(H @ H.conj().T)
        side = 1 << (mb // 2)
        ui = u.astype(np.int64)
        ul = (2 * (ui // side) - (side - 1)) + 1j * (2 * (ui % side) - (side - 1))
        tau = o.vpp_tau(mb)
        assert tau == 2 * side
        base = np.linalg.norm(W @ ul) ** 2
        for _ in range(20):
            d = rng.integers(-1, 2, 2 * n_u).astype(np.int8)
            v = d[:n_u] + 1j * d[n_u:]
            ref = (np.linalg.norm(W @ (ul + tau * v)) ** 2 - base) * 2.0 ** 14 / (4 * 2.0 ** b["sigma_exp"])
            E = o.energy_q(b["Aq"], b["hq"], d)
            assert abs(E - ref) <= 0.5 * (np.abs(d).sum() ** 2 + np.abs(d).sum()) + 1e-6
            vv, x, pw = o.precode_output(H, b["Q"], u, d, mb)
            assert np.array_equal(vv[:, 0], d[:n_u]) and np.array_equal(vv[:, 1], d[n_u:])
            xr = W @ (ul + tau * v)
            assert np.allclose(x, xr, rtol=1e-5, atol=1e-5 * np.abs(xr).max())
            assert math.isclose(pw, np.linalg.norm(xr) ** 2, rel_tol=1e-5)


def test_vpp_ground_state_is_best_perturbation():
    """Brute-force Ising ground state of the VPP problem equals the best
    v in {-1,0,1}^{2 n_u} of Eq. 8 (enumerated with numpy)."""
    rng = np.random.default_rng(93)
    for _ in range(4):
        H = synth.channels(rng, 1, 2, 2)[0].astype(np.complex64).astype(np.complex128)
        u = rng.integers(0, 16, 2).astype(np.uint8)
        b = o.build_precode(H, u, 4)
        J = o.dense_J(b["G"], b["h"])
        _, s = o.ising_bruteforce(J)
        n = 4
        d = s[2 * n] * (s[:n].astype(int) + s[n:2 * n]) // 2
        W = H.conj().T @ np.linalg.inv(H @ H.conj().T)
        ui = u.astype(np.int64)
        ul = (2 * (ui // 4) - 3) + 1j * (2 * (ui % 4) - 3)
        best = min(np.linalg.norm(W @ (ul + 8 * (np.array(c[:2]) + 1j * np.array(c[2:])))) ** 2
                   for c in itertools.product([-1, 0, 1], repeat=4))
        got = np.linalg.norm(W @ (ul + 8 * (d[:2] + 1j * d[2:]))) ** 2
        assert math.isclose(got, best, rel_tol=1e-9)


# ------------------------------------------------------------- MMGaP-E
def _slice(v, L):
    v = min(max(v, -L), L)
    return 2 * math.floor(v / 2) + 1


def test_sic_single_user_is_mmse():
    """With one user there is nothing to cancel: SIC = MMSE hard decision."""
    rng = np.random.default_rng(201)
    for mb in (2, 4, 6):
        H, y = _rand_problem(rng, 3, 1, mb, 0.3)
        H32, y32 = H.astype(np.complex64), y.astype(np.complex64)
        g, perm, st = o.sic_guess32(H32, y32, 0.3, mb)
        b = o.build_detect32(H32, y32, np.float32(0.3), mb)
        assert st == 0 and list(perm) == [0] and np.array_equal(g, b["g"])


def test_sic_is_successive_mmse_on_reduced_systems():
    """Sec. 3.2.2's MMSE-SIC guess: the user detected at each step is the slice of
    the MMSE estimate of the system with the users detected so far cancelled
    (explicit FP64 inverses here, a Cholesky back substitution in the oracle),
    in the oracle's order; the first factored user has the smallest B_ii."""
    rng = np.random.default_rng(202)
    checked = 0
    for _ in range(40):
        n_t, mb, nv = 6, 4, 0.05
        H, y = _rand_problem(rng, 6, n_t, mb, nv)
        H32, y32 = H.astype(np.complex64), y.astype(np.complex64)
        g, perm, st = o.sic_guess32(H32, y32, nv, mb)
        k = o.qam_kappa(mb)
        Hs = k * H32.astype(np.complex128)
        yy = y32.astype(np.complex128)
        rho = np.float32(nv) * k * k
        B = Hs.conj().T @ Hs + rho * np.eye(n_t)
        assert perm[0] == int(np.argmin(np.real(np.diag(B))))
        L = (1 << (mb // 2)) - 1
        remaining = list(range(n_t))
        resid = yy.copy()
        ok = True
        for pos in range(n_t - 1, -1, -1):
            u = int(perm[pos])
            Hr = Hs[:, remaining]
            est = np.linalg.solve(Hr.conj().T @ Hr + rho * np.eye(len(remaining)), Hr.conj().T @ resid)
            xu = est[remaining.index(u)]
            near = min(abs(xu.real - round(xu.real / 2) * 2), abs(xu.imag - round(xu.imag / 2) * 2))
            if near < 1e-3:  # too close to a decision boundary for an FP32 / FP64 comparison
                ok = False
                break
            dec = complex(_slice(xu.real, L), _slice(xu.imag, L))
            assert (g[u], g[n_t + u]) == (int(dec.real), int(dec.imag))
            resid = resid - Hs[:, u] * dec
            remaining.remove(u)
        checked += ok
    assert checked >= 30


def test_sic_recovers_noise_free_symbols():
    rng = np.random.default_rng(203)
    for _ in range(10):
        n_t, mb = 8, 4
        H = synth.channels(rng, 1, 8, n_t)[0].astype(np.complex64)
        sym = rng.integers(0, 16, n_t)
        y = (H.astype(np.complex128) @ synth.symbols_to_complex(sym, mb)).astype(np.complex64)
        g, _, _ = o.sic_guess32(H, y, 1e-6, mb)
        assert np.array_equal(o.decode_detect(n_t, mb, g, np.zeros(2 * n_t, np.int8)), sym)


def test_detect_e_candidates_and_selection():
    """MMGaP-E: candidates are [MMSE guess, SIC guess, stage solutions]; the
    output is the candidate with the smallest ML objective (Eq. 2, checked in
    FP64), and the FP32 objective matches FP64 to 1e-5."""
    w = synth.uplink(204, 8, 8, 6, n_sub=12, n_sym=1, snr_db=22.0, hold="problem")
    prm = o.Params(steps=80)
    for p in range(12):
        r = o.detect_e(w["H"][p], w["y"][p], w["noise_var"][p], 6, 2, prm, 9, p)
        X = r["candidates"]
        b = o.build_detect32(w["H"][p], w["y"][p], w["noise_var"][p], 6)
        gs, _, _ = o.sic_guess32(w["H"][p], w["y"][p], w["noise_var"][p], 6)
        assert np.array_equal(X[0], b["g"]) and np.array_equal(X[1], gs)
        H64, y64 = w["H"][p].astype(np.complex128), w["y"][p].astype(np.complex128)
        objs = [o.ml_objective(H64, y64, x, 6) for x in X]
        assert abs(r["obj"] - objs[r["best"]]) <= 1e-5 * max(1.0, objs[r["best"]])
        assert objs[r["best"]] <= min(objs) * (1 + 1e-5) + 1e-6
        assert np.array_equal(r["sym"], o.decode_detect(8, 6, X[r["best"]], np.zeros(16, np.int8)))
    assert o.stage_seed(9, 1, 0) == 9


def test_mmgap_e_improves_on_mmgap_at_64qam():
    """Behaviour (Sec. 5.2): at 64-QAM and high SNR the single MMSE guess limits
    MMGaP; MMGaP-E with the SIC guess does better."""
    w = synth.uplink(205, 8, 8, 6, n_sub=40, n_sym=1, snr_db=22.0, hold="problem")
    prm = o.Params()
    r0 = o.detect_batch(w["H"], w["y"], w["noise_var"], 6, prm, 5, w["chan_index"])
    se = np.array([o.detect_e(w["H"][p], w["y"][p], w["noise_var"][p], 6, 1, prm, 5, p)["sym"] for p in range(40)])
    assert synth.bit_errors(se, w["sym"], 6) < synth.bit_errors(r0["sym"], w["sym"], 6)
