"""Pins of the oracle's early-exit rule (a budget lever of this implementation;
the paper anneals every run for a fixed N_I steps, Appendix A).

The rule: a problem's anneals advance together; every K-th refresh point
t = j K f_mvm (0 < t < S) compares the spin signs [x >= 0] of all anneals with
those at t - K f_mvm, and the anneals stop at the first such t where none
changed.  The pins check it against the plain per-anneal integrator
(orc_anneal, a separate code path): the stopped state is the plain anneal
truncated at t, the signs there equal those K f_mvm steps earlier, and at
every earlier check point some sign had changed.  With no check point before
S the rule is a no-op.
"""
import numpy as np
import pytest

import oracle as o
import synth


def _plain_states(A, h, prm, seed, problem, steps):
    """Every anneal's final amplitudes after `steps` plain Euler steps (K = 0)."""
    if steps == 0:
        xs = o.cac_consts(prm).xs
        N = 2 * len(h) + 1
        return np.array([[o.initial_x(seed, problem, r, k, xs) for k in range(N)] for r in range(prm.runs)])
    q = o.Params(**{**prm.__dict__, "steps": steps, "early_exit": 0})
    return o.cac_solve(A, h, None, 0, q, seed, problem, want_states=True)["x_final"]


@pytest.mark.parametrize("K,f", [(2, 2), (3, 2), (4, 1), (3, 3)])
def test_early_exit_stops_at_the_first_stable_check_point(K, f):
    A, h = synth.random_ising(5, 12, 8)
    prm = o.Params(runs=8, steps=200, f_mvm=f, early_exit=K)
    stopped = 0
    for i in range(12):
        r = o.cac_solve(A[i], h[i], None, 0, prm, 21, i, want_states=True)
        t = r["steps"]
        period = K * f
        assert t == prm.steps or (t % period == 0 and 0 < t < prm.steps)
        # the final state is the plain anneal truncated at t
        assert np.array_equal(r["x_final"], _plain_states(A[i], h[i], prm, 21, i, t))
        # every earlier check point saw a sign change; the stopping one saw none
        last = t if t < prm.steps else (prm.steps - 1) // period * period + period
        for c in range(period, last + 1, period):
            if c >= prm.steps:
                break
            now = _plain_states(A[i], h[i], prm, 21, i, c) >= 0
            before = _plain_states(A[i], h[i], prm, 21, i, c - period) >= 0
            if c < t:
                assert (now != before).any(), (i, c)
            else:
                assert (now == before).all(), (i, c)
        stopped += t < prm.steps
    assert stopped >= 6  # the rule is exercised on these instances


def test_early_exit_without_a_check_point_changes_nothing():
    """K f_mvm >= S: no check point before S, so the results are the plain
    solver's (offsets, energy, winning anneal, divergence count, states)."""
    A, h = synth.random_ising(6, 6, 16)
    for K, f, S in ((100, 2, 200), (41, 1, 41), (5, 9, 40)):
        base = o.Params(runs=8, steps=S, f_mvm=f)
        ee = o.Params(runs=8, steps=S, f_mvm=f, early_exit=K)
        for i in range(6):
            r0 = o.cac_solve(A[i], h[i], None, 0, base, 3, i, want_states=True)
            r1 = o.cac_solve(A[i], h[i], None, 0, ee, 3, i, want_states=True)
            assert r1["steps"] == S
            for k in ("d", "x_final", "E_runs"):
                assert np.array_equal(r0[k], r1[k])
            assert (r0["E"], r0["run"], r0["n_div"]) == (r1["E"], r1["run"], r1["n_div"])


def test_early_exit_selection_is_the_plain_selection_at_the_stop():
    """After a stop at t the selection (offsets, fallback, arg-min) is the plain
    solver's with S = t, on a detection problem with clipping."""
    w = synth.uplink(8, 8, 8, 4, n_sub=6, n_sym=1, snr_db=14.0, hold="problem")
    for p in range(6):
        b = o.build_detect32(w["H"][p], w["y"][p], w["noise_var"][p], 4)
        ee = o.Params(runs=32, steps=200, early_exit=3)
        r = o.cac_solve(b["Aq"], b["hq"], b["g"], 3, ee, 9, p)
        r0 = o.cac_solve(b["Aq"], b["hq"], b["g"], 3, o.Params(runs=32, steps=r["steps"]), 9, p)
        assert (r["E"], r["run"], r["n_div"]) == (r0["E"], r0["run"], r0["n_div"])
        assert np.array_equal(r["d"], r0["d"])


def test_early_exit_rejects_negative_k():
    A, h = synth.random_ising(7, 1, 4)
    with pytest.raises(ValueError):
        o.cac_solve(A[0], h[0], None, 0, o.Params(runs=4, steps=10, early_exit=-1), 1, 0)
