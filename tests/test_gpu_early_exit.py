"""Early exit (mmgap_params.early_exit = K) on the GPU against the oracle.

The rule (a budget lever, not in the paper): a problem's anneals advance
together, and every K-th field refresh compares all spin signs of all anneals
with the previous check point; when none changed the anneals stop there.  The
CUDA path must reproduce the oracle's stopping step, offsets, energies,
winning anneal and divergence counts bit for bit, on every bit-identical
launch shape that supports it.
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


def _oracle_one(w, p, prm, seed):
    c = int(w["chan_index"][p])
    n_t, mb = w["n_t"], w["mod_bits"]
    b = oracle.build_detect32(w["H"][c], w["y"][p], w["noise_var"][p], mb)
    r = oracle.cac_solve(b["Aq"], b["hq"], b["g"], (1 << (mb // 2)) - 1, oparams(prm), seed, p)
    return dict(sym=oracle.decode_detect(n_t, mb, b["g"], r["d"]), E=r["E"], d=r["d"], ndiv=r["n_div"],
                steps=r["steps"])


# (n_t, n_r, runs, f_mvm, steps, K, launch shape): shapes 1 plain, 2 tpa1, 3 tpa1 packed, 4 tpa2,
# 6 paired refresh, 9 tpa4, 10 tpa8; f_mvm 3 and 5 run the plain kernel with a runtime period
CASES = [(1, 2, 32, 2, 200, 2, 0), (2, 3, 64, 2, 150, 3, 0), (3, 5, 32, 3, 101, 2, 0),
         (4, 4, 32, 2, 200, 3, 3), (4, 6, 32, 1, 120, 4, 4),
         (8, 8, 32, 2, 200, 4, 3), (8, 8, 32, 2, 200, 3, 9), (8, 10, 64, 1, 99, 5, 4), (8, 8, 32, 2, 200, 1, 2),
         (8, 8, 32, 3, 200, 2, 0), (8, 8, 96, 2, 200, 2, 1),
         (16, 16, 32, 2, 200, 4, 6), (16, 16, 32, 2, 200, 4, 10), (16, 16, 32, 2, 201, 3, 3),
         (16, 16, 96, 2, 160, 2, 4), (16, 16, 32, 1, 200, 4, 9), (16, 16, 32, 2, 200, 3, 1), (16, 16, 32, 5, 200, 2, 0)]


@pytest.mark.parametrize("nt,n_r,runs,f_mvm,steps,K,shape", CASES)
def test_detect_early_exit_bit_exact(mm, nt, n_r, runs, f_mvm, steps, K, shape):
    pkg, ctx = mm
    w = synth.uplink(500 + 7 * nt + K, n_r, nt, 4, n_sub=12, n_sym=3, snr_db=16.0)
    prm = pkg.Params.default(runs=runs, f_mvm=f_mvm, steps=steps, early_exit=K)
    if nt in (4, 8, 16):
        ctx.set_solver_variant(nt, shape)
    try:
        out = ctx.detect(T(w["H"]), T(w["y"]), T(w["noise_var"]), 4, prm, 31, chan_index=T(w["chan_index"]),
                         want_energy=True, want_offset=True, want_ndiv=True, want_steps=True)
        torch.cuda.synchronize()
    finally:
        if nt in (4, 8, 16):
            ctx.set_solver_variant(nt, 0)
    got = {k: v.cpu().numpy() for k, v in out.items()}
    P = w["y"].shape[0]
    stopped = 0
    for p in range(P):
        r = _oracle_one(w, p, prm, 31)
        assert got["steps"][p] == r["steps"], p
        assert np.array_equal(got["sym"][p], r["sym"]), p
        assert got["energy"][p] == r["E"] and got["ndiv"][p] == r["ndiv"], p
        assert np.array_equal(got["offset"][p], r["d"]), p
        stopped += r["steps"] < steps
    if steps >= 150 and K * f_mvm <= 8:
        assert stopped > 0  # the rule stopped some problems


def test_solve_ising_early_exit_bit_exact(mm):
    """Random Appendix-style instances (no clipping), including a step size
    that diverges; the winning anneal index is compared too."""
    pkg, ctx = mm
    A, h = synth.random_ising(17, 20, 16)
    for dt, K in ((0.02, 2), (0.02, 5), (0.3, 1)):
        prm = pkg.Params.default(dt=dt, steps=150, early_exit=K)
        got = ctx.solve_ising(T(A), T(h), prm, seed=5)
        torch.cuda.synchronize()
        ref = oracle.solve_batch(A, h, None, 0, oparams(prm), 5)
        for k, rk in (("d", "d"), ("E", "E"), ("run", "run"), ("ndiv", "n_div")):
            assert np.array_equal(got[k].cpu().numpy(), ref[rk]), (dt, K, k)


def test_precode_early_exit_bit_exact(mm):
    pkg, ctx = mm
    rng = np.random.default_rng(8)
    H = synth.channels(rng, 20, 8, 8).astype(np.complex64)
    u = rng.integers(0, 16, (20, 8)).astype(np.uint8)
    prm = pkg.Params.default(steps=160, early_exit=3)
    got = ctx.precode(T(H), T(u), 4, prm, 12, want_energy=True, want_ndiv=True)
    torch.cuda.synchronize()
    ref = oracle.precode_batch(H, u, 4, oparams(prm), 12)
    assert np.array_equal(got["v"].cpu().numpy(), ref["v"])
    assert np.array_equal(got["energy"].cpu().numpy(), ref["E"])
    assert np.array_equal(got["power"].cpu().numpy(), ref["power"])


def test_early_exit_sampled_full_slot_16x16(mm):
    """The full 100 MHz 16x16 16-QAM slot (45,864 problems) with early exit
    K = 4 in the benchmark's launch configuration (paired refresh); sampled
    problems checked one by one, properties checked on every problem."""
    pkg, _ = mm
    w = synth.uplink(2025, 16, 16, 4, snr_db=16.0)
    prm = pkg.Params.default(early_exit=4)
    with pkg.Context(0, workspace_bytes=512 << 20) as big:
        big.set_solver_variant(16, 6)
        out = big.detect(T(w["H"]), T(w["y"]), T(w["noise_var"]), 4, prm, 77, chan_index=T(w["chan_index"]),
                         want_energy=True, want_ndiv=True, want_steps=True)
        torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    P = w["y"].shape[0]
    idx = [0, 1, 13, P // 2, P - 1] + list(np.random.default_rng(6).integers(0, P, 11))
    for p in idx:
        r = _oracle_one(w, int(p), prm, 77)
        assert got["steps"][p] == r["steps"] and got["energy"][p] == r["E"], p
        assert np.array_equal(got["sym"][p], r["sym"]) and got["ndiv"][p] == r["ndiv"], p
    s = got["steps"]
    assert np.all((s == 200) | ((s % 8 == 0) & (s > 0) & (s < 200)))
    assert np.all(got["energy"] <= 0)
    assert 0.05 < np.mean(s < 200) < 1.0


@pytest.mark.parametrize("shape", [1, 3, 6])
def test_early_exit_without_a_check_point_is_the_plain_call(mm, shape):
    """steps = 0, or no check point before S: the outputs equal the call
    without early exit, and every problem reports all S steps."""
    pkg, ctx = mm
    w = synth.uplink(77, 16, 16, 4, n_sub=6, n_sym=3, snr_db=15.0)
    args = (T(w["H"]), T(w["y"]), T(w["noise_var"]), 4)
    kw = dict(chan_index=T(w["chan_index"]), want_energy=True, want_offset=True, want_ndiv=True, want_steps=True)
    ctx.set_solver_variant(16, shape)
    try:
        for steps, K in ((0, 2), (7, 4), (40, 20)):
            a = ctx.detect(*args, pkg.Params.default(steps=steps), 3, **kw)
            b = ctx.detect(*args, pkg.Params.default(steps=steps, early_exit=K), 3, **kw)
            torch.cuda.synchronize()
            for k in ("sym", "energy", "offset", "ndiv", "steps"):
                assert torch.equal(a[k], b[k]), (steps, K, k)
            assert bool((b["steps"] == steps).all())
    finally:
        ctx.set_solver_variant(16, 0)


def test_mmgap_e_early_exit_bit_exact(mm):
    """MMGaP-E's stages anneal with the same early-exit rule (both instances of
    every stage), bit-exact against the oracle's detect_e under it."""
    pkg, ctx = mm
    w = synth.uplink(88, 8, 8, 6, n_sub=6, n_sym=2, snr_db=22.0, hold="problem")
    prm = pkg.Params.default(steps=160, early_exit=3)
    out = ctx.detect_e(T(w["H"]), T(w["y"]), T(w["noise_var"]), 6, prm, 17, stages=2,
                       chan_index=T(w["chan_index"]), want_candidates=True)
    torch.cuda.synchronize()
    cands = out["candidates"].cpu().numpy()
    for p in range(w["y"].shape[0]):
        r = oracle.detect_e(w["H"][p], w["y"][p], w["noise_var"][p], 6, 2, oparams(prm), 17, p)
        assert np.array_equal(cands[:, p, :], r["candidates"].astype(np.int8)), p
        assert int(out["best"][p]) == r["best"] and np.array_equal(out["sym"][p].cpu().numpy(), r["sym"]), p


def test_early_exit_refusals(mm):
    """Shapes and calls without early exit refuse K > 0 before launching."""
    pkg, ctx = mm
    prm = pkg.Params.default(early_exit=2)
    w = synth.uplink(9, 16, 16, 4, n_sub=2, n_sym=2)
    args = (T(w["H"]), T(w["y"]), T(w["noise_var"]), 4, prm, 1)
    for shape in (5, 7, 8):
        ctx.set_solver_variant(16, shape)
        with pytest.raises(pkg.MMGaPError) as e:
            ctx.detect(*args, chan_index=T(w["chan_index"]))
        assert e.value.status == 5
    ctx.set_solver_variant(16, 0)
    with pytest.raises(pkg.MMGaPError) as e:  # direct mapping
        ctx.detect(*args, chan_index=T(w["chan_index"]), mapping=1)
    assert e.value.status == 5
    w32 = synth.uplink(10, 32, 32, 4, n_sub=1, n_sym=2)
    with pytest.raises(pkg.MMGaPError) as e:  # 32 users
        ctx.detect(T(w32["H"]), T(w32["y"]), T(w32["noise_var"]), 4, prm, 1, chan_index=T(w32["chan_index"]))
    assert e.value.status == 5
    A, h = synth.random_ising(3, 2, 8)
    with pytest.raises(pkg.MMGaPError) as e:
        ctx.anneal_spins(T(A), T(h), prm, 1)
    assert e.value.status == 5
    with pytest.raises(pkg.MMGaPError) as e:
        ctx.detect(*args[:4], pkg.Params.default(early_exit=-1), 1, chan_index=T(w["chan_index"]))
    assert e.value.status == 1


def test_batch_and_server_early_exit_equal_the_per_job_path(mm):
    """The batched launch and the server anneal with the same early-exit rule:
    every job's symbols, energies, divergence counts and steps equal the
    per-job call's, across 4-, 8- and 16-user jobs."""
    pkg, ctx = mm
    prm = pkg.Params.default(steps=160, early_exit=3)
    specs = [(16, 4, 20, "subcarrier"), (8, 2, 36, "prb"), (4, 6, 30, "problem"), (8, 4, 24, "subcarrier")]
    keep, jobs, outs, refs = [], [], [], []
    for i, (nt, mb, n_sub, hold) in enumerate(specs):
        w = synth.uplink(150 + i, nt, nt, mb, n_sub=n_sub, n_sym=4, snr_db=14.0, model="kron", hold=hold)
        t = [T(w[k]) for k in ("H", "y", "noise_var", "chan_index")]
        P = w["y"].shape[0]

        def outs_of():
            return {"sym": torch.full((P, nt), 255, dtype=torch.uint8, device=DEV),
                    "energy": torch.full((P,), 3, dtype=torch.int32, device=DEV),
                    "ndiv": torch.full((P,), -1, dtype=torch.int32, device=DEV),
                    "steps": torch.full((P,), -1, dtype=torch.int32, device=DEV)}
        r = outs_of()
        ctx.detect_jobs([ctx.detect_job(t[0], t[1], t[2], mb, 20 + i, r, t[3])], prm)
        o = outs_of()
        keep.append(t)
        outs.append(o)
        refs.append(r)
        jobs.append(ctx.detect_job(t[0], t[1], t[2], mb, 20 + i, o, t[3]))
    torch.cuda.synchronize()
    assert any(bool((r["steps"] < 160).any()) for r in refs)
    with pkg.Batch(0, prm, jobs, keepalive=(keep, outs)) as b:
        b.run(use_graph=True)
        torch.cuda.synchronize()
    for o, r in zip(outs, refs):
        for k in o:
            assert torch.equal(o[k], r[k]), k
    for o in outs:
        for v in o.values():
            v.fill_(-7)
    with pkg.Server(0, prm, scratch_bytes=32 << 20, n_lanes=2, max_jobs_per_group=2) as srv:
        for tk in [srv.submit(j) for j in jobs]:
            srv.wait(tk, timeout_us=60_000_000)
    for o, r in zip(outs, refs):
        for k in o:
            assert torch.equal(o[k], r[k]), k
    # refused: the tcgen05 tiles, and a 32-user job
    with pytest.raises(pkg.MMGaPError):
        pkg.Batch(0, prm, jobs[:1], tensor_core=True)
    with pytest.raises(pkg.MMGaPError):
        pkg.Server(0, prm, tensor_core=True)
    w32 = synth.uplink(160, 32, 32, 4, n_sub=1, n_sym=2)
    o32 = {"sym": torch.empty((2, 32), dtype=torch.uint8, device=DEV)}
    t32 = [T(w32[k]) for k in ("H", "y", "noise_var", "chan_index")]
    with pytest.raises(pkg.MMGaPError):
        pkg.Batch(0, prm, [ctx.detect_job(t32[0], t32[1], t32[2], 4, 1, o32, t32[3])])
