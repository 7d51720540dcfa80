"""GPU parity over seeded random samples of configurations.

Each case draws the sizes and parameters at random, within what the C ABI
accepts: users, antennas, modulation, anneals, refresh period, step count,
early exit, integration step, solver launch shape, call size (which picks the
latency clusters for small calls), and how channels are held.  Every output
of every problem must equal the oracle's (FP32 mirror) bit for bit.  The same
for precoding, and for random groups of jobs through the batched launch
against the per-job path.  Each sample is fixed by its seed, so a failure
names a reproducible case.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)
N_CASES = 96


@pytest.fixture(scope="module")
def mm():
    import paper_2510_01579_gb300 as pkg
    ctx = pkg.Context(0)
    yield pkg, ctx
    ctx.close()


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def draw(i: int) -> dict:
    rng = np.random.default_rng(91000 + i)
    n_t = int(rng.choice([1, 2, 3, 4, 8, 16, 32], p=[0.05, 0.05, 0.05, 0.2, 0.25, 0.3, 0.1]))
    n_r = int(rng.integers(n_t, min(64, max(n_t + 8, 2 * n_t)) + 1))
    cfg = dict(
        n_t=n_t, n_r=n_r,
        mod_bits=int(rng.choice([2, 4, 6])),
        runs=int(rng.choice([32, 64, 96, 128])),
        f_mvm=int(rng.integers(1, 6)),
        steps=int(rng.integers(0, 161)),
        dt=float(rng.choice([0.01, 0.02, 0.04])),
        early_exit=int(rng.choice([0, 0, 2, 3, 4])) if n_t <= 16 else 0,
        # exact launch shapes: 0 default, 1 plain, 2-4, 6, 9, 10 (resolved where not compiled)
        shape=int(rng.choice([0, 0, 1, 2, 3, 4, 6, 9, 10])),
        n_sub=int(rng.choice([1, 3, 12, 30, 40, 77, 90])),
        n_sym=int(rng.choice([1, 2, 14])),
        hold=str(rng.choice(["problem", "subcarrier", "prb"])),
        model=str(rng.choice(["iid", "kron"])),
        snr_db=float(rng.uniform(0.0, 30.0)),
        seed=int(rng.integers(0, 2 ** 40)),
    )
    if n_t == 32:  # the 32-user path: fewer problems keep the oracle quick
        cfg.update(n_sub=int(rng.choice([1, 3, 5])), n_sym=1, runs=int(rng.choice([32, 64, 128])))
    # bound the oracle's work (problems x anneals x steps x n^2, about 4e9 per second of one core)
    def work(n_sub, n_sym):
        return n_sub * n_sym * cfg["runs"] * max(cfg["steps"], 1) * (2 * n_t) ** 2
    while work(cfg["n_sub"], cfg["n_sym"]) > 1.5e9:
        if cfg["n_sym"] > 1:
            cfg["n_sym"] = 1
        else:
            cfg["n_sub"] = max(1, cfg["n_sub"] // 2)
            if cfg["n_sub"] == 1:
                break
    return cfg


@pytest.mark.parametrize("i", range(N_CASES))
def test_random_detection_config_bit_exact(mm, i):
    pkg, ctx = mm
    c = draw(i)
    w = synth.uplink(c["seed"] % 100000, c["n_r"], c["n_t"], c["mod_bits"], n_sub=c["n_sub"], n_sym=c["n_sym"],
                     snr_db=c["snr_db"], model=c["model"], hold=c["hold"])
    prm = pkg.Params.default(runs=c["runs"], steps=c["steps"], f_mvm=c["f_mvm"], dt=c["dt"],
                             early_exit=c["early_exit"])
    tuned = c["n_t"] in (4, 8, 16)
    if tuned:
        ctx.set_solver_variant(c["n_t"], c["shape"])
    try:
        out = ctx.detect(T(w["H"]), T(w["y"]), T(w["noise_var"]), c["mod_bits"], prm, c["seed"],
                         chan_index=T(w["chan_index"]), want_energy=True, want_guess=True, want_offset=True,
                         want_ndiv=True, want_steps=True)
        torch.cuda.synchronize()
    finally:
        if tuned:
            ctx.set_solver_variant(c["n_t"], 0)
    got = {k: v.cpu().numpy() for k, v in out.items()}
    op = oracle.Params(runs=prm.runs, steps=prm.steps, f_mvm=prm.f_mvm, dt=prm.dt, p=prm.p, a=prm.a, zeta=prm.zeta,
                       eps=prm.eps, sigma0=prm.sigma0, x_max=prm.x_max, early_exit=prm.early_exit)
    ref = oracle.detect_batch(w["H"], w["y"], w["noise_var"], c["mod_bits"], op, c["seed"], w["chan_index"])
    assert np.array_equal(got["guess"].astype(np.int32), ref["g"]), c
    assert np.array_equal(got["offset"], ref["d"]), c
    assert np.array_equal(got["energy"], ref["E"]), c
    assert np.array_equal(got["ndiv"], ref["n_div"]), c
    assert np.array_equal(got["steps"], ref["steps"]), c
    assert np.array_equal(got["sym"], ref["sym"]), c


def oparams(prm):
    return oracle.Params(runs=prm.runs, steps=prm.steps, f_mvm=prm.f_mvm, dt=prm.dt, p=prm.p, a=prm.a,
                         zeta=prm.zeta, eps=prm.eps, sigma0=prm.sigma0, x_max=prm.x_max, early_exit=prm.early_exit)


@pytest.mark.parametrize("i", range(32))
def test_random_precoding_config_bit_exact(mm, i):
    """Downlink VPP with the FP64 channel inverse: perturbations, energies,
    divergence counts, transmit vectors and powers equal the oracle's."""
    pkg, ctx = mm
    rng = np.random.default_rng(92000 + i)
    n_u = int(rng.choice([1, 2, 3, 4, 8, 16]))
    n_t = int(rng.integers(n_u, min(64, n_u + 8) + 1))
    mb = int(rng.choice([2, 4, 6]))
    runs = int(rng.choice([32, 64, 96, 128]))
    steps = int(rng.integers(0, 141))
    f_mvm = int(rng.integers(1, 4))
    n_sub = int(rng.choice([1, 5, 17, 40]))
    n_sym = int(rng.choice([1, 3]))
    while n_sub * n_sym * runs * max(steps, 1) * (2 * n_u) ** 2 > 1.5e9 and n_sub > 1:
        n_sub //= 2
    shape = int(rng.choice([0, 1, 3, 6, 9, 10]))
    d = synth.downlink(int(rng.integers(0, 100000)), n_u, n_t, mb, n_sub=n_sub, n_sym=n_sym,
                       model=str(rng.choice(["iid", "kron"])))
    prm = pkg.Params.default(runs=runs, steps=steps, f_mvm=f_mvm)
    seed = int(rng.integers(0, 2 ** 31))
    tuned = n_u in (4, 8, 16)
    if tuned:
        ctx.set_solver_variant(n_u, shape)
    try:
        out = ctx.precode(T(d["H"]), T(d["u_sym"]), mb, prm, seed, chan_index=T(d["chan_index"]),
                          want_energy=True, want_ndiv=True)
        torch.cuda.synchronize()
    finally:
        if tuned:
            ctx.set_solver_variant(n_u, 0)
    ref = oracle.precode_batch(d["H"], d["u_sym"], mb, oparams(prm), seed, d["chan_index"])
    case = (n_u, n_t, mb, runs, steps, f_mvm, n_sub * n_sym, shape)
    assert np.array_equal(out["v"].cpu().numpy(), ref["v"]), case
    assert np.array_equal(out["energy"].cpu().numpy(), ref["E"]), case
    assert np.array_equal(out["ndiv"].cpu().numpy(), ref["n_div"]), case
    assert np.array_equal(out["x"].cpu().numpy(), ref["x"]), case
    assert np.array_equal(out["power"].cpu().numpy(), ref["power"]), case


def _outs(P, n_t):
    return {"sym": torch.full((P, n_t), 255, dtype=torch.uint8, device=DEV),
            "energy": torch.full((P,), 9, dtype=torch.int32, device=DEV),
            "guess": torch.zeros((P, 2 * n_t), dtype=torch.int8, device=DEV),
            "offset": torch.zeros((P, 2 * n_t), dtype=torch.int8, device=DEV),
            "ndiv": torch.full((P,), -1, dtype=torch.int32, device=DEV),
            "steps": torch.full((P,), -1, dtype=torch.int32, device=DEV)}


@pytest.mark.parametrize("i", range(16))
def test_random_job_groups_batched_equal_per_job(mm, i):
    """A random group of detection jobs (4 to 32 users, uneven sizes, channels
    held per problem, subcarrier or PRB) through the batched launch, replayed
    twice (graph or not), equals each job's own per-job call on every output."""
    pkg, ctx = mm
    rng = np.random.default_rng(93000 + i)
    n_jobs = int(rng.integers(1, 9))
    sizes = [int(rng.choice([4, 8, 16, 32], p=[0.3, 0.3, 0.3, 0.1])) for _ in range(n_jobs)]
    ee = 0 if 32 in sizes else int(rng.choice([0, 0, 3]))
    prm = pkg.Params.default(steps=int(rng.integers(1, 81)), f_mvm=int(rng.choice([1, 2])), early_exit=ee)
    keep, outs, refs, jobs = [], [], [], []
    for j, n_t in enumerate(sizes):
        n_r = n_t if n_t == 32 else int(rng.integers(n_t, n_t + 9))
        w = synth.uplink(int(rng.integers(0, 100000)), n_r, n_t, int(rng.choice([2, 4, 6])),
                         n_sub=int(rng.choice([1, 7, 24, 60])) if n_t < 32 else int(rng.choice([1, 3])),
                         n_sym=int(rng.choice([1, 2, 14])) if n_t < 32 else 1,
                         snr_db=float(rng.uniform(3, 28)), hold=str(rng.choice(["problem", "subcarrier", "prb"])))
        t = (T(w["H"]), T(w["y"]), T(w["noise_var"]), T(w["chan_index"]))
        P = w["y"].shape[0]
        seed = int(rng.integers(0, 2 ** 31))
        o, r = _outs(P, n_t), _outs(P, n_t)
        ctx.detect_jobs([ctx.detect_job(*t[:3], w["mod_bits"], seed, r, t[3])], prm)
        jobs.append(ctx.detect_job(*t[:3], w["mod_bits"], seed, o, t[3]))
        keep += list(t)
        outs.append(o)
        refs.append(r)
    graph = bool(rng.integers(0, 2))
    with pkg.Batch(0, prm, jobs, keepalive=(keep, outs)) as b:
        for _ in range(2):
            for o in outs:
                for v in o.values():
                    v.fill_(7)
            b.run(use_graph=graph)
            torch.cuda.synchronize()
            for j in range(n_jobs):
                for k in refs[j]:
                    assert torch.equal(outs[j][k], refs[j][k]), (sizes, j, k, graph, ee)


@pytest.mark.parametrize("i", range(16))
def test_random_detect_e_bit_exact(mm, i):
    """MMGaP-E (MMSE and MMSE-SIC guesses, 1-3 stages, early exit at times):
    every candidate, the chosen candidate, its objective and the symbols equal
    the oracle's."""
    pkg, ctx = mm
    rng = np.random.default_rng(94000 + i)
    n_t = int(rng.choice([1, 2, 3, 4, 8, 16]))
    n_r = int(rng.integers(n_t, n_t + 9))
    mb = int(rng.choice([2, 4, 6]))
    stages = int(rng.integers(1, 4))
    prm = pkg.Params.default(runs=int(rng.choice([32, 64])), steps=int(rng.integers(0, 101)),
                             f_mvm=int(rng.integers(1, 4)), early_exit=int(rng.choice([0, 0, 3])))
    w = synth.uplink(int(rng.integers(0, 100000)), n_r, n_t, mb, n_sub=int(rng.choice([1, 4, 9])),
                     n_sym=int(rng.choice([1, 3])), snr_db=float(rng.uniform(5, 28)),
                     hold=str(rng.choice(["problem", "subcarrier", "prb"])))
    seed = int(rng.integers(0, 2 ** 31))
    out = ctx.detect_e(T(w["H"]), T(w["y"]), T(w["noise_var"]), mb, prm, seed, stages=stages,
                       chan_index=T(w["chan_index"]), want_candidates=True)
    torch.cuda.synchronize()
    cands = out["candidates"].cpu().numpy()
    case = (n_t, n_r, mb, stages, prm.runs, prm.steps, prm.f_mvm, prm.early_exit)
    for p in range(w["y"].shape[0]):
        c = int(w["chan_index"][p])
        r = oracle.detect_e(w["H"][c], w["y"][p], w["noise_var"][p], mb, stages, oparams(prm), seed, p)
        assert np.array_equal(cands[:, p, :], r["candidates"].astype(np.int8)), (case, p)
        assert int(out["best"][p]) == r["best"], (case, p)
        assert float(out["obj"][p]) == np.float32(r["obj"]), (case, p)
        assert np.array_equal(out["sym"][p].cpu().numpy(), r["sym"]), (case, p)


@pytest.mark.parametrize("i", range(16))
def test_random_static_entry_equals_context_path(mm, i):
    """The allocation-free entry point gives the context path's bits on
    random jobs (1-32 users, early exit and caller guesses at times), twice in
    a row (its scratch keeps the previous call's contents)."""
    pkg, ctx = mm
    rng = np.random.default_rng(95000 + i)
    n_t = int(rng.choice([1, 3, 4, 8, 16, 32]))
    n_r = n_t if n_t == 32 else int(rng.integers(n_t, n_t + 9))
    mb = int(rng.choice([2, 4, 6]))
    prm = pkg.Params.default(runs=int(rng.choice([32, 64, 128])), steps=int(rng.integers(1, 121)),
                             f_mvm=int(rng.integers(1, 3)),
                             early_exit=0 if n_t == 32 else int(rng.choice([0, 0, 2])))
    w = synth.uplink(int(rng.integers(0, 100000)), n_r, n_t, mb,
                     n_sub=int(rng.choice([1, 6, 40])) if n_t < 32 else 2,
                     n_sym=int(rng.choice([1, 14])) if n_t < 32 else 1, snr_db=float(rng.uniform(5, 28)),
                     hold=str(rng.choice(["problem", "subcarrier", "prb"])))
    P = w["y"].shape[0]
    guess = None
    if rng.integers(0, 3) == 0:
        L = (1 << (mb // 2)) - 1
        guess = T((2 * rng.integers(0, L + 1, size=(P, 2 * n_t)) - L).astype(np.int8))
    t = (T(w["H"]), T(w["y"]), T(w["noise_var"]), T(w["chan_index"]))
    seed = int(rng.integers(0, 2 ** 31))
    ref, out = _outs(P, n_t), _outs(P, n_t)
    ctx.detect_jobs([ctx.detect_job(*t[:3], mb, seed, ref, t[3], guess=guess)], prm)
    job = ctx.detect_job(*t[:3], mb, seed, out, t[3], guess=guess)
    for _ in range(2):
        for v in out.values():
            v.fill_(5)
        ctx.detect_static(job, prm)
        torch.cuda.synchronize()
        for k in ref:
            if guess is not None and k == "guess":
                continue
            assert torch.equal(out[k], ref[k]), (n_t, n_r, mb, prm.runs, prm.steps, prm.early_exit, k)
