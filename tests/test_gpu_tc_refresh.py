"""Tensor-core field refresh (solver launch shapes 5, 7 and 8).

A precision variant of the CIM-CAC solver: the field m = A u of the 32
anneals of a warp is one mma.sync product with FP16-split operands and FP32
accumulation (shape 5; shape 7 with two threads per anneal), or the same
product for a CTA's 128 anneals as tcgen05 MMAs with the accumulator in
tensor memory (shape 8), so its results are not bit-identical to the FP32
path's.  What is required of it:
  * the selection stays exact: every reported energy is the integer energy of
    the reported offsets (checked with the oracle's energy);
  * over a few steps, where the FP32 path's rounding has not yet been
    amplified by the dynamics, it takes the same decisions;
  * over full anneals it detects at the same bit error rate as the FP32 path
    (within the binomial spread of the error counts) and better than MMSE;
  * it is never chosen by the autotuner and is refused for sizes it lacks.
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


@pytest.mark.parametrize("shape", [5, 7, 8])
@pytest.mark.parametrize("n_t,f,runs", [(8, 1, 32), (8, 2, 64), (16, 2, 32), (16, 1, 128), (16, 2, 64),
                                        (8, 2, 128)])
def test_short_anneals_agree_and_energies_are_exact(mm, shape, n_t, f, runs):
    """1,501 problems (a ragged last CTA for shape 8's 128 / runs problems per CTA)."""
    pkg, ctx = mm
    n = 2 * n_t
    Aq, hq = synth.random_ising(40 + n_t + f, 1501, n)
    prm = pkg.Params.default(steps=7, f_mvm=f, runs=runs)
    res = {}
    for v in (3, shape):
        ctx.set_solver_variant(n_t, v)
        res[v] = ctx.solve_ising(T(Aq), T(hq), prm, 9)
    ctx.set_solver_variant(n_t, 0)
    torch.cuda.synchronize()
    d3, d5 = res[3]["d"].cpu().numpy(), res[shape]["d"].cpu().numpy()
    same = np.all(d3 == d5, axis=1).mean()
    assert same >= 0.99, same
    E5 = res[shape]["E"].cpu().numpy()
    for p in list(range(0, 1501, 7)) + [1499, 1500]:
        assert E5[p] == oracle.energy_q(Aq[p], hq[p], d5[p]), p
    assert ctx.device_errors() == 0


@pytest.mark.parametrize("n_t,runs", [(8, 32), (16, 32), (16, 64)])
def test_tcgen05_shared_couplings(mm, n_t, runs):
    """Shape 8 on problems whose couplings repeat in runs of 6 (a channel serving
    consecutive problems; fields differ): tiles inside a run multiply by one C,
    tiles across runs by the stacked C's; both agree with the FP32 path over
    short anneals and report exact energies."""
    pkg, ctx = mm
    n = 2 * n_t
    Aq, hq = synth.random_ising(120 + n_t + runs, 1203, n)
    Aq = np.ascontiguousarray(Aq[(np.arange(1203) // 6) * 6])
    prm = pkg.Params.default(steps=7, runs=runs)
    res = {}
    for v in (3, 8):
        ctx.set_solver_variant(n_t, v)
        res[v] = ctx.solve_ising(T(Aq), T(hq), prm, 12)
    ctx.set_solver_variant(n_t, 0)
    torch.cuda.synchronize()
    d3, d8 = res[3]["d"].cpu().numpy(), res[8]["d"].cpu().numpy()
    assert np.all(d3 == d8, axis=1).mean() >= 0.99
    E8 = res[8]["E"].cpu().numpy()
    for p in list(range(0, 1203, 5)) + [1202]:
        assert E8[p] == oracle.energy_q(Aq[p], hq[p], d8[p]), p
    assert ctx.device_errors() == 0


@pytest.mark.parametrize("n_t", [8, 16])
def test_tcgen05_results_do_not_depend_on_tiling(mm, n_t):
    """Shape 8 groups 4 problems per CTA from each chunk's start; a workspace
    that forces chunks of a few problems regroups them (and changes which tiles
    share one coupling operand), yet every problem's bits stay the same: each
    product element depends only on its own row and column."""
    pkg, ctx = mm
    w = synth.uplink(300 + n_t, n_t, n_t, 4, n_sub=9, n_sym=14, snr_db=14.0)
    prm = pkg.Params.default(steps=60)
    outs = []
    for ws in (96 * 1024 if n_t == 16 else 24 * 1024, 0):
        with pkg.Context(0, workspace_bytes=ws) as c:
            c.set_solver_variant(n_t, 8)
            o = c.detect(T(w["H"]), T(w["y"]), T(w["noise_var"]), 4, prm, 5, chan_index=T(w["chan_index"]),
                         want_energy=True, want_offset=True, want_ndiv=True)
            torch.cuda.synchronize()
            assert c.device_errors() == 0
            outs.append({k: v.cpu().numpy() for k, v in o.items()})
    for k in outs[0]:
        assert np.array_equal(outs[0][k], outs[1][k]), k


@pytest.mark.parametrize("n_t", [8, 16])
def test_tcgen05_long_anneals_and_96_runs(mm, n_t):
    """Shape 8 over full 200-step anneals (every refresh through tensor memory):
    energies stay exact and no wait expires; 96 anneals (not a divisor of the
    128-row tile) run shape 5's kernel, bit for bit."""
    pkg, ctx = mm
    n = 2 * n_t
    Aq, hq = synth.random_ising(90 + n_t, 777, n)
    ctx.set_solver_variant(n_t, 8)
    r8 = ctx.solve_ising(T(Aq), T(hq), pkg.Params.default(), 4)
    r96 = ctx.solve_ising(T(Aq), T(hq), pkg.Params.default(runs=96), 4)
    ctx.set_solver_variant(n_t, 5)
    r5 = ctx.solve_ising(T(Aq), T(hq), pkg.Params.default(runs=96), 4)
    ctx.set_solver_variant(n_t, 0)
    torch.cuda.synchronize()
    assert ctx.device_errors() == 0
    d8, E8 = r8["d"].cpu().numpy(), r8["E"].cpu().numpy()
    for p in range(0, 777, 11):
        assert E8[p] == oracle.energy_q(Aq[p], hq[p], d8[p]), p
    assert (E8 <= 0).all()
    for key in r5:
        assert torch.equal(r96[key], r5[key]), key


@pytest.mark.parametrize("shape", [5, 7, 8])
@pytest.mark.parametrize("n_t,mb,snr,model,hold", [(16, 4, 16.0, "iid", "subcarrier"), (8, 4, 15.0, "kron", "prb")])
def test_detection_ber_equals_the_fp32_path(mm, shape, n_t, mb, snr, model, hold):
    """16x16 16-QAM i.i.d. and 8x8 16-QAM Kronecker, 32 anneals x 200 steps:
    the bit-error counts of the two refreshes differ by less than four
    standard deviations of a binomial count (and by less than 12 %)."""
    pkg, ctx = mm
    w = synth.uplink(77 + n_t, n_t, n_t, mb, n_sub=600, n_sym=14, snr_db=snr, model=model, hold=hold)
    P = w["y"].shape[0]
    prm = pkg.Params.default()
    H, y, nv, ci = (T(w[k]) for k in ("H", "y", "noise_var", "chan_index"))
    errs = {}
    for v in (3, shape):
        ctx.set_solver_variant(n_t, v)
        out = ctx.detect(H, y, nv, mb, prm, 5, chan_index=ci, want_guess=(v == 3))
        torch.cuda.synchronize()
        errs[v] = synth.bit_errors(out["sym"].cpu().numpy(), w["sym"], mb)
        if v == 3:
            g = out["guess"].cpu().numpy().astype(int)
            side = 1 << (mb // 2)
            mmse = ((g[:, :n_t] + side - 1) // 2) * side + (g[:, n_t:] + side - 1) // 2
            errs["mmse"] = synth.bit_errors(mmse, w["sym"], mb)
    ctx.set_solver_variant(n_t, 0)
    nbits = P * n_t * mb
    e3, e5 = errs[3], errs[shape]
    sd = np.sqrt(e3 * (1 - e3 / nbits))
    assert abs(e5 - e3) <= 4 * sd and abs(e5 - e3) <= 0.12 * e3, (e3, e5, sd)
    assert e5 < errs["mmse"]


def test_refused_where_not_built_and_never_autotuned(mm):
    pkg, ctx = mm
    for shape in (5, 7, 8):
        with pytest.raises(pkg.MMGaPError) as e:
            ctx.set_solver_variant(4, shape)
        assert e.value.status == 5
    v, ms = ctx.autotune(pkg.Params.default(steps=40), 16, 2048)
    assert v in (1, 2, 3, 4, 6, 9, 10) and 5 not in ms and 7 not in ms and 8 not in ms


@pytest.mark.parametrize("n_t,runs", [(16, 32), (8, 64)])
def test_tcgen05_wait_expiry_returns_guesses_and_flags_the_context(n_t, runs):
    """A device wait limit of 0 makes the shape-8 waits on the tensor-core
    product give up at once: every problem of an affected CTA returns its
    guess (energy 0, offsets 0, every anneal counted as diverged) and bit 1 of
    the device error word is set.  The CTA still drains its product before
    freeing tensor memory, so the next call on the same context, with the
    default limit, equals a call made before the expiry and leaves the word
    clear.  No GPU fault is involved: the limit is what runs out."""
    import paper_2510_01579_gb300 as pkg
    w = synth.uplink(130 + n_t, n_t, n_t, 4, n_sub=4, n_sym=3, snr_db=14.0)
    P = w["y"].shape[0]
    prm = pkg.Params.default(runs=runs, steps=60)
    args = (T(w["H"]), T(w["y"]), T(w["noise_var"]), 4, prm, 23)
    kw = dict(chan_index=T(w["chan_index"]), want_energy=True, want_guess=True, want_offset=True, want_ndiv=True)
    with pkg.Context(0) as ctx:
        ctx.set_solver_variant(n_t, 8)
        before = {k: v.cpu() for k, v in ctx.detect(*args, **kw).items()}
        assert ctx.device_errors() == 0
        ctx.set_device_wait(0)
        bad = {k: v.cpu() for k, v in ctx.detect(*args, **kw).items()}
        assert ctx.device_errors() == 2
        ctx.set_device_wait(200_000_000)
        after = {k: v.cpu() for k, v in ctx.detect(*args, **kw).items()}
        assert ctx.device_errors() == 0
    for k in before:
        assert torch.equal(after[k], before[k]), k
    # every problem of an affected CTA fell back to its guess
    hit = bad["ndiv"] == runs
    assert bool(hit.any())
    assert bool((bad["energy"][hit] == 0).all()) and bool((bad["offset"][hit] == 0).all())
    g = bad["guess"][hit].numpy().astype(int)
    side = 4
    mm_sym = ((g[:, :n_t] + 3) // 2) * side + (g[:, n_t:] + 3) // 2
    assert np.array_equal(bad["sym"][hit].numpy(), mm_sym)
    assert torch.equal(bad["guess"], before["guess"])
    assert P > 0
