"""VPP channel inverse Q = (H H^H)^-1 (Sec. 2.2, Eq. 5) on the GPU.

The FP64 kernel follows the oracle's operation order and must equal it bit for
bit.  The FP32 kernel with iterative refinement is a precision variant: per
channel, max|Q - Q_fp64| <= (2^-44 kappa + 2^-28) max|Q| up to a small
constant (kappa = cond(H H^H)), where 2^-44 kappa is the floor set by the
double-FP32 residual (about 16 2^-48 kappa for 16 users) and 2^-28 the
acceptance test on the last correction; channels that do not pass it are
recomputed by the FP64 kernel.  End to end, the perturbations it yields agree
with the FP64 path's except where a Q14 coupling code rounds the other way.
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


def _channels(seed, n_chan, n_u, n_t, model="iid"):
    return synth.downlink(seed, n_u, n_t, 4, n_sub=n_chan, n_sym=1, model=model)["H"]


@pytest.mark.parametrize("nu,nt", [(1, 1), (2, 3), (3, 3), (4, 4), (4, 8), (8, 8), (8, 16), (16, 16), (16, 64)])
def test_fp64_inverse_equals_oracle(mm, nu, nt):
    pkg, ctx = mm
    H = _channels(700 + nu + nt, 40, nu, nt)
    Q, st = ctx.vpp_inverse(T(H), 0)
    torch.cuda.synchronize()
    assert not st.any()
    Qg = Q.cpu().numpy()
    for c in range(H.shape[0]):
        assert np.array_equal(Qg[c], oracle.vpp_inverse64(H[c].astype(np.complex128))), c


@pytest.mark.parametrize("nu,nt,model", [(4, 4, "iid"), (8, 8, "iid"), (8, 8, "kron"), (16, 16, "iid"),
                                         (16, 16, "kron"), (16, 32, "iid"), (3, 5, "iid")])
def test_fp32_refined_inverse_within_bound(mm, nu, nt, model):
    pkg, ctx = mm
    H = _channels(800 + nu + nt, 600, nu, nt, model)
    Q, st = ctx.vpp_inverse(T(H), 1)
    torch.cuda.synchronize()
    assert not st.any()
    Qg = Q.cpu().numpy()
    worst = 0.0
    for c in range(H.shape[0]):
        Hc = H[c].astype(np.complex128)
        ref = oracle.vpp_inverse64(Hc)
        kappa = np.linalg.cond(Hc @ Hc.conj().T)
        err = np.abs(Qg[c] - ref).max() / np.abs(ref).max()
        bound = 2.0 ** -44 * kappa + 2.0 ** -28
        worst = max(worst, err / bound)
        assert err <= 2.0 * bound, (c, err, kappa)
        assert np.array_equal(Qg[c], Qg[c].conj().T)  # Hermitian by construction
    print(f"worst error / bound = {worst:.3g}")


def test_fp32_refined_inverse_falls_back_on_ill_conditioned_channels(mm):
    pkg, ctx = mm
    H = _channels(901, 24, 8, 8)
    rng = np.random.default_rng(5)
    for c in range(0, 24, 3):  # two users with nearly the same channel: cond(H H^H) ~ 1e10
        H[c, 1] = H[c, 0] + 1e-5 * (rng.standard_normal(8) + 1j * rng.standard_normal(8))
    H[23] = 0  # singular: not positive definite in either precision
    Q64, s64 = ctx.vpp_inverse(T(H), 0)
    Qir, sir = ctx.vpp_inverse(T(H), 1)
    torch.cuda.synchronize()
    assert s64.cpu().tolist() == sir.cpu().tolist() == [0] * 23 + [1]
    Q64, Qir = Q64.cpu().numpy(), Qir.cpu().numpy()
    assert not Qir[23].any() and not Q64[23].any()
    for c in range(0, 23, 3):  # recomputed by the FP64 kernel
        assert np.array_equal(Qir[c], Q64[c]), c
        assert np.array_equal(Qir[c], oracle.vpp_inverse64(H[c].astype(np.complex128))), c


def test_inverse_arguments(mm):
    pkg, ctx = mm
    H = T(_channels(3, 2, 4, 4))
    with pytest.raises(pkg.MMGaPError) as e:
        ctx.vpp_inverse(H, 2)
    assert e.value.status == 1
    Q, st = ctx.vpp_inverse(H[:0], 1)
    assert Q.shape == (0, 4, 4)
    with pytest.raises(pkg.MMGaPError) as e:
        ctx.vpp_inverse(T(np.zeros((2, 5, 5), np.complex64)), 0)
    assert e.value.status == 5


@pytest.mark.parametrize("nu,mb", [(8, 4), (16, 4)])
def test_precode_with_refined_inverse_matches_fp64_path(mm, nu, mb):
    """Config: n_u = n_t users and antennas, 16-QAM, one channel per subcarrier,
    two symbols each.  Identical Q14 couplings give identical anneals, so the
    perturbations agree except on the rare problems where a coupling code
    rounds differently; there the transmit power is still that of a valid
    VPP candidate."""
    pkg, ctx = mm
    d = synth.downlink(950 + nu, nu, nu, mb, n_sub=256, n_sym=2)
    prm = pkg.Params.default(steps=120)
    args = (T(d["H"]), T(d["u_sym"]), mb, prm, 21)
    ref = ctx.precode(*args, chan_index=T(d["chan_index"]), inv_precision=0)
    got = ctx.precode(*args, chan_index=T(d["chan_index"]), inv_precision=1)
    torch.cuda.synchronize()
    v_eq = (got["v"] == ref["v"]).all(dim=(1, 2)).cpu().numpy()
    pr, pg = ref["power"].cpu().numpy(), got["power"].cpu().numpy()
    assert v_eq.mean() >= 0.97, v_eq.mean()
    assert np.allclose(pg[v_eq], pr[v_eq], rtol=1e-5, atol=0)
    assert abs(pg.sum() / pr.sum() - 1.0) < 0.01


@pytest.mark.parametrize("inv_precision", [0, 1])
def test_precode_chunked_workspace_is_deterministic(mm, inv_precision):
    """A workspace that holds the channel inverses and a few problems per chunk gives the same bits as
    one chunk; the FP64 path also equals the oracle."""
    pkg, ctx = mm
    d = synth.downlink(31, 8, 8, 4, n_sub=10, n_sym=4)
    prm = pkg.Params.default(steps=60)
    outs = []
    for ws in (16 * 1024, 0):
        with pkg.Context(0, workspace_bytes=ws) as c:
            o = c.precode(T(d["H"]), T(d["u_sym"]), 4, prm, 3, chan_index=T(d["chan_index"]), want_energy=True,
                          want_ndiv=True, inv_precision=inv_precision)
            torch.cuda.synchronize()
            outs.append({k: v.cpu().numpy() for k, v in o.items()})
    for k in outs[0]:
        assert np.array_equal(outs[0][k], outs[1][k]), k
    if inv_precision == 0:
        fields = ("runs", "steps", "f_mvm", "dt", "p", "a", "zeta", "eps", "sigma0", "x_max")
        ref = oracle.precode_batch(d["H"], d["u_sym"], 4, oracle.Params(**{f: getattr(prm, f) for f in fields}), 3,
                                   d["chan_index"])
        assert np.array_equal(outs[0]["v"], ref["v"]) and np.array_equal(outs[0]["energy"], ref["E"])
