"""CPU oracle of the MMGaP hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (the CUDA library and its
binding) never imports it and shares no code with it.

numpy wrappers over ``oracle.c`` (plain single-threaded C):

* FP64 truth -- the plain definitions: system model and MMSE (Sec. 2.1,
  Eqs. 1-3), delta-Ising mapping (Sec. 2.3 Eq. 9, Sec. 3.2.1 / Fig. 5),
  exhaustive ML (Eq. 2), brute-force Ising ground state, downlink inverse
  (Sec. 2.2 Eq. 5) and VPP mapping (Sec. 3.3, Eqs. 12-13).
* FP32 mirror -- the same method in the GPU path's precision and operation
  order (build, CIM-CAC solve of Eqs. 10-11, selection, decode), so that
  integer results (guesses, quantised couplings, spins, symbols) can be
  compared bit for bit.

The CIM-CAC trajectory has no worked example in the paper.  It is pinned by
closed forms (eps = 0), the dense-J identity of the half-size field, and, over
short horizons, by an FP64 forward-Euler integration of Eqs. 10-11 written in
the tests; beyond those horizons the FP32 trajectory has no independent
reference (see tests/test_oracle_*).
"""
from __future__ import annotations

import ctypes as C
import dataclasses

import numpy as np

from . import build as _build

_lib = C.CDLL(_build.build())

_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_i16p = np.ctypeslib.ndpointer(np.int16, flags="C_CONTIGUOUS")
_i8p = np.ctypeslib.ndpointer(np.int8, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")


def _nullable(ptr_type):
    """ndpointer that also accepts None (passed as NULL)."""
    class _P(ptr_type):
        @classmethod
        def from_param(cls, obj):
            if obj is None:
                return None
            return ptr_type.from_param(obj)
    return _P


class CParams(C.Structure):
    _fields_ = [("runs", C.c_int), ("steps", C.c_int), ("f_mvm", C.c_int),
                ("dt", C.c_float), ("p", C.c_float), ("a", C.c_float),
                ("zeta", C.c_float), ("eps", C.c_float), ("sigma0", C.c_float),
                ("x_max", C.c_float), ("early_exit", C.c_int)]


class CConsts(C.Structure):
    _fields_ = [("c1", C.c_float), ("cdt", C.c_float), ("cz", C.c_float),
                ("c2", C.c_float), ("ce", C.c_float), ("xs", C.c_float)]


@dataclasses.dataclass
class Params:
    """CIM-CAC / anneal parameters (Eqs. 10-11, Sec. 3.2)."""
    runs: int = 32
    steps: int = 200
    f_mvm: int = 2
    dt: float = 0.02
    p: float = 1.2
    a: float = 1.0
    zeta: float = 3.0
    eps: float = 0.5
    sigma0: float = 0.1
    x_max: float = 1000.0
    early_exit: int = 0  # K > 0: stop at the first K-th refresh point with no sign change since the last

    def c(self) -> CParams:
        return CParams(self.runs, self.steps, self.f_mvm, self.dt, self.p, self.a,
                       self.zeta, self.eps, self.sigma0, self.x_max, self.early_exit)


_lib.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
_lib.orc_qam_kappa.restype = C.c_double
_lib.orc_qam_kappa.argtypes = [C.c_int]
_lib.orc_vpp_tau.argtypes = [C.c_int]
_lib.orc_build_detect64.argtypes = [C.c_int, C.c_int, C.c_int, _f64p, _f64p, C.c_double, _nullable(_i32p),
                                    _nullable(_f64p), _nullable(_i32p), _nullable(_f64p), _nullable(_f64p),
                                    _nullable(_f64p)]
_lib.orc_build_detect32.argtypes = [C.c_int, C.c_int, C.c_int, _f32p, _f32p, C.c_float, _nullable(_i32p),
                                    _nullable(_i32p), _nullable(_f32p), _nullable(_f32p),
                                    C.POINTER(C.c_int), _i16p, _i16p]
_lib.orc_quantise64.argtypes = [C.c_int, _f64p, _f64p, C.POINTER(C.c_int), _i32p, _i32p]
_lib.orc_dense_J.argtypes = [C.c_int, _f64p, _f64p, _f64p]
_lib.orc_ising_energy.restype = C.c_double
_lib.orc_ising_energy.argtypes = [C.c_int, _f64p, _i8p]
_lib.orc_ml_objective.restype = C.c_double
_lib.orc_ml_objective.argtypes = [C.c_int, C.c_int, C.c_int, _f64p, _f64p, _i32p]
_lib.orc_ml_exhaustive.restype = C.c_double
_lib.orc_ml_exhaustive.argtypes = [C.c_int, C.c_int, C.c_int, _f64p, _f64p, _i32p]
_lib.orc_ising_bruteforce.restype = C.c_double
_lib.orc_ising_bruteforce.argtypes = [C.c_int, _f64p, _nullable(_i32p), C.c_int, _i8p]
_lib.orc_energy_q.restype = C.c_int32
_lib.orc_energy_q.argtypes = [C.c_int, _i16p, _i16p, _i8p]
_lib.orc_cac_consts.argtypes = [C.POINTER(CParams), C.POINTER(CConsts)]
_lib.orc_initial_x.restype = C.c_float
_lib.orc_initial_x.argtypes = [C.c_uint64, C.c_uint64, C.c_int, C.c_int, C.c_float]
_lib.orc_coupling_field.argtypes = [C.c_int, _f32p, _f32p, _f32p, _f32p]
_lib.orc_euler_spin.argtypes = [C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_float, C.POINTER(CConsts)]
_lib.orc_anneal.argtypes = [C.c_int, _f32p, _f32p, C.POINTER(CParams), C.POINTER(CConsts), _f32p, _f32p]
_lib.orc_cac_solve.argtypes = [C.c_int, _i16p, _i16p, _nullable(_i32p), C.c_int, C.POINTER(CParams),
                               C.c_uint64, C.c_uint64, _i8p, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                               C.POINTER(C.c_int32), _nullable(_f32p), _nullable(_i32p)]
_lib.orc_cac_solve_steps.argtypes = _lib.orc_cac_solve.argtypes + [_nullable(_i32p)]
_lib.orc_decode_detect.argtypes = [C.c_int, C.c_int, _i32p, _i8p, _u8p]
_lib.orc_vpp_inverse64.argtypes = [C.c_int, C.c_int, _f64p, _f64p]
_lib.orc_build_precode.argtypes = [C.c_int, C.c_int, C.c_int, _f64p, _u8p, _nullable(_f64p), _nullable(_f64p),
                                   _nullable(_f64p), C.POINTER(C.c_int), _i16p, _i16p]
_lib.orc_precode_output.argtypes = [C.c_int, C.c_int, C.c_int, _f64p, _f64p, _u8p, _i8p, _i8p, _f32p,
                                    C.POINTER(C.c_float)]
_lib.orc_detect_batch.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _nullable(_i32p), _f32p, _f32p, _f32p,
                                  C.POINTER(CParams), C.c_uint64, _u8p, _i32p, _i32p, _i32p, _nullable(_i32p),
                                  _nullable(_i8p), _nullable(_i32p)]

_lib.orc_sic_guess32.argtypes = [C.c_int, C.c_int, C.c_int, _f32p, _f32p, C.c_float, _i32p, _nullable(_i32p)]
_lib.orc_ml_objective32.restype = C.c_float
_lib.orc_ml_objective32.argtypes = [C.c_int, C.c_int, C.c_int, _f32p, _f32p, _i32p]
_lib.orc_stage_seed.restype = C.c_uint64
_lib.orc_stage_seed.argtypes = [C.c_uint64, C.c_int, C.c_int]
_lib.orc_detect_e.argtypes = [C.c_int, C.c_int, C.c_int, _f32p, _f32p, C.c_float, C.c_int, C.POINTER(CParams),
                              C.c_uint64, C.c_uint64, _u8p, C.POINTER(C.c_int), C.POINTER(C.c_float),
                              _nullable(_i32p)]

QBITS = 14


def _c128(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128)).view(np.float64)


def _c64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex64)).view(np.float32)


# ---------------------------------------------------------------- primitives
def philox4x32_10(ctr, key) -> np.ndarray:
    out = np.zeros(4, np.uint32)
    _lib.orc_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def qam_side(mod_bits: int) -> int:
    return 1 << (mod_bits // 2)


def qam_kappa(mod_bits: int) -> float:
    return _lib.orc_qam_kappa(mod_bits)


def vpp_tau(mod_bits: int) -> int:
    return _lib.orc_vpp_tau(mod_bits)


# ------------------------------------------------------------- FP64 truth
def build_detect64(H, y, noise_var, mod_bits, g_in=None):
    """FP64 delta-Ising build of one problem.  H: (n_r, n_t) complex, y: (n_r,)."""
    H = np.asarray(H)
    n_r, n_t = H.shape
    n = 2 * n_t
    xm = np.zeros(n)
    g = np.zeros(n, np.int32)
    G = np.zeros(n * n)
    h = np.zeros(n)
    zn = np.zeros(1)
    gi = None if g_in is None else np.ascontiguousarray(g_in, np.int32)
    st = _lib.orc_build_detect64(n_r, n_t, mod_bits, _c128(H), _c128(y), float(noise_var), gi, xm, g, G, h, zn)
    return dict(status=st, x_mmse=xm, g=g, G=G.reshape(n, n), h=h, znorm2=float(zn[0]))


def quantise64(G, h):
    n = len(h)
    se = C.c_int()
    Aq = np.zeros(n * n, np.int32)
    hq = np.zeros(n, np.int32)
    _lib.orc_quantise64(n, np.ascontiguousarray(G, np.float64).ravel(), np.ascontiguousarray(h, np.float64),
                        C.byref(se), Aq, hq)
    return se.value, Aq.reshape(n, n), hq


def dense_J(G, h) -> np.ndarray:
    n = len(h)
    N = 2 * n + 1
    J = np.zeros(N * N)
    _lib.orc_dense_J(n, np.ascontiguousarray(G, np.float64).ravel(), np.ascontiguousarray(h, np.float64), J)
    return J.reshape(N, N)


def ising_energy(J, s) -> float:
    J = np.ascontiguousarray(J, np.float64)
    return _lib.orc_ising_energy(J.shape[0], J.ravel(), np.ascontiguousarray(s, np.int8))


def ml_objective(H, y, x, mod_bits) -> float:
    n_r, n_t = np.asarray(H).shape
    return _lib.orc_ml_objective(n_r, n_t, mod_bits, _c128(H), _c128(y), np.ascontiguousarray(x, np.int32))


def ml_exhaustive(H, y, mod_bits):
    n_r, n_t = np.asarray(H).shape
    x = np.zeros(2 * n_t, np.int32)
    best = _lib.orc_ml_exhaustive(n_r, n_t, mod_bits, _c128(H), _c128(y), x)
    return best, x


def ising_bruteforce(J, g=None, level_max=0):
    J = np.ascontiguousarray(J, np.float64)
    N = J.shape[0]
    n = (N - 1) // 2
    s = np.zeros(N, np.int8)
    gi = None if g is None else np.ascontiguousarray(g, np.int32)
    best = _lib.orc_ising_bruteforce(n, J.ravel(), gi, int(level_max), s)
    return best, s


def vpp_inverse64(H) -> np.ndarray:
    H = np.asarray(H)
    n_u, n_t = H.shape
    Q = np.zeros(2 * n_u * n_u)
    st = _lib.orc_vpp_inverse64(n_u, n_t, _c128(H), Q)
    if st:
        raise ArithmeticError("HH^H not positive definite")
    return Q.view(np.complex128).reshape(n_u, n_u)


# ------------------------------------------------------------ FP32 mirror
def build_detect32(H, y, noise_var, mod_bits, g_in=None):
    """FP32 build in the pinned order.  H: (n_r, n_t) complex64, y: (n_r,) complex64."""
    H = np.asarray(H)
    n_r, n_t = H.shape
    n = 2 * n_t
    g = np.zeros(n, np.int32)
    G = np.zeros(n * n, np.float32)
    h = np.zeros(n, np.float32)
    se = C.c_int()
    Aq = np.zeros(n * n, np.int16)
    hq = np.zeros(n, np.int16)
    gi = None if g_in is None else np.ascontiguousarray(g_in, np.int32)
    st = _lib.orc_build_detect32(n_r, n_t, mod_bits, _c64(H), _c64(y), np.float32(noise_var), gi, g, G, h,
                                 C.byref(se), Aq, hq)
    return dict(status=st, g=g, G32=G.reshape(n, n), h32=h, sigma_exp=se.value, Aq=Aq.reshape(n, n), hq=hq)


def energy_q(Aq, hq, d) -> int:
    Aq = np.ascontiguousarray(Aq, np.int16)
    return int(_lib.orc_energy_q(len(hq), Aq.ravel(), np.ascontiguousarray(hq, np.int16),
                                 np.ascontiguousarray(d, np.int8)))


def cac_consts(params: Params) -> CConsts:
    c = CConsts()
    cp = params.c()
    _lib.orc_cac_consts(C.byref(cp), C.byref(c))
    return c


def initial_x(seed, problem, run, k, xs) -> np.float32:
    return np.float32(_lib.orc_initial_x(seed, problem, run, k, xs))


def coupling_field(Af, hf, x) -> np.ndarray:
    n = len(hf)
    mu = np.zeros(2 * n + 1, np.float32)
    _lib.orc_coupling_field(n, np.ascontiguousarray(Af, np.float32).ravel(), np.ascontiguousarray(hf, np.float32),
                            np.ascontiguousarray(x, np.float32), mu)
    return mu


def euler_spin(x, eh, mu, consts: CConsts):
    xc, ec = C.c_float(x), C.c_float(eh)
    _lib.orc_euler_spin(C.byref(xc), C.byref(ec), float(mu), C.byref(consts))
    return np.float32(xc.value), np.float32(ec.value)


def anneal(Af, hf, params: Params, x0, eh0):
    n = len(hf)
    x = np.array(x0, np.float32)
    eh = np.array(eh0, np.float32)
    cp = params.c()
    cc = cac_consts(params)
    _lib.orc_anneal(n, np.ascontiguousarray(Af, np.float32).ravel(), np.ascontiguousarray(hf, np.float32),
                    C.byref(cp), C.byref(cc), x, eh)
    return x, eh


def cac_solve(Aq, hq, g, level_max, params: Params, seed, problem, want_states=False):
    n = len(hq)
    N = 2 * n + 1
    d = np.zeros(n, np.int8)
    E, run, nd = C.c_int32(), C.c_int32(), C.c_int32()
    xf = np.zeros(params.runs * N, np.float32) if want_states else None
    Er = np.zeros(params.runs, np.int32) if want_states else None
    gi = None if g is None else np.ascontiguousarray(g, np.int32)
    cp = params.c()
    taken = np.zeros(1, np.int32)
    st = _lib.orc_cac_solve_steps(n, np.ascontiguousarray(Aq, np.int16).ravel(), np.ascontiguousarray(hq, np.int16),
                                  gi, int(level_max), C.byref(cp), int(seed), int(problem), d, C.byref(E),
                                  C.byref(run), C.byref(nd), xf, Er, taken)
    if st:
        raise ValueError("invalid solver arguments")
    out = dict(d=d, E=E.value, run=run.value, n_div=nd.value, steps=int(taken[0]))
    if want_states:
        out["x_final"] = xf.reshape(params.runs, N)
        out["E_runs"] = Er
    return out


def decode_detect(n_t, mod_bits, g, d) -> np.ndarray:
    sym = np.zeros(n_t, np.uint8)
    _lib.orc_decode_detect(n_t, mod_bits, np.ascontiguousarray(g, np.int32), np.ascontiguousarray(d, np.int8), sym)
    return sym


def build_precode(H, u_sym, mod_bits):
    """FP64 VPP delta-Ising build (Sec. 3.3).  H: (n_u, n_t) complex (complex64 values)."""
    H = np.asarray(H)
    n_u, n_t = H.shape
    n = 2 * n_u
    Q = np.zeros(2 * n_u * n_u)
    G = np.zeros(n * n)
    h = np.zeros(n)
    se = C.c_int()
    Aq = np.zeros(n * n, np.int16)
    hq = np.zeros(n, np.int16)
    st = _lib.orc_build_precode(n_u, n_t, mod_bits, _c128(H), np.ascontiguousarray(u_sym, np.uint8), Q, G, h,
                                C.byref(se), Aq, hq)
    return dict(status=st, Q=Q.view(np.complex128).reshape(n_u, n_u), G=G.reshape(n, n), h=h,
                sigma_exp=se.value, Aq=Aq.reshape(n, n), hq=hq)


def precode_output(H, Q, u_sym, d, mod_bits):
    H = np.asarray(H)
    n_u, n_t = H.shape
    v = np.zeros(2 * n_u, np.int8)
    x = np.zeros(2 * n_t, np.float32)
    pw = C.c_float()
    _lib.orc_precode_output(n_u, n_t, mod_bits, _c128(H), _c128(Q), np.ascontiguousarray(u_sym, np.uint8),
                            np.ascontiguousarray(d, np.int8), v, x, C.byref(pw))
    return v.reshape(n_u, 2), x.view(np.complex64), float(pw.value)


# ------------------------------------------------------------ batch drivers
def detect_batch(H, y, noise_var, mod_bits, params: Params, seed, chan_index=None):
    """Full uplink pipeline (FP32 mirror) over P problems.

    H: (n_chan, n_r, n_t) complex64, y: (P, n_r) complex64, noise_var: (P,).
    """
    H = np.asarray(H, np.complex64)
    n_chan, n_r, n_t = H.shape
    y = np.asarray(y, np.complex64)
    P = y.shape[0]
    n = 2 * n_t
    sym = np.zeros(P * n_t, np.uint8)
    E = np.zeros(P, np.int32)
    run = np.zeros(P, np.int32)
    nd = np.zeros(P, np.int32)
    g = np.zeros(P * n, np.int32)
    d = np.zeros(P * n, np.int8)
    steps = np.zeros(P, np.int32)
    ci = None if chan_index is None else np.ascontiguousarray(chan_index, np.int32)
    cp = params.c()
    _lib.orc_detect_batch(n_r, n_t, mod_bits, P, ci, _c64(H), _c64(y),
                          np.ascontiguousarray(noise_var, np.float32), C.byref(cp), int(seed), sym, E, run, nd, g, d,
                          steps)
    return dict(sym=sym.reshape(P, n_t), E=E, run=run, n_div=nd, g=g.reshape(P, n), d=d.reshape(P, n), steps=steps)


def solve_batch(Aq, hq, g, level_max, params: Params, seed):
    """CAC solve over P problems: Aq (P, n, n) int16, hq (P, n) int16, g (P, n) or None."""
    Aq = np.asarray(Aq, np.int16)
    P, n, _ = Aq.shape
    d = np.zeros((P, n), np.int8)
    E = np.zeros(P, np.int32)
    run = np.zeros(P, np.int32)
    nd = np.zeros(P, np.int32)
    for p in range(P):
        r = cac_solve(Aq[p], hq[p], None if g is None else g[p], level_max, params, seed, p)
        d[p], E[p], run[p], nd[p] = r["d"], r["E"], r["run"], r["n_div"]
    return dict(d=d, E=E, run=run, n_div=nd)


def precode_batch(H, u_sym, mod_bits, params: Params, seed, chan_index=None):
    """Full VPP pipeline over P problems.  H: (n_chan, n_u, n_t) complex64, u_sym: (P, n_u)."""
    H = np.asarray(H, np.complex64)
    u_sym = np.asarray(u_sym, np.uint8)
    P, n_u = u_sym.shape
    n_t = H.shape[2]
    n = 2 * n_u
    out = dict(v=np.zeros((P, n_u, 2), np.int8), x=np.zeros((P, n_t), np.complex64),
               power=np.zeros(P, np.float32), E=np.zeros(P, np.int32), run=np.zeros(P, np.int32),
               n_div=np.zeros(P, np.int32), Aq=np.zeros((P, n, n), np.int16), hq=np.zeros((P, n), np.int16))
    for p in range(P):
        c = p if chan_index is None else int(chan_index[p])
        Hc = H[c].astype(np.complex128)
        b = build_precode(Hc, u_sym[p], mod_bits)
        r = cac_solve(b["Aq"], b["hq"], None, 0, params, seed, p)
        v, x, pw = precode_output(Hc, b["Q"], u_sym[p], r["d"], mod_bits)
        out["v"][p], out["x"][p], out["power"][p] = v, x, pw
        out["E"][p], out["run"][p], out["n_div"][p] = r["E"], r["run"], r["n_div"]
        out["Aq"][p], out["hq"][p] = b["Aq"], b["hq"]
    return out


# -------------------------------------------------------------- MMGaP-E
def sic_guess32(H, y, noise_var, mod_bits):
    """MMSE-SIC guess (sorted-Cholesky order), FP32 mirror; returns (g, perm, status)."""
    H = np.asarray(H)
    n_r, n_t = H.shape
    g = np.zeros(2 * n_t, np.int32)
    perm = np.zeros(n_t, np.int32)
    st = _lib.orc_sic_guess32(n_r, n_t, mod_bits, _c64(H), _c64(y), np.float32(noise_var), g, perm)
    return g, perm, st


def ml_objective32(H, y, x, mod_bits) -> np.float32:
    n_r, n_t = np.asarray(H).shape
    return np.float32(_lib.orc_ml_objective32(n_r, n_t, mod_bits, _c64(H), _c64(y),
                                              np.ascontiguousarray(x, np.int32)))


def stage_seed(seed, stage, inst) -> int:
    return int(_lib.orc_stage_seed(seed, stage, inst))


def detect_e(H, y, noise_var, mod_bits, stages, params: Params, seed, problem):
    """MMGaP-E of one problem: dict(sym, best, obj, candidates)."""
    H = np.asarray(H)
    n_r, n_t = H.shape
    nc = 2 + 2 * stages
    sym = np.zeros(n_t, np.uint8)
    best, obj = C.c_int(), C.c_float()
    X = np.zeros(nc * 2 * n_t, np.int32)
    cp = params.c()
    _lib.orc_detect_e(n_r, n_t, mod_bits, _c64(H), _c64(y), np.float32(noise_var), stages, C.byref(cp), int(seed),
                      int(problem), sym, C.byref(best), C.byref(obj), X)
    return dict(sym=sym, best=best.value, obj=obj.value, candidates=X.reshape(nc, 2 * n_t))


# ------------------------------------------------- direct (binary) mapping
_lib.orc_build_direct64.argtypes = [C.c_int, C.c_int, C.c_int, _f64p, _f64p, _nullable(_f64p), _nullable(_f64p),
                                    C.POINTER(C.c_double)]
_lib.orc_direct_lattice.argtypes = [C.c_int, C.c_int, _i8p, _i32p]
_lib.orc_direct_spins.argtypes = [C.c_int, C.c_int, _i32p, _i8p]
_lib.orc_energy_direct.restype = C.c_int32
_lib.orc_energy_direct.argtypes = [C.c_int, _i16p, _i16p, _i8p]
_lib.orc_build_direct32.argtypes = [C.c_int, C.c_int, C.c_int, _f32p, _f32p, C.c_float, _i32p, _nullable(_f32p),
                                    _nullable(_f32p), C.POINTER(C.c_int), _i16p, _i16p]
_lib.orc_general_field.argtypes = [C.c_int, _f32p, _f32p, _f32p, _f32p]
_lib.orc_cac_solve_general.argtypes = [C.c_int, _i16p, _i16p, _nullable(_i8p), C.POINTER(CParams), C.c_uint64,
                                       C.c_uint64, _i8p, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                       C.POINTER(C.c_int32), _nullable(_i32p), _nullable(_f32p)]
_lib.orc_detect_direct.argtypes = [C.c_int, C.c_int, C.c_int, _f32p, _f32p, C.c_float, C.POINTER(CParams),
                                   C.c_uint64, C.c_uint64, _u8p, _i32p, _i8p, C.POINTER(C.c_int32),
                                   C.POINTER(C.c_int32), C.POINTER(C.c_int32)]


def direct_spins_count(n_t, mod_bits) -> int:
    return 2 * n_t * (mod_bits // 2)


def build_direct64(H, y, mod_bits):
    """FP64 direct-mapping Ising form: dict(J (N, N), c (N,), const)."""
    H = np.asarray(H)
    n_r, n_t = H.shape
    N = direct_spins_count(n_t, mod_bits)
    J = np.zeros(N * N)
    c = np.zeros(N)
    k = C.c_double()
    st = _lib.orc_build_direct64(n_r, n_t, mod_bits, _c128(H), _c128(y), J, c, C.byref(k))
    if st:
        raise ValueError("invalid arguments")
    return dict(J=J.reshape(N, N), c=c, const=k.value)


def direct_lattice(n_t, mod_bits, s) -> np.ndarray:
    x = np.zeros(2 * n_t, np.int32)
    _lib.orc_direct_lattice(n_t, mod_bits, np.ascontiguousarray(s, np.int8), x)
    return x


def direct_spins(n_t, mod_bits, x) -> np.ndarray:
    s = np.zeros(direct_spins_count(n_t, mod_bits), np.int8)
    _lib.orc_direct_spins(n_t, mod_bits, np.ascontiguousarray(x, np.int32), s)
    return s


def energy_direct(Jq, cq, s) -> int:
    return int(_lib.orc_energy_direct(len(cq), np.ascontiguousarray(Jq, np.int16).ravel(),
                                      np.ascontiguousarray(cq, np.int16), np.ascontiguousarray(s, np.int8)))


def build_direct32(H, y, noise_var, mod_bits):
    """FP32 direct build in the pinned order: dict(g, J32, c32, sigma_exp, Jq, cq, status)."""
    H = np.asarray(H)
    n_r, n_t = H.shape
    N = direct_spins_count(n_t, mod_bits)
    g = np.zeros(2 * n_t, np.int32)
    J = np.zeros(N * N, np.float32)
    c = np.zeros(N, np.float32)
    se = C.c_int()
    Jq = np.zeros(N * N, np.int16)
    cq = np.zeros(N, np.int16)
    st = _lib.orc_build_direct32(n_r, n_t, mod_bits, _c64(H), _c64(y), np.float32(noise_var), g, J, c, C.byref(se),
                                 Jq, cq)
    return dict(status=st, g=g, J32=J.reshape(N, N), c32=c, sigma_exp=se.value, Jq=Jq.reshape(N, N), cq=cq)


def general_field(Jf, cf, x) -> np.ndarray:
    N = len(cf)
    mu = np.zeros(N + 1, np.float32)
    _lib.orc_general_field(N, np.ascontiguousarray(Jf, np.float32).ravel(), np.ascontiguousarray(cf, np.float32),
                           np.ascontiguousarray(x, np.float32), mu)
    return mu


def cac_solve_general(Jq, cq, s_ref, params: Params, seed, problem, want_energies=False, want_states=False):
    N = len(cq)
    s = np.zeros(N, np.int8)
    E, run, nd = C.c_int32(), C.c_int32(), C.c_int32()
    Er = np.zeros(params.runs, np.int32) if want_energies else None
    xf = np.zeros(params.runs * (N + 1), np.float32) if want_states else None
    sr = None if s_ref is None else np.ascontiguousarray(s_ref, np.int8)
    cp = params.c()
    st = _lib.orc_cac_solve_general(N, np.ascontiguousarray(Jq, np.int16).ravel(), np.ascontiguousarray(cq, np.int16),
                                    sr, C.byref(cp), int(seed), int(problem), s, C.byref(E), C.byref(run),
                                    C.byref(nd), Er, xf)
    if st:
        raise ValueError("invalid solver arguments")
    out = dict(s=s, E=E.value, run=run.value, n_div=nd.value)
    if want_energies:
        out["E_runs"] = Er
    if want_states:
        out["x_final"] = xf.reshape(params.runs, N + 1)
    return out


def detect_direct(H, y, noise_var, mod_bits, params: Params, seed, problem):
    """Direct-mapping detection of one problem: dict(sym, g, s, E, run, n_div)."""
    H = np.asarray(H)
    n_r, n_t = H.shape
    N = direct_spins_count(n_t, mod_bits)
    sym = np.zeros(n_t, np.uint8)
    g = np.zeros(2 * n_t, np.int32)
    s = np.zeros(N, np.int8)
    E, run, nd = C.c_int32(), C.c_int32(), C.c_int32()
    cp = params.c()
    _lib.orc_detect_direct(n_r, n_t, mod_bits, _c64(H), _c64(y), np.float32(noise_var), C.byref(cp), int(seed),
                           int(problem), sym, g, s, C.byref(E), C.byref(run), C.byref(nd))
    return dict(sym=sym, g=g, s=s, E=E.value, run=run.value, n_div=nd.value)
