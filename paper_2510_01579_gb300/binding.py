"""Thin ctypes binding of the MMGaP C ABI (include/mmgap.h).

Argument marshalling only: torch CUDA tensors are checked (device, dtype,
shape, contiguity) and passed as raw device pointers together with the
current torch stream.  Every step of the detection / precoding path runs in
the library's CUDA kernels; there is no CPU fallback.  If libmmgap.so is
missing or fails to load, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
from typing import Optional

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmmgap.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libmmgap.so not built at {LIB_PATH}; run __graft_entry__.build() "
                      "or python -m paper_2510_01579_gb300.build")
_lib = C.CDLL(LIB_PATH)

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED, EBUSY = range(7)
_STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "EUNSUPPORTED", 6: "EBUSY"}

# User counts of every call; detect / build_detect (delta mapping, FP32 Gram) and
# solve_ising (n = 64) also take 32 users.
SUPPORTED_NT = (1, 2, 3, 4, 8, 16)


class MMGaPError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class _Params(C.Structure):
    _fields_ = [("runs", C.c_int32), ("steps", C.c_int32), ("f_mvm", C.c_int32), ("dt", C.c_float),
                ("p", C.c_float), ("a", C.c_float), ("zeta", C.c_float), ("eps", C.c_float),
                ("sigma0", C.c_float), ("x_max", C.c_float), ("early_exit", C.c_int32)]


class _DetectJob(C.Structure):
    _fields_ = [("n_r", C.c_int32), ("n_t", C.c_int32), ("mod_bits", C.c_int32), ("n_problems", C.c_int32),
                ("n_chan", C.c_int32), ("chan_index", C.c_void_p), ("H", C.c_void_p), ("y", C.c_void_p),
                ("noise_var", C.c_void_p), ("seed", C.c_uint64), ("sym_out", C.c_void_p),
                ("energy_out", C.c_void_p), ("guess_out", C.c_void_p), ("offset_out", C.c_void_p),
                ("ndiv_out", C.c_void_p), ("gram_precision", C.c_int32), ("mapping", C.c_int32),
                ("guess_in", C.c_void_p), ("steps_out", C.c_void_p), ("problem_offset", C.c_uint64)]


class _PrecodeJob(C.Structure):
    _fields_ = [("n_u", C.c_int32), ("n_t", C.c_int32), ("mod_bits", C.c_int32), ("n_problems", C.c_int32),
                ("n_chan", C.c_int32), ("inv_precision", C.c_int32), ("chan_index", C.c_void_p), ("H", C.c_void_p),
                ("u_sym", C.c_void_p), ("seed", C.c_uint64), ("v_out", C.c_void_p), ("x_out", C.c_void_p), ("power_out", C.c_void_p),
                ("energy_out", C.c_void_p), ("ndiv_out", C.c_void_p)]


_vp = C.c_void_p
_lib.mmgap_default_params.argtypes = [C.POINTER(_Params)]
_lib.mmgap_create.argtypes = [C.POINTER(_vp), C.c_int, C.c_size_t]
_lib.mmgap_destroy.argtypes = [_vp]
_lib.mmgap_last_error.argtypes = [_vp]
_lib.mmgap_last_error.restype = C.c_char_p
_lib.mmgap_detect.argtypes = [_vp, C.POINTER(_Params), C.POINTER(_DetectJob), C.c_int, _vp]
_lib.mmgap_precode.argtypes = [_vp, C.POINTER(_Params), C.POINTER(_PrecodeJob), C.c_int, _vp]
_lib.mmgap_solve_ising.argtypes = [_vp, C.POINTER(_Params), C.c_int, C.c_int, _vp, _vp, _vp, C.c_int, C.c_uint64,
                                   _vp, _vp, _vp, _vp, _vp]
_lib.mmgap_build_detect.argtypes = [_vp, C.POINTER(_DetectJob), _vp, _vp, _vp, _vp, _vp, _vp, _vp]
_lib.mmgap_set_timing.argtypes = [_vp, C.c_int]
_lib.mmgap_stage_times.argtypes = [_vp, C.POINTER(C.c_float), C.POINTER(C.c_int)]
_lib.mmgap_device_errors.argtypes = [_vp, C.POINTER(C.c_int), C.c_int]
_lib.mmgap_detect_static.argtypes = [C.POINTER(_Params), C.POINTER(_DetectJob), _vp]
_lib.mmgap_set_solver_variant.argtypes = [_vp, C.c_int, C.c_int]
_lib.mmgap_set_device_wait.argtypes = [_vp, C.c_uint64]
_lib.mmgap_detect_e.argtypes = [_vp, C.POINTER(_Params), C.POINTER(_DetectJob), C.c_int, _vp, _vp, _vp, _vp]
_lib.mmgap_vpp_inverse.argtypes = [_vp, C.c_int, C.c_int, C.c_int, _vp, C.c_int, _vp, _vp, _vp]
_lib.mmgap_solve_general.argtypes = [_vp, C.POINTER(_Params), C.c_int, C.c_int, _vp, _vp, _vp, C.c_uint64, _vp, _vp,
                                     _vp, _vp, _vp]
_lib.mmgap_anneal_spins.argtypes = [_vp, C.POINTER(_Params), C.c_int, C.c_int, _vp, _vp, C.c_uint64, _vp, _vp]
_lib.mmgap_get_solver_variant.argtypes = [_vp, C.c_int, C.c_int, C.POINTER(C.c_int)]
_lib.mmgap_autotune.argtypes = [_vp, C.POINTER(_Params), C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_float)]
_lib.mmgap_batch_create.argtypes = [C.POINTER(_vp), C.c_int, C.POINTER(_Params), C.POINTER(_DetectJob), C.c_int,
                                    C.c_int]
_lib.mmgap_batch_run.argtypes = [_vp, C.c_int, _vp]
_lib.mmgap_batch_destroy.argtypes = [_vp]


class _ServerConfig(C.Structure):
    _fields_ = [("n_lanes", C.c_int32), ("max_jobs_per_group", C.c_int32), ("max_problems_per_group", C.c_int64),
                ("scratch_bytes", C.c_size_t), ("max_n_t", C.c_int32), ("max_n_r", C.c_int32),
                ("deadline_us", C.c_double), ("inject_delay_us", C.c_double), ("use_graph", C.c_int32),
                ("tensor_core", C.c_int32)]


class _JobInfo(C.Structure):
    _fields_ = [("ticket", C.c_uint64), ("status", C.c_int32), ("submit_us", C.c_double), ("start_us", C.c_double),
                ("done_us", C.c_double)]


class _ServerStats(C.Structure):
    _fields_ = [("completed", C.c_int64), ("problems", C.c_int64), ("deadline_misses", C.c_int64),
                ("groups", C.c_int64), ("max_group_jobs", C.c_int64), ("queued", C.c_int64), ("p50_us", C.c_double),
                ("p99_us", C.c_double), ("max_us", C.c_double), ("mean_us", C.c_double), ("span_us", C.c_double)]


_lib.mmgap_server_create.argtypes = [C.POINTER(_vp), C.c_int, C.POINTER(_Params), C.POINTER(_ServerConfig)]
_lib.mmgap_server_submit.argtypes = [_vp, C.POINTER(_DetectJob), C.POINTER(C.c_uint64)]
_lib.mmgap_server_submit_precode.argtypes = [_vp, C.POINTER(_PrecodeJob), C.POINTER(C.c_uint64)]
_lib.mmgap_server_wait.argtypes = [_vp, C.c_uint64, C.c_int64, C.POINTER(_JobInfo)]
_lib.mmgap_server_stats.argtypes = [_vp, C.POINTER(_ServerStats), C.c_int]
_lib.mmgap_server_destroy.argtypes = [_vp]
for _f in ("mmgap_default_params", "mmgap_create", "mmgap_destroy", "mmgap_detect", "mmgap_precode",
           "mmgap_solve_ising", "mmgap_build_detect", "mmgap_set_timing", "mmgap_stage_times",
           "mmgap_device_errors", "mmgap_detect_static", "mmgap_set_solver_variant", "mmgap_get_solver_variant",
           "mmgap_set_device_wait",
           "mmgap_detect_e", "mmgap_anneal_spins", "mmgap_vpp_inverse", "mmgap_solve_general",
           "mmgap_autotune", "mmgap_batch_create", "mmgap_batch_run", "mmgap_batch_destroy", "mmgap_server_create",
           "mmgap_server_submit", "mmgap_server_submit_precode", "mmgap_server_wait", "mmgap_server_stats",
           "mmgap_server_destroy"):
    getattr(_lib, _f).restype = C.c_int

ABI_SYMBOLS = ("mmgap_default_params", "mmgap_create", "mmgap_destroy", "mmgap_last_error", "mmgap_detect",
               "mmgap_precode", "mmgap_solve_ising", "mmgap_build_detect", "mmgap_set_timing",
               "mmgap_stage_times", "mmgap_device_errors", "mmgap_detect_static", "mmgap_set_solver_variant",
               "mmgap_detect_e", "mmgap_anneal_spins", "mmgap_vpp_inverse", "mmgap_solve_general",
               "mmgap_get_solver_variant", "mmgap_autotune", "mmgap_batch_create", "mmgap_batch_run",
               "mmgap_batch_destroy", "mmgap_server_create", "mmgap_server_submit", "mmgap_server_submit_precode",
               "mmgap_server_wait", "mmgap_server_stats", "mmgap_server_destroy", "mmgap_set_device_wait")

VARIANT_NAMES = {0: "default", 1: "plain", 2: "tpa1", 3: "tpa1-packed", 4: "tpa2-packed", 5: "tensor-core",
                 6: "pair-packed", 7: "tensor-core-tpa2", 8: "tcgen05", 9: "tpa4-packed", 10: "tpa8-packed"}


@dataclasses.dataclass
class Params:
    """Solver parameters (mmgap_params); defaults from mmgap_default_params."""
    runs: int
    steps: int
    f_mvm: int
    dt: float
    p: float
    a: float
    zeta: float
    eps: float
    sigma0: float
    x_max: float
    early_exit: int = 0

    @classmethod
    def default(cls, **overrides) -> "Params":
        c = _Params()
        _lib.mmgap_default_params(C.byref(c))
        kw = {f: getattr(c, f) for f, _ in _Params._fields_}
        kw.update(overrides)
        return cls(**kw)

    def _c(self) -> _Params:
        return _Params(self.runs, self.steps, self.f_mvm, self.dt, self.p, self.a, self.zeta, self.eps,
                       self.sigma0, self.x_max, self.early_exit)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _check(t, name, dtype, shape, device):
    if t is None:
        return
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.device != device:
        raise ValueError(f"{name} is on {t.device}, expected {device}")
    if t.dtype != dtype:
        raise TypeError(f"{name} has dtype {t.dtype}, expected {dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class Context:
    """An mmgap_ctx on one CUDA device (owns the device workspace)."""

    def __init__(self, device: int = 0, workspace_bytes: int = 0):
        self.device = torch.device("cuda", device)
        h = C.c_void_p()
        st = _lib.mmgap_create(C.byref(h), device, workspace_bytes)
        if st != OK:
            raise MMGaPError(st, "mmgap_create failed")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib.mmgap_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _stream(self):
        return C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def _raise(self, st):
        if st != OK:
            raise MMGaPError(st, _lib.mmgap_last_error(self._h).decode())

    # ------------------------------------------------------------------ API
    def detect(self, H, y, noise_var, mod_bits: int, params: Params, seed: int, chan_index=None,
               want_energy=False, want_guess=False, want_offset=False, want_ndiv=False, gram_precision: int = 0,
               mapping: int = 0, guess=None, want_steps=False):
        """Uplink detection of P problems.  H: complex64 (n_chan, n_r, n_t),
        y: complex64 (P, n_r), noise_var: float32 (P,), chan_index: int32 (P,)
        or None, guess: int8 (P, 2 n_t) lattice guess replacing MMSE, or None.
        Returns a dict of CUDA tensors (sym uint8 (P, n_t), ...)."""
        n_chan, n_r, n_t = H.shape
        P = y.shape[0]
        dev = self.device
        _check(H, "H", torch.complex64, (n_chan, n_r, n_t), dev)
        _check(y, "y", torch.complex64, (P, n_r), dev)
        _check(noise_var, "noise_var", torch.float32, (P,), dev)
        _check(chan_index, "chan_index", torch.int32, (P,), dev)
        _check(guess, "guess", torch.int8, (P, 2 * n_t), dev)
        out = {"sym": torch.empty((P, n_t), dtype=torch.uint8, device=dev)}
        if want_steps:
            out["steps"] = torch.empty(P, dtype=torch.int32, device=dev)
        if want_energy:
            out["energy"] = torch.empty(P, dtype=torch.int32, device=dev)
        if want_guess:
            out["guess"] = torch.empty((P, 2 * n_t), dtype=torch.int8, device=dev)
        if want_offset:
            out["offset"] = torch.empty((P, 2 * n_t), dtype=torch.int8, device=dev)
        if want_ndiv:
            out["ndiv"] = torch.empty(P, dtype=torch.int32, device=dev)
        job = self.detect_job(H, y, noise_var, mod_bits, seed, out, chan_index, gram_precision, mapping, guess)
        self.detect_jobs([job], params)
        return out

    def detect_e(self, H, y, noise_var, mod_bits: int, params: Params, seed: int, stages: int = 1, chan_index=None,
                 want_candidates=False, gram_precision: int = 0):
        """MMGaP-E (multi-stage, MMSE and MMSE-SIC guesses).  Returns dict(sym,
        best, obj[, candidates (2 + 2 stages, P, 2 n_t)])."""
        n_chan, n_r, n_t = H.shape
        P = y.shape[0]
        dev = self.device
        _check(H, "H", torch.complex64, (n_chan, n_r, n_t), dev)
        _check(y, "y", torch.complex64, (P, n_r), dev)
        _check(noise_var, "noise_var", torch.float32, (P,), dev)
        _check(chan_index, "chan_index", torch.int32, (P,), dev)
        out = {"sym": torch.empty((P, n_t), dtype=torch.uint8, device=dev),
               "best": torch.empty(P, dtype=torch.int32, device=dev),
               "obj": torch.empty(P, dtype=torch.float32, device=dev)}
        if want_candidates:
            out["candidates"] = torch.empty((2 + 2 * stages, P, 2 * n_t), dtype=torch.int8, device=dev)
        job = self.detect_job(H, y, noise_var, mod_bits, seed, out, chan_index, gram_precision)
        cp = params._c()
        self._raise(_lib.mmgap_detect_e(self._h, C.byref(cp), C.byref(job), stages, _ptr(out["best"]),
                                        _ptr(out["obj"]), _ptr(out.get("candidates")), self._stream()))
        return out

    def detect_job(self, H, y, noise_var, mod_bits, seed, out, chan_index=None, gram_precision=0,
                   mapping=0, guess=None, problem_offset=0) -> _DetectJob:
        """A detection job descriptor over device tensors.  out: dict with "sym" and optional
        "energy", "guess", "offset", "ndiv", "steps"; guess: int8 (P, 2 n_t) input guess or None;
        problem_offset: Philox counter index of problem 0 (a shard of a larger job)."""
        n_chan, n_r, n_t = H.shape
        return _DetectJob(n_r, n_t, mod_bits, y.shape[0], n_chan, _ptr(chan_index), _ptr(H), _ptr(y),
                          _ptr(noise_var), seed, _ptr(out["sym"]), _ptr(out.get("energy")), _ptr(out.get("guess")),
                          _ptr(out.get("offset")), _ptr(out.get("ndiv")), gram_precision, mapping, _ptr(guess),
                          _ptr(out.get("steps")), problem_offset)

    def detect_jobs(self, jobs, params: Params, stream=None):
        arr = (_DetectJob * len(jobs))(*jobs)
        cp = params._c()
        s = self._stream() if stream is None else C.c_void_p(stream.cuda_stream)
        self._raise(_lib.mmgap_detect(self._h, C.byref(cp), arr, len(jobs), s))

    def precode_job(self, H, u_sym, mod_bits, seed, out, chan_index=None, inv_precision=0) -> _PrecodeJob:
        """A precoding job descriptor over device tensors (for Server.submit_precode).
        out: dict with "v" int8 (P, n_u, 2) and optional "x" complex64 (P, n_t), "power" float32 (P,),
        "energy" / "ndiv" int32 (P,)."""
        n_chan, n_u, n_t = H.shape
        return _PrecodeJob(n_u, n_t, mod_bits, u_sym.shape[0], n_chan, inv_precision, _ptr(chan_index), _ptr(H),
                           _ptr(u_sym), seed, _ptr(out["v"]), _ptr(out.get("x")), _ptr(out.get("power")),
                           _ptr(out.get("energy")), _ptr(out.get("ndiv")))

    def precode_jobs(self, jobs, params: Params, stream=None):
        arr = (_PrecodeJob * len(jobs))(*jobs)
        cp = params._c()
        s = self._stream() if stream is None else C.c_void_p(stream.cuda_stream)
        self._raise(_lib.mmgap_precode(self._h, C.byref(cp), arr, len(jobs), s))

    def precode(self, H, u_sym, mod_bits: int, params: Params, seed: int, chan_index=None, want_x=True,
                want_power=True, want_energy=False, want_ndiv=False, inv_precision=0):
        """Downlink VPP of P problems.  H: complex64 (n_chan, n_u, n_t), u_sym: uint8 (P, n_u);
        inv_precision 0 = FP64 channel inverse, 1 = FP32 with iterative refinement."""
        n_chan, n_u, n_t = H.shape
        P = u_sym.shape[0]
        dev = self.device
        _check(H, "H", torch.complex64, (n_chan, n_u, n_t), dev)
        _check(u_sym, "u_sym", torch.uint8, (P, n_u), dev)
        _check(chan_index, "chan_index", torch.int32, (P,), dev)
        out = {"v": torch.empty((P, n_u, 2), dtype=torch.int8, device=dev)}
        if want_x:
            out["x"] = torch.empty((P, n_t), dtype=torch.complex64, device=dev)
        if want_power:
            out["power"] = torch.empty(P, dtype=torch.float32, device=dev)
        if want_energy:
            out["energy"] = torch.empty(P, dtype=torch.int32, device=dev)
        if want_ndiv:
            out["ndiv"] = torch.empty(P, dtype=torch.int32, device=dev)
        job = _PrecodeJob(n_u, n_t, mod_bits, P, n_chan, inv_precision, _ptr(chan_index), _ptr(H), _ptr(u_sym),
                          seed, _ptr(out["v"]), _ptr(out.get("x")), _ptr(out.get("power")), _ptr(out.get("energy")),
                          _ptr(out.get("ndiv")))
        cp = params._c()
        arr = (_PrecodeJob * 1)(job)
        self._raise(_lib.mmgap_precode(self._h, C.byref(cp), arr, 1, self._stream()))
        return out

    def vpp_inverse(self, H, inv_precision=0):
        """Q = (H H^H)^-1 per channel.  H: complex64 (n_chan, n_u, n_t).  Returns Q complex128
        (n_chan, n_u, n_u) and status int32 (n_chan,)."""
        n_chan, n_u, n_t = H.shape
        _check(H, "H", torch.complex64, (n_chan, n_u, n_t), self.device)
        Q = torch.empty((n_chan, n_u, n_u), dtype=torch.complex128, device=self.device)
        st = torch.empty(n_chan, dtype=torch.int32, device=self.device)
        self._raise(_lib.mmgap_vpp_inverse(self._h, n_u, n_t, n_chan, _ptr(H), inv_precision, _ptr(Q), _ptr(st),
                                           self._stream()))
        return Q, st

    def solve_general(self, J_q, c_q, params: Params, seed: int, s_ref=None):
        """Anneal P general Ising problems with an auxiliary spin: J_q int16 (P, N, N), c_q int16 (P, N),
        s_ref int8 (P, N) or None.  Returns s int8 (P, N), E, run, ndiv int32 (P,)."""
        P, N, _ = J_q.shape
        dev = self.device
        _check(J_q, "J_q", torch.int16, (P, N, N), dev)
        _check(c_q, "c_q", torch.int16, (P, N), dev)
        _check(s_ref, "s_ref", torch.int8, (P, N), dev)
        out = dict(s=torch.empty((P, N), dtype=torch.int8, device=dev),
                   E=torch.empty(P, dtype=torch.int32, device=dev),
                   run=torch.empty(P, dtype=torch.int32, device=dev),
                   ndiv=torch.empty(P, dtype=torch.int32, device=dev))
        cp = params._c()
        self._raise(_lib.mmgap_solve_general(self._h, C.byref(cp), N, P, _ptr(J_q), _ptr(c_q), _ptr(s_ref), seed,
                                             _ptr(out["s"]), _ptr(out["E"]), _ptr(out["run"]), _ptr(out["ndiv"]),
                                             self._stream()))
        return out

    def solve_ising(self, A_q, h_q, params: Params, seed: int, g=None, level_max: int = 0):
        """Anneal P quantised delta-Ising problems: A_q int16 (P, n, n), h_q int16 (P, n),
        g int8 (P, n) or None.  Returns d int8 (P, n), E, run, ndiv int32 (P,)."""
        P, n, _ = A_q.shape
        dev = self.device
        _check(A_q, "A_q", torch.int16, (P, n, n), dev)
        _check(h_q, "h_q", torch.int16, (P, n), dev)
        _check(g, "g", torch.int8, (P, n), dev)
        d = torch.empty((P, n), dtype=torch.int8, device=dev)
        E = torch.empty(P, dtype=torch.int32, device=dev)
        run = torch.empty(P, dtype=torch.int32, device=dev)
        nd = torch.empty(P, dtype=torch.int32, device=dev)
        cp = params._c()
        self._raise(_lib.mmgap_solve_ising(self._h, C.byref(cp), n, P, _ptr(A_q), _ptr(h_q), _ptr(g), level_max,
                                           seed, _ptr(d), _ptr(E), _ptr(run), _ptr(nd), self._stream()))
        return dict(d=d, E=E, run=run, ndiv=nd)

    def anneal_spins(self, A_q, h_q, params: Params, seed: int):
        """Final sign bits of every anneal (Appendix A study): uint64 (P, runs, 2),
        word 1 bit 63 = diverged."""
        P, n, _ = A_q.shape
        dev = self.device
        _check(A_q, "A_q", torch.int16, (P, n, n), dev)
        _check(h_q, "h_q", torch.int16, (P, n), dev)
        out = torch.empty((P, params.runs, 2), dtype=torch.int64, device=dev)
        cp = params._c()
        self._raise(_lib.mmgap_anneal_spins(self._h, C.byref(cp), n, P, _ptr(A_q), _ptr(h_q), seed, _ptr(out),
                                            self._stream()))
        return out

    def build_detect(self, H, y, noise_var, mod_bits: int, chan_index=None, want_float=True, gram_precision=0,
                     mapping=0, guess=None):
        """Builder only: quantised Ising coefficients of P detection problems (delta form:
        A_q (P, n, n), h_q (P, n); direct form, mapping=1: J_q (P, N, N), c_q (P, N) in the same keys)."""
        n_chan, n_r, n_t = H.shape
        P = y.shape[0]
        n = 2 * n_t if mapping == 0 else 2 * n_t * (mod_bits // 2)
        dev = self.device
        _check(H, "H", torch.complex64, (n_chan, n_r, n_t), dev)
        _check(y, "y", torch.complex64, (P, n_r), dev)
        _check(noise_var, "noise_var", torch.float32, (P,), dev)
        _check(chan_index, "chan_index", torch.int32, (P,), dev)
        out = dict(A_q=torch.empty((P, n, n), dtype=torch.int16, device=dev),
                   h_q=torch.empty((P, n), dtype=torch.int16, device=dev),
                   g=torch.empty((P, 2 * n_t), dtype=torch.int8, device=dev))
        if want_float:
            out["G"] = torch.empty((P, n, n), dtype=torch.float32, device=dev)
            out["h"] = torch.empty((P, n), dtype=torch.float32, device=dev)
            out["sigma_exp"] = torch.empty(P, dtype=torch.int32, device=dev)
        _check(guess, "guess", torch.int8, (P, 2 * n_t), dev)
        job = _DetectJob(n_r, n_t, mod_bits, P, n_chan, _ptr(chan_index), _ptr(H), _ptr(y), _ptr(noise_var), 0,
                         None, None, None, None, None, gram_precision, mapping, _ptr(guess), None)
        self._raise(_lib.mmgap_build_detect(self._h, C.byref(job), _ptr(out["A_q"]), _ptr(out["h_q"]),
                                            _ptr(out["g"]), _ptr(out.get("G")), _ptr(out.get("h")),
                                            _ptr(out.get("sigma_exp")), self._stream()))
        return out

    def detect_static(self, job: _DetectJob, params: Params):
        """mmgap_detect_static on this context's device: the same detection
        without any allocation (scratch in a fixed array inside the library),
        for callers that must not allocate device memory."""
        cp = params._c()
        st = _lib.mmgap_detect_static(C.byref(cp), C.byref(job), self._stream())
        if st != OK:
            raise MMGaPError(st, "mmgap_detect_static failed (see stderr)")

    def set_device_wait(self, limit_ns: int):
        """Limit of the bounded device-side waits of later calls (default 0.2 s; 0 = give up at once)."""
        self._raise(_lib.mmgap_set_device_wait(self._h, int(limit_ns)))

    def set_solver_variant(self, n_t: int, variant: int):
        """Force the solver's launch shape for n_t users (0 = size default)."""
        self._raise(_lib.mmgap_set_solver_variant(self._h, n_t, variant))

    def solver_variant(self, n_t: int, f_mvm: int = 2) -> int:
        v = C.c_int()
        self._raise(_lib.mmgap_get_solver_variant(self._h, n_t, f_mvm, C.byref(v)))
        return v.value

    def autotune(self, params: Params, n_t: int, n_problems: int = 0):
        """Time every compiled launch shape, keep the fastest; returns (shape, {shape: ms})."""
        v = C.c_int()
        ms = (C.c_float * 16)()
        cp = params._c()
        self._raise(_lib.mmgap_autotune(self._h, C.byref(cp), n_t, n_problems, C.byref(v), ms))
        return v.value, {i: ms[i] for i in range(1, 16) if ms[i] >= 0}

    def set_timing(self, enable: bool):
        self._raise(_lib.mmgap_set_timing(self._h, 1 if enable else 0))

    def stage_times(self):
        """(build_ms, solve_ms, output_ms, total_ms, n_chunks) of the last timed call."""
        ms = (C.c_float * 4)()
        nc = C.c_int()
        self._raise(_lib.mmgap_stage_times(self._h, ms, C.byref(nc)))
        return (ms[0], ms[1], ms[2], ms[3], nc.value)

    def device_errors(self, clear: bool = True) -> int:
        f = C.c_int()
        self._raise(_lib.mmgap_device_errors(self._h, C.byref(f), 1 if clear else 0))
        return f.value


class Batch:
    """mmgap_batch: a fixed set of uplink jobs of mixed sizes run by one
    builder and one solver launch (optionally replayed from a CUDA graph):
    one CTA per problem, or tcgen05 tiles of 4 problems for 8 and 16 users
    (tensor_core=True, the precision variant of solver shape 8).  The jobs' tensors must stay alive (and at the same
    addresses) for the life of the batch; their contents may change between
    runs."""

    def __init__(self, device: int, params: Params, jobs, keepalive=(), tensor_core: bool = False):
        self._keep = list(keepalive)
        arr = (_DetectJob * len(jobs))(*jobs)
        cp = params._c()
        h = C.c_void_p()
        flags = 2 if tensor_core else 0
        st = _lib.mmgap_batch_create(C.byref(h), device, C.byref(cp), arr, len(jobs), flags)
        if st != OK:
            raise MMGaPError(st, "mmgap_batch_create failed (see stderr)")
        self._h = h
        self.device = torch.device("cuda", device)

    def run(self, use_graph: bool = False, stream=None):
        s = torch.cuda.current_stream(self.device) if stream is None else stream
        st = _lib.mmgap_batch_run(self._h, 1 if use_graph else 0, C.c_void_p(s.cuda_stream))
        if st != OK:
            raise MMGaPError(st, "mmgap_batch_run failed (see stderr)")

    def close(self):
        if getattr(self, "_h", None):
            _lib.mmgap_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Server:
    """mmgap_server: continuous-batching serving loop on one device.

    submit() queues a detection job and submit_precode() a VPP precoding job
    (device tensors, kept alive by the caller or via `keepalive`); both return a ticket; wait() blocks until it is
    done (or raises MMGaPError with ETIMEOUT); stats() gives latency
    percentiles of completed jobs."""

    def __init__(self, device: int, params: Params, scratch_bytes: int = 1 << 30, n_lanes: int = 2,
                 max_jobs_per_group: int = 64, max_problems_per_group: int = 1 << 20, max_n_t: int = 16,
                 max_n_r: int = 16, deadline_us: float = 0.0, inject_delay_us: float = 0.0, use_graph: bool = True,
                 tensor_core: bool = False):
        cfg = _ServerConfig(n_lanes, max_jobs_per_group, max_problems_per_group, scratch_bytes, max_n_t, max_n_r,
                            deadline_us, inject_delay_us, 1 if use_graph else 0, 1 if tensor_core else 0)
        cp = params._c()
        h = C.c_void_p()
        st = _lib.mmgap_server_create(C.byref(h), device, C.byref(cp), C.byref(cfg))
        if st != OK:
            raise MMGaPError(st, "mmgap_server_create failed (see stderr)")
        self._h = h
        self._keep = {}

    def submit(self, job: _DetectJob, keepalive=None) -> int:
        t = C.c_uint64()
        st = _lib.mmgap_server_submit(self._h, C.byref(job), C.byref(t))
        if st != OK:
            raise MMGaPError(st, "mmgap_server_submit failed")
        if keepalive is not None:
            self._keep[t.value] = keepalive
        return t.value

    def submit_precode(self, job: _PrecodeJob, keepalive=None) -> int:
        t = C.c_uint64()
        st = _lib.mmgap_server_submit_precode(self._h, C.byref(job), C.byref(t))
        if st != OK:
            raise MMGaPError(st, "mmgap_server_submit_precode failed")
        if keepalive is not None:
            self._keep[t.value] = keepalive
        return t.value

    def wait(self, ticket: int, timeout_us: int = -1) -> dict:
        info = _JobInfo()
        st = _lib.mmgap_server_wait(self._h, ticket, timeout_us, C.byref(info))
        if st != OK:
            raise MMGaPError(st, f"ticket {ticket}")
        self._keep.pop(ticket, None)
        return {"submit_us": info.submit_us, "start_us": info.start_us, "done_us": info.done_us,
                "latency_us": info.done_us - info.submit_us}

    def stats(self, reset: bool = False) -> dict:
        s = _ServerStats()
        st = _lib.mmgap_server_stats(self._h, C.byref(s), 1 if reset else 0)
        if st != OK:
            raise MMGaPError(st, "server fault")
        return {f: getattr(s, f) for f, _ in _ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            _lib.mmgap_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
