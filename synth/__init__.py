"""Seeded synthetic workloads for the MIMO detector / precoder.

Stands in for the paper's Sionna UMi channels and Aerial PUSCH/PDSCH chains
(Sec. 5.1), which are not available: i.i.d. Rayleigh or Kronecker-correlated
CN(0,1) channels, uniform QAM symbols and AWGN, shaped like a 100 MHz / 30 kHz
NR slot (273 PRBs x 12 subcarriers = 3276 subcarriers, 14 OFDM symbols).

This module simulates the transmitter and the channel only (Eq. 1: y = Hx + n).
It holds none of the detector's or precoder's arithmetic; both the CUDA path
and the CPU oracle consume its arrays.

Conventions:
  * QAM symbol index q in [0, M): lattice point re = 2 (q // sqrt(M)) - L,
    im = 2 (q % sqrt(M)) - L with L = sqrt(M) - 1, physical symbol
    kappa * lattice with kappa = 1 / sqrt(2 (M - 1) / 3), so E|x|^2 = 1.
  * SNR is per user: noise variance sigma^2 = 10^(-SNR/10) per receive antenna.
  * Problem p = subcarrier * n_sym + symbol.  The channel is held constant over
    the 14 symbols of a subcarrier ("subcarrier") or over the 12 x 14 resource
    elements of a PRB ("prb"); chan_index[p] names the channel of problem p.
"""
from __future__ import annotations

import numpy as np

SUBCARRIERS_100MHZ_30KHZ = 3276
SUBCARRIERS_10MHZ_30KHZ = 288  # 24 PRBs: the high-connectivity 32x32 evaluation (Sec. 5)
SYMBOLS_PER_SLOT = 14
SUBCARRIERS_PER_PRB = 12


def _kappa(mod_bits: int) -> float:
    M = 1 << mod_bits
    return 1.0 / np.sqrt(2.0 * (M - 1) / 3.0)


def symbols_to_complex(sym: np.ndarray, mod_bits: int) -> np.ndarray:
    """Physical complex symbols of QAM indices (transmitter modulation)."""
    side = 1 << (mod_bits // 2)
    L = side - 1
    sym = np.asarray(sym, np.int64)
    re = 2 * (sym // side) - L
    im = 2 * (sym % side) - L
    return _kappa(mod_bits) * (re + 1j * im)


def gray_bits(sym: np.ndarray, mod_bits: int) -> np.ndarray:
    """Gray-coded bits of QAM indices, shape sym.shape + (mod_bits,)."""
    side = 1 << (mod_bits // 2)
    half = mod_bits // 2
    sym = np.asarray(sym, np.int64)
    out = []
    for comp in (sym // side, sym % side):
        gcode = comp ^ (comp >> 1)
        out += [(gcode >> b) & 1 for b in range(half)]
    return np.stack(out, axis=-1).astype(np.uint8)


def bit_errors(sym_hat: np.ndarray, sym_ref: np.ndarray, mod_bits: int) -> int:
    return int(np.count_nonzero(gray_bits(sym_hat, mod_bits) != gray_bits(sym_ref, mod_bits)))


def _cn01(rng, shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)


def _exp_corr_chol(n: int, rho: float) -> np.ndarray:
    idx = np.arange(n)
    R = rho ** np.abs(idx[:, None] - idx[None, :])
    return np.linalg.cholesky(R)


def channels(rng, n_chan: int, n_r: int, n_t: int, model: str = "iid", rho: float = 0.5) -> np.ndarray:
    """(n_chan, n_r, n_t) complex128 channels: 'iid' CN(0,1) entries, or
    'kron': L_r H_w L_t^T with exponential correlation rho^|i-j| at both ends."""
    Hw = _cn01(rng, (n_chan, n_r, n_t))
    if model == "iid":
        return Hw
    if model == "kron":
        Lr = _exp_corr_chol(n_r, rho)
        Lt = _exp_corr_chol(n_t, rho)
        return np.einsum("ij,cjk,lk->cil", Lr, Hw, Lt)
    raise ValueError(f"unknown channel model {model!r}")


def uplink(seed: int, n_r: int, n_t: int, mod_bits: int, n_sub: int = SUBCARRIERS_100MHZ_30KHZ,
           n_sym: int = SYMBOLS_PER_SLOT, snr_db=10.0, model: str = "iid", rho: float = 0.5,
           hold: str = "subcarrier"):
    """Uplink slot: P = n_sub * n_sym detection problems.

    snr_db: scalar, or one value per problem (e.g. an SNR sweep).
    Returns dict with H (n_chan, n_r, n_t) complex64, chan_index (P,) int32,
    y (P, n_r) complex64, noise_var (P,) float32, sym (P, n_t) uint8.
    """
    rng = np.random.default_rng(seed)
    P = n_sub * n_sym
    sub = np.arange(P) // n_sym
    if hold == "subcarrier":
        chan_index = sub
    elif hold == "prb":
        chan_index = sub // SUBCARRIERS_PER_PRB
    elif hold == "problem":
        chan_index = np.arange(P)
    else:
        raise ValueError(hold)
    n_chan = int(chan_index.max()) + 1 if P else 0
    H = channels(rng, n_chan, n_r, n_t, model, rho).astype(np.complex64)
    sym = rng.integers(0, 1 << mod_bits, size=(P, n_t)).astype(np.uint8)
    x = symbols_to_complex(sym, mod_bits)
    snr = np.broadcast_to(np.asarray(snr_db, np.float64), (P,))
    noise_var = (10.0 ** (-snr / 10.0)).astype(np.float32)
    noise = _cn01(rng, (P, n_r)) * np.sqrt(noise_var.astype(np.float64))[:, None]
    Hp = H.astype(np.complex128)[chan_index]
    y = (np.einsum("prt,pt->pr", Hp, x) + noise).astype(np.complex64)
    return dict(H=H, chan_index=chan_index.astype(np.int32), y=y, noise_var=noise_var, sym=sym,
                n_r=n_r, n_t=n_t, mod_bits=mod_bits)


def downlink(seed: int, n_u: int, n_t: int, mod_bits: int, n_sub: int = SUBCARRIERS_100MHZ_30KHZ,
             n_sym: int = 1, model: str = "iid", rho: float = 0.5):
    """Downlink precoding problems: one per (subcarrier, symbol); H (n_chan, n_u, n_t)
    is the users' channel, u_sym (P, n_u) the intended QAM indices."""
    rng = np.random.default_rng(seed)
    P = n_sub * n_sym
    chan_index = (np.arange(P) // n_sym).astype(np.int32)
    H = channels(rng, n_sub, n_u, n_t, model, rho).astype(np.complex64)
    u_sym = rng.integers(0, 1 << mod_bits, size=(P, n_u)).astype(np.uint8)
    return dict(H=H, chan_index=chan_index, u_sym=u_sym, n_u=n_u, n_t=n_t, mod_bits=mod_bits)


def random_ising(seed: int, P: int, n: int, scale: int = 1 << 14):
    """Random quantised delta-Ising problems (symmetric A_q, h_q) drawn the way
    the Appendix draws random instances: i.i.d. couplings, here uniform in
    [-scale, scale] as int16."""
    rng = np.random.default_rng(seed)
    A = rng.integers(-scale, scale + 1, size=(P, n, n))
    A = np.triu(A) + np.transpose(np.triu(A, 1), (0, 2, 1))
    h = rng.integers(-scale, scale + 1, size=(P, n))
    return A.astype(np.int16), h.astype(np.int16)
