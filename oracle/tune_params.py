"""Grid search of the CIM-CAC parameters the paper leaves open (p, a, zeta, eps
of Eqs. 10-11), on the oracle only.

The paper names these parameters (Sec. 2.3) but prints no values; Delta t =
0.02 and f_mvm = 2 are fixed by Appendix A.  Score = mean ML objective
||y - H x_hat||^2 (Eq. 2) of the detected vectors over seeded 16x16 16-QAM
problems at 16 dB (lower is better); the divergence count breaks ties.

    python -m oracle.tune_params [n_t] [mod_bits] [snr_db] [problems]
"""
import itertools
import sys
import time
from multiprocessing import get_context

import numpy as np

GRID = list(itertools.product([1.0, 1.1, 1.2, 1.3], [0.75, 1.0, 1.5], [2.0, 3.0, 4.0], [0.5, 1.0, 2.0]))


def _score(args):
    import oracle as o
    import synth
    (p, a, zeta, eps), n_t, mb, snr, P = args
    w = synth.uplink(11, n_t, n_t, mb, n_sub=P, n_sym=1, snr_db=snr, hold="problem")
    prm = o.Params(runs=32, steps=200, f_mvm=2, dt=0.02, p=p, a=a, zeta=zeta, eps=eps, sigma0=0.1)
    r = o.detect_batch(w["H"], w["y"], w["noise_var"], mb, prm, 99, w["chan_index"])
    obj = np.mean([np.linalg.norm(w["y"][i] - w["H"][i] @ synth.symbols_to_complex(r["sym"][i], mb)) ** 2
                   for i in range(P)])
    return (p, a, zeta, eps), float(obj), int(r["n_div"].sum())


def main(argv):
    n_t, mb, snr, P = int(argv[0]) if argv else 16, int(argv[1]) if len(argv) > 1 else 4, \
        float(argv[2]) if len(argv) > 2 else 16.0, int(argv[3]) if len(argv) > 3 else 96
    t0 = time.time()
    with get_context("spawn").Pool() as pool:
        res = pool.map(_score, [(g, n_t, mb, snr, P) for g in GRID])
    res.sort(key=lambda r: (r[1], r[2]))
    for r in res[:10]:
        print(r)
    print(f"{len(GRID)} settings in {time.time() - t0:.1f} s")


if __name__ == "__main__":
    main(sys.argv[1:])
