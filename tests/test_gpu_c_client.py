"""The C ABI from a plain C program (tests/c_client/detect_client.c): no
Python in the process that calls the library.  The program is compiled here
against include/mmgap.h and the built library, runs mmgap_detect and
mmgap_detect_static on a job read from a file, and its outputs must equal the
CPU oracle's bit for bit."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _nvcc():
    return shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"


def test_c_client_detect_equals_the_oracle(tmp_path):
    from paper_2510_01579_gb300 import binding
    libdir = os.path.dirname(binding.LIB_PATH)
    exe = str(tmp_path / "detect_client")
    subprocess.run([_nvcc(), "-O2", "-o", exe, os.path.join(ROOT, "tests", "c_client", "detect_client.c"),
                    "-I", os.path.join(ROOT, "include"), "-L", libdir, "-lmmgap", "-Xlinker", "-rpath," + libdir],
                   check=True, capture_output=True)
    w = synth.uplink(404, 8, 8, 4, n_sub=24, n_sym=3, snr_db=14.0, model="kron", hold="prb")
    P, n_t, steps, seed = w["y"].shape[0], 8, 90, 0x0123456789AB
    job = str(tmp_path / "job.bin")
    with open(job, "wb") as f:
        np.array([8, n_t, 4, P, w["H"].shape[0], steps], np.int32).tofile(f)
        np.array([seed], np.uint64).tofile(f)
        w["H"].astype(np.complex64).tofile(f)
        w["y"].astype(np.complex64).tofile(f)
        w["noise_var"].astype(np.float32).tofile(f)
        w["chan_index"].astype(np.int32).tofile(f)
    out = str(tmp_path / "out.bin")
    r = subprocess.run([exe, job, out], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    raw = np.fromfile(out, np.uint8)
    per = P * n_t + 4 * P
    assert raw.size == 2 * per
    ref = oracle.detect_batch(w["H"], w["y"], w["noise_var"], 4, oracle.Params(steps=steps), seed, w["chan_index"])
    for part in (raw[:per], raw[per:]):  # mmgap_detect, then mmgap_detect_static
        sym = part[:P * n_t].reshape(P, n_t)
        E = part[P * n_t:].view(np.int32)
        assert np.array_equal(sym, ref["sym"])
        assert np.array_equal(E, ref["E"])
