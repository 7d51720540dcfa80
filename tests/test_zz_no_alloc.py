"""mmgap_detect_static against mmgap_detect.

mmgap_detect_static is for callers that cannot allocate device memory: a
real-time slot loop that must not call cudaMalloc once running (an
allocation can synchronise the device and miss the slot), or a plug-in inside
an application that owns all device memory.  It takes its scratch from a fixed
array inside the library instead of a context workspace.  Its results must be
the same bits as the context path's, call after call, although the array
keeps the previous call's contents, and a repeated call must not change the
device's free memory.

This file sorts last so that a run stopping at the first failure has already
run every other test.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


def _T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _outputs(P, n_t):
    return {"sym": torch.full((P, n_t), 255, dtype=torch.uint8, device=DEV),
            "energy": torch.full((P,), 7, dtype=torch.int32, device=DEV),
            "guess": torch.zeros((P, 2 * n_t), dtype=torch.int8, device=DEV),
            "offset": torch.zeros((P, 2 * n_t), dtype=torch.int8, device=DEV),
            "ndiv": torch.full((P,), -1, dtype=torch.int32, device=DEV)}


def test_static_scratch_matches_context_path_two_calls_in_a_row():
    import paper_2510_01579_gb300 as pkg
    prm = pkg.Params.default(steps=120)
    cases = [synth.uplink(61, 16, 16, 4, n_sub=20, n_sym=10, snr_db=14.0),      # 200 problems, 16 users
             synth.uplink(62, 8, 8, 2, n_sub=30, n_sym=10, snr_db=8.0, model="kron", hold="prb"),  # 300, 8 users
             synth.uplink(64, 32, 32, 4, n_sub=12, n_sym=10, snr_db=18.0)]     # 120 problems, 32 users
    with pkg.Context(0) as ctx:
        for i, w in enumerate(cases):
            P, n_t = w["y"].shape[0], w["n_t"]
            H, y, nv, ci = _T(w["H"]), _T(w["y"]), _T(w["noise_var"]), _T(w["chan_index"])
            ref = _outputs(P, n_t)
            ctx.detect_jobs([ctx.detect_job(H, y, nv, w["mod_bits"], 900 + i, ref, ci)], prm)
            got = _outputs(P, n_t)
            ctx.detect_static(ctx.detect_job(H, y, nv, w["mod_bits"], 900 + i, got, ci), prm)
            torch.cuda.synchronize()
            for k in ref:
                assert torch.equal(got[k], ref[k]), (i, k)
            # the same call again: same bits, and no device memory taken (the outputs are allocated
            # before the free memory is read)
            again = _outputs(P, n_t)
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info(DEV)[0]
            ctx.detect_static(ctx.detect_job(H, y, nv, w["mod_bits"], 900 + i, again, ci), prm)
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info(DEV)[0] == free0, i
            for k in ref:
                assert torch.equal(again[k], ref[k]), (i, k)


def test_static_scratch_with_guess_and_early_exit():
    """A caller-supplied guess, early exit and the steps output through the
    static entry point equal the context path, on two calls in a row."""
    import paper_2510_01579_gb300 as pkg
    prm = pkg.Params.default(early_exit=3)
    w = synth.uplink(65, 16, 16, 4, n_sub=30, n_sym=8, snr_db=15.0)
    P = w["y"].shape[0]
    side, L = 4, 3
    sym = w["sym"].astype(int)
    g = np.concatenate([2 * (sym // side) - L, 2 * (sym % side) - L], axis=1).astype(np.int8)
    g[::3, 0] = np.where(g[::3, 0] > -L, g[::3, 0] - 2, g[::3, 0] + 2)
    H, y, nv, ci, gt = _T(w["H"]), _T(w["y"]), _T(w["noise_var"]), _T(w["chan_index"]), _T(g)
    with pkg.Context(0) as ctx:
        ref = dict(_outputs(P, 16), steps=torch.full((P,), -1, dtype=torch.int32, device=DEV))
        ctx.detect_jobs([ctx.detect_job(H, y, nv, 4, 5, ref, ci, guess=gt)], prm)
        for _ in range(2):
            got = dict(_outputs(P, 16), steps=torch.full((P,), -1, dtype=torch.int32, device=DEV))
            ctx.detect_static(ctx.detect_job(H, y, nv, 4, 5, got, ci, guess=gt), prm)
            torch.cuda.synchronize()
            for k in ref:
                assert torch.equal(got[k], ref[k]), k
        assert bool((ref["steps"] < 200).any())


def test_static_scratch_rejects_a_job_larger_than_the_array():
    import paper_2510_01579_gb300 as pkg
    w = synth.uplink(63, 16, 16, 4, n_sub=300, n_sym=14)  # 4200 problems > 8 MiB of scratch
    P = w["y"].shape[0]
    with pkg.Context(0) as ctx:
        got = _outputs(P, 16)
        job = ctx.detect_job(_T(w["H"]), _T(w["y"]), _T(w["noise_var"]), 4, 1, got, _T(w["chan_index"]))
        with pytest.raises(pkg.MMGaPError) as e:
            ctx.detect_static(job, pkg.Params.default())
        assert e.value.status == 2  # MMGAP_ENOMEM
        torch.cuda.synchronize()
        assert bool((got["sym"] == 255).all())  # nothing was launched
