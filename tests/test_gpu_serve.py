"""Serving loop (continuous batching): every job's result is the same alone
and in the mix; admission by memory; bounded waits and deadline accounting
under a host-injected stall (no GPU fault involved)."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _jobs(ctx, specs):
    out = []
    for i, (n_t, mb, n_sub, model, hold) in enumerate(specs):
        w = synth.uplink(900 + i, n_t, n_t, mb, n_sub=n_sub, n_sym=1, snr_db=14.0, model=model, hold=hold)
        t = [T(w[k]) for k in ("H", "y", "noise_var", "chan_index")]
        P = w["y"].shape[0]
        o = {"sym": torch.full((P, n_t), 255, dtype=torch.uint8, device=DEV),
             "energy": torch.full((P,), 5, dtype=torch.int32, device=DEV),
             "ndiv": torch.full((P,), -1, dtype=torch.int32, device=DEV)}
        out.append((w, t, o, ctx.detect_job(t[0], t[1], t[2], mb, 40 + i, o, t[3])))
    return out


SPECS = [(16, 4, 300, "iid", "subcarrier"), (8, 2, 1200, "kron", "prb"), (4, 6, 500, "iid", "problem"),
         (16, 6, 150, "iid", "problem"), (8, 4, 800, "iid", "subcarrier"), (4, 2, 2000, "iid", "subcarrier"),
         (16, 4, 64, "kron", "prb"), (8, 6, 333, "iid", "problem")]


@pytest.mark.parametrize("graph", [True, False])
def test_each_job_same_alone_and_in_the_mix(graph):
    import paper_2510_01579_gb300 as pkg
    prm = pkg.Params.default(steps=80)
    with pkg.Context(0) as ctx:
        jobs = _jobs(ctx, SPECS)
        refs = []
        for w, t, o, job in jobs:  # alone, through mmgap_detect
            r = {k: torch.empty_like(v) for k, v in o.items()}
            ctx.detect_jobs([ctx.detect_job(t[0], t[1], t[2], w["mod_bits"], job.seed, r, t[3])], prm)
            refs.append(r)
        torch.cuda.synchronize()
        # in the mix: all submitted at once; a budget that forces several groups per lane
        with pkg.Server(0, prm, scratch_bytes=8 << 20, n_lanes=2, max_jobs_per_group=3, use_graph=graph) as srv:
            tickets = [srv.submit(job) for _, _, _, job in jobs]
            infos = [srv.wait(tk, timeout_us=60_000_000) for tk in tickets]
            st = srv.stats()
        for (w, t, o, job), r in zip(jobs, refs):
            for k in o:
                assert torch.equal(o[k], r[k]), k
        assert st["completed"] == len(jobs) and st["groups"] >= 3 and st["max_group_jobs"] <= 3
        assert st["problems"] == sum(w["y"].shape[0] for w, _, _, _ in jobs)
        assert st["p50_us"] <= st["p99_us"] <= st["max_us"]
        assert all(i["submit_us"] <= i["start_us"] <= i["done_us"] for i in infos)


def test_admission_by_memory():
    import paper_2510_01579_gb300 as pkg
    prm = pkg.Params.default(steps=20)
    with pkg.Context(0) as ctx:
        jobs = _jobs(ctx, [(16, 4, 400, "iid", "problem")] * 4)
        # one lane with room for exactly one of these jobs at a time
        need = 400 * (32 * 32 * 2) + 3 * 256 + 400 * 96
        with pkg.Server(0, prm, scratch_bytes=need + 1024, n_lanes=1) as srv:
            tks = [srv.submit(j) for _, _, _, j in jobs]
            for tk in tks:
                srv.wait(tk)
            st = srv.stats()
            assert st["groups"] == 4 and st["max_group_jobs"] == 1
            big = _jobs(ctx, [(16, 4, 2000, "iid", "problem")])[0][3]
            with pytest.raises(pkg.MMGaPError) as e:
                srv.submit(big)
            assert e.value.status == 2  # MMGAP_ENOMEM: can never be admitted


def test_stalled_dispatcher_times_out_and_misses_deadlines():
    import paper_2510_01579_gb300 as pkg
    prm = pkg.Params.default(steps=10)
    with pkg.Context(0) as ctx:
        jobs = _jobs(ctx, [(4, 2, 100, "iid", "problem")] * 2)
        with pkg.Server(0, prm, n_lanes=1, deadline_us=1000.0, inject_delay_us=300_000.0) as srv:
            tk = srv.submit(jobs[0][3])
            with pytest.raises(pkg.MMGaPError) as e:
                srv.wait(tk, timeout_us=1000)
            assert e.value.status == 4  # MMGAP_ETIMEOUT, job still pending
            info = srv.wait(tk, timeout_us=30_000_000)
            assert info["latency_us"] >= 300_000.0
            assert srv.stats()["deadline_misses"] == 1


PRE_SPECS = [(16, 16, 4, 200, 2, 0), (8, 8, 4, 300, 1, 1), (4, 6, 2, 250, 1, 0), (16, 24, 6, 64, 3, 1),
             (8, 12, 4, 100, 2, 0)]  # (n_u, n_t, mod_bits, channels, symbols per channel, inv_precision)


def _precode_jobs(ctx, specs):
    out = []
    for i, (n_u, n_t, mb, n_sub, n_sym, ip) in enumerate(specs):
        d = synth.downlink(700 + i, n_u, n_t, mb, n_sub=n_sub, n_sym=n_sym)
        t = [T(d[k]) for k in ("H", "u_sym", "chan_index")]
        P = d["u_sym"].shape[0]
        o = {"v": torch.full((P, n_u, 2), 9, dtype=torch.int8, device=DEV),
             "x": torch.zeros((P, n_t), dtype=torch.complex64, device=DEV),
             "power": torch.full((P,), -1.0, dtype=torch.float32, device=DEV),
             "energy": torch.full((P,), 5, dtype=torch.int32, device=DEV),
             "ndiv": torch.full((P,), -1, dtype=torch.int32, device=DEV)}
        out.append((d, t, o, ip, ctx.precode_job(t[0], t[1], mb, 60 + i, o, t[2], inv_precision=ip)))
    return out


@pytest.mark.parametrize("graph", [True, False])
def test_precoding_jobs_in_the_mix_equal_mmgap_precode(graph):
    """Detection and VPP jobs of several sizes, both inverse precisions, submitted together: every
    precoding output (v, x, power, energy, divergence count) equals mmgap_precode's alone, and every
    detection output equals mmgap_detect's."""
    import paper_2510_01579_gb300 as pkg
    prm = pkg.Params.default(steps=80)
    with pkg.Context(0) as ctx:
        det = _jobs(ctx, SPECS[:4])
        pre = _precode_jobs(ctx, PRE_SPECS)
        det_ref, pre_ref = [], []
        for w, t, o, job in det:
            r = {k: torch.empty_like(v) for k, v in o.items()}
            ctx.detect_jobs([ctx.detect_job(t[0], t[1], t[2], w["mod_bits"], job.seed, r, t[3])], prm)
            det_ref.append(r)
        for d, t, o, ip, job in pre:
            pre_ref.append(ctx.precode(t[0], t[1], d["mod_bits"], prm, job.seed, chan_index=t[2], want_energy=True,
                                       want_ndiv=True, inv_precision=ip))
        torch.cuda.synchronize()
        with pkg.Server(0, prm, scratch_bytes=16 << 20, n_lanes=2, max_jobs_per_group=3, max_n_r=16,
                        use_graph=graph) as srv:
            tickets = []
            for i in range(max(len(det), len(pre))):  # interleaved arrivals
                if i < len(det):
                    tickets.append(srv.submit(det[i][3]))
                if i < len(pre):
                    tickets.append(srv.submit_precode(pre[i][4]))
            for tk in tickets:
                srv.wait(tk, timeout_us=60_000_000)
            st = srv.stats()
        for (w, t, o, job), r in zip(det, det_ref):
            for k in o:
                assert torch.equal(o[k], r[k]), k
        for (d, t, o, ip, job), r in zip(pre, pre_ref):
            for k in ("v", "x", "power", "energy", "ndiv"):
                assert torch.equal(o[k], r[k]), (k, ip)
        assert st["completed"] == len(tickets) and st["groups"] >= 3
        assert st["problems"] == sum(w["y"].shape[0] for w, _, _, _ in det) + \
            sum(d["u_sym"].shape[0] for d, _, _, _, _ in pre)


def test_server_rejects_sizes_above_its_limits():
    import paper_2510_01579_gb300 as pkg
    prm = pkg.Params.default(steps=20)
    with pkg.Context(0) as ctx:
        det = _jobs(ctx, [(16, 4, 10, "iid", "subcarrier")])
        pre = _precode_jobs(ctx, [(16, 16, 4, 10, 1, 0)])
        with pkg.Server(0, prm, scratch_bytes=8 << 20, n_lanes=1, max_n_t=8) as srv:
            with pytest.raises(pkg.MMGaPError) as e:
                srv.submit(det[0][3])
            assert e.value.status == 5
            with pytest.raises(pkg.MMGaPError) as e:
                srv.submit_precode(pre[0][4])
            assert e.value.status == 5


def test_tensor_core_server_equals_per_job_tensor_core_shape():
    """A server (and a batch) with the tensor-core refresh returns, for 8- and
    16-user jobs, exactly what mmgap_detect returns with solver shape 8 (the
    same 4-problem tcgen05 tiles), and for 4-user jobs what the exact shapes
    return."""
    import paper_2510_01579_gb300 as pkg
    prm = pkg.Params.default(steps=80)
    with pkg.Context(0) as ctx:
        jobs = _jobs(ctx, SPECS[:6])
        refs = []
        for w, t, o, job in jobs:
            n_t = w["n_t"]
            if n_t in (8, 16):
                ctx.set_solver_variant(n_t, 8)
            r = {k: torch.empty_like(v) for k, v in o.items()}
            ctx.detect_jobs([ctx.detect_job(t[0], t[1], t[2], w["mod_bits"], job.seed, r, t[3])], prm)
            ctx.set_solver_variant(n_t, 0)
            refs.append(r)
        torch.cuda.synchronize()
        with pkg.Server(0, prm, scratch_bytes=16 << 20, n_lanes=2, max_jobs_per_group=3, tensor_core=True) as srv:
            for tk in [srv.submit(job) for _, _, _, job in jobs]:
                srv.wait(tk, timeout_us=60_000_000)
        for (w, t, o, job), r in zip(jobs, refs):
            for k in o:
                assert torch.equal(o[k], r[k]), (w["n_t"], k)
        # the batch object with the same flag
        for (w, t, o, job), r in zip(jobs, refs):
            for v in o.values():
                v.fill_(0)
        with pkg.Batch(0, prm, [j for _, _, _, j in jobs], keepalive=jobs, tensor_core=True) as b:
            b.run(use_graph=True)
            torch.cuda.synchronize()
        for (w, t, o, job), r in zip(jobs, refs):
            for k in o:
                assert torch.equal(o[k], r[k]), (w["n_t"], k)


def test_server_with_32_user_jobs():
    """A server sized for 32 users: 32x32 jobs grouped with smaller ones equal
    their mmgap_detect results bit for bit."""
    import paper_2510_01579_gb300 as pkg
    prm = pkg.Params.default(steps=60)
    specs = [(32, 4, 40, "iid", "subcarrier"), (16, 4, 200, "iid", "subcarrier"), (32, 2, 25, "iid", "problem"),
             (8, 2, 300, "kron", "prb")]
    with pkg.Context(0) as ctx:
        jobs = _jobs(ctx, specs)
        refs = []
        for w, t, o, job in jobs:
            r = {k: torch.empty_like(v) for k, v in o.items()}
            ctx.detect_jobs([ctx.detect_job(t[0], t[1], t[2], w["mod_bits"], job.seed, r, t[3])], prm)
            refs.append(r)
        torch.cuda.synchronize()
        with pkg.Server(0, prm, scratch_bytes=8 << 20, n_lanes=2, max_jobs_per_group=2, max_n_t=32,
                        max_n_r=32) as srv:
            tickets = [srv.submit(job) for _, _, _, job in jobs]
            for tk in tickets:
                srv.wait(tk, timeout_us=60_000_000)
            st = srv.stats()
        for (w, t, o, job), r in zip(jobs, refs):
            for k in o:
                assert torch.equal(o[k], r[k]), (w["n_t"], k)
        assert st["completed"] == len(jobs)
