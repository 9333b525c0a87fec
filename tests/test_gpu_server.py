"""The serving engine (fcm_server_*): continuous batching per grid class, HBM admission,
bounded waits, cancellation, passes replayed from captured CUDA graphs.

The central check is "alone = in the mix": every request served in a mixed
stream (several grid classes, uneven sizes, submitted from several threads so
that same-class requests share passes) equals fcm_apply on that system alone,
and the oracle for a sample of them.
"""
import threading

import numpy as np
import pytest

from gpu_util import FP32_TOL, System, assert_parity, ensure_built, params_for, rel_l2, run_gpu, torch_cuda
from oracle import params as op
from paper_2310_12651_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fcm():
    torch_cuda()
    return ensure_built()


def _class(L, M, Sigma, tol=1e-6):
    MG = op.support_points(Sigma, L / M, 4.8)
    rc = op.cutoff_radius(Sigma, tol, torques=True)
    return dict(L=L, M=M, Sigma=Sigma, MG=MG, rc=rc)


CLASSES = [_class(40.0, 40, 1.6), _class(60.0, 48, 2.0), _class(32.0, 32, 1.5)]


def _request(k, seed):
    c = CLASSES[k % len(CLASSES)]
    rng = np.random.default_rng(seed)
    n = int(rng.integers(50, 1500))
    return System(n, c["L"], c["M"], c["Sigma"], c["MG"], c["rc"], seed)


def test_alone_equals_in_the_mix(fcm):
    systems = [_request(k, inputs.BASE_SEED + 300 + k) for k in range(36)]
    with fcm.Server(hbm_budget=4 << 30, max_batch=16) as srv:
        tickets = [None] * len(systems)

        def client(ids):
            for i in ids:
                s = systems[i]
                tickets[i] = srv.submit(params_for(fcm, s, fcm.FCM_FP32), s.Y, s.F, s.T)

        threads = [threading.Thread(target=client, args=(range(t, len(systems), 4),)) for t in range(4)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        for t in tickets:
            assert srv.wait(t, 60.0) and t.status == fcm.FCM_OK
        st = srv.stats()
    assert st["completed"] == len(systems) and st["failed"] == 0 and st["rejected"] == 0
    assert st["batches"] < len(systems), st     # same-class requests shared passes
    assert st["graph_passes"] == st["batches"], st   # every FP32 pass replayed a captured graph
    assert st["latency_p99_us"] >= st["latency_p50_us"] > 0
    for i, s in enumerate(systems):
        Ua, Wa = run_gpu(s, fcm.FCM_FP32)
        assert rel_l2(tickets[i].U.astype(np.float64), Ua) < 1e-6, i
        assert rel_l2(tickets[i].W.astype(np.float64), Wa) < 1e-6, i
    for i in (0, 1, 2, 35):
        Uo, Wo = systems[i].oracle(fcm.FCM_FP32)
        assert_parity(tickets[i].U.astype(np.float64), Uo, FP32_TOL, f"U request {i} in the mix")
        assert_parity(tickets[i].W.astype(np.float64), Wo, FP32_TOL, f"W request {i} in the mix")


def test_forces_only_and_fp64_requests(fcm):
    s32 = _request(0, inputs.BASE_SEED + 350)
    s64 = _request(1, inputs.BASE_SEED + 351)
    with fcm.Server(hbm_budget=2 << 30) as srv:
        a = srv.submit(params_for(fcm, s32, fcm.FCM_FP32), s32.Y, s32.F, None, want_W=False)
        b = srv.submit(params_for(fcm, s64, fcm.FCM_FP64), s64.Y, s64.F, s64.T)
        c = srv.submit(params_for(fcm, s64, fcm.FCM_FP64), s64.Y[:0], s64.F[:0], s64.T[:0])
        for t in (a, b, c):
            assert srv.wait(t, 60.0) and t.status == fcm.FCM_OK
    assert a.W is None and c.U.shape == (0, 3)
    s32.T = None
    Ua, _ = run_gpu(s32, fcm.FCM_FP32, want_W=False)
    assert rel_l2(a.U.astype(np.float64), Ua) < 1e-6
    Ub, Wb = s64.oracle(fcm.FCM_FP64)
    assert_parity(b.U, Ub, 1e-10, "U fp64 request")
    assert_parity(b.W, Wb, 1e-10, "W fp64 request")


def test_budget_evicts_idle_handles_and_rejects_oversize(fcm):
    """Two 128^3 classes whose handles (about 52 MB each: grid, spectrum, FFT work) do not fit an
    80 MB budget together, and a 320^3 class that does not fit at all."""
    ca, cb = _class(176.0, 128, 2.0), _class(170.0, 128, 2.0)
    small = [System(500, c["L"], c["M"], c["Sigma"], c["MG"], c["rc"], inputs.BASE_SEED + 360 + k)
             for k, c in enumerate((ca, cb))]
    big = _class(400.0, 320, 2.0)
    huge = System(100, big["L"], big["M"], big["Sigma"], big["MG"], big["rc"], inputs.BASE_SEED + 362)
    with fcm.Server(hbm_budget=80 << 20, max_batch=4) as srv:
        t = srv.submit(params_for(fcm, huge, fcm.FCM_FP32), huge.Y, huge.F, huge.T)
        assert srv.wait(t, 60.0) and t.status == fcm.FCM_ERR_OOM
        results = []
        for rep in range(3):              # alternate classes: each new handle evicts the other
            for s in small:
                tk = srv.submit(params_for(fcm, s, fcm.FCM_FP32), s.Y, s.F, s.T)
                assert srv.wait(tk, 60.0) and tk.status == fcm.FCM_OK
                results.append((s, tk))
        st = srv.stats()
    assert st["rejected"] == 1 and st["hbm_bytes"] <= st["hbm_budget"]
    assert st["graph_passes"] == st["batches"]        # graphs are re-captured after each eviction
    assert st["handles_evicted"] >= 4 and st["handles_created"] >= 6, st
    for s, tk in results[:2]:
        Ua, Wa = run_gpu(s, fcm.FCM_FP32)
        assert rel_l2(tk.U.astype(np.float64), Ua) < 1e-6 and rel_l2(tk.W.astype(np.float64), Wa) < 1e-6


def test_invalid_request_is_rejected_at_submit(fcm):
    s = _request(0, inputs.BASE_SEED + 370)
    with fcm.Server(hbm_budget=1 << 30) as srv:
        p = params_for(fcm, s, fcm.FCM_FP32)
        p.r_c = 0.9 * s.L
        with pytest.raises(fcm.FcmError) as e:
            srv.submit(p, s.Y, s.F, s.T)
        assert e.value.code == fcm.FCM_ERR_ARG and "r_c" in str(e.value)
        assert srv.stats()["rejected"] == 1


def test_poll_timeout_and_cancel(fcm):
    c = _class(176.41391792668995, 128, 2.0)
    systems = [System(65536, c["L"], c["M"], c["Sigma"], c["MG"], c["rc"], inputs.BASE_SEED + 380 + k)
               for k in range(2)]
    arrays = [tuple(np.ascontiguousarray(a, dtype=np.float32) for a in (s.Y, s.F, s.T)) for s in systems]
    with fcm.Server(hbm_budget=8 << 30, max_batch=1) as srv:
        # the first request creates the class's handle (allocation and FFT plans), so the rest queue
        tickets = [srv.submit(params_for(fcm, systems[k % 2], fcm.FCM_FP32), *arrays[k % 2]) for k in range(12)]
        assert srv.wait(tickets[0], 0.0) is False       # a 65,536-particle pass is not done at once
        canceled = srv.cancel(tickets[-1])              # the last of 12 one-system passes is still queued
        for t in tickets:
            assert srv.wait(t, 60.0)
        assert tickets[-1].status == (fcm.FCM_ERR_CANCELED if canceled else fcm.FCM_OK)
        assert canceled
        assert all(t.status == fcm.FCM_OK for t in tickets[:-1])
        with pytest.raises(fcm.FcmError):
            srv.cancel(tickets[0])                      # already forgotten after its wait
    Ua, Wa = run_gpu(systems[1], fcm.FCM_FP32)
    assert rel_l2(tickets[1].U.astype(np.float64), Ua) < 1e-6


def test_destroy_with_queued_requests_returns(fcm):
    c = _class(176.41391792668995, 128, 2.0)
    s = System(65536, c["L"], c["M"], c["Sigma"], c["MG"], c["rc"], inputs.BASE_SEED + 390)
    srv = fcm.Server(hbm_budget=8 << 30, max_batch=1)
    keep = [srv.submit(params_for(fcm, s, fcm.FCM_FP32), s.Y, s.F, s.T) for _ in range(6)]
    srv.close()   # cancels what is queued, waits for what runs
    assert len(keep) == 6
