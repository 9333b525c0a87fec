"""Batched passes (fcm_create_batch / fcm_batch_apply): many systems with one set of
parameters stacked along the particle axis, each stage one launch over all of them.

Each system's result must equal what the oracle gives for that system alone
(element by element, the precision's bar), and the single-system CUDA path on
the same inputs. The systems have ragged sizes, one is empty, and a pass may use
fewer systems than the handle holds (an FFT bucket with unused grids).
"""
import numpy as np
import pytest

from gpu_util import FP32_TOL, FP64_TOL, System, assert_parity, ensure_built, params_for, rel_l2, suspension, torch_cuda
from paper_2310_12651_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fcm():
    torch_cuda()
    return ensure_built()


def _systems(sizes, seed, L=40.0, M=40, Sigma=1.6, tol=1e-6, torques=True):
    from oracle import params as op
    MG = op.support_points(Sigma, L / M, 4.8)
    rc = op.cutoff_radius(Sigma, tol, torques=torques)
    out = []
    for k, n in enumerate(sizes):
        out.append(System(n, L, M, Sigma, MG, rc, seed + 17 * k, torques=torques))
    return out


def _stack(torch, systems, dt):
    dev = torch.device("cuda:0")
    Y = np.concatenate([s.Y for s in systems]) if systems else np.zeros((0, 3))
    F = np.concatenate([s.F for s in systems])
    T = np.concatenate([s.T for s in systems]) if systems[0].T is not None else None
    off = np.concatenate([[0], np.cumsum([s.n for s in systems])]).astype(int).tolist()
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev) if a is not None else None
    return off, t(Y), t(F), t(T)


def _run_batch(fcm, systems, precision, max_systems=None, stages=3, handle=None):
    import torch
    dt = torch.float32 if precision == fcm.FCM_FP32 else torch.float64
    off, pos, F, T = _stack(torch, systems, dt)
    ntot = off[-1]
    U = torch.zeros((ntot, 3), dtype=dt, device="cuda:0")
    W = torch.zeros((ntot, 3), dtype=dt, device="cuda:0") if T is not None else None
    own = handle is None
    h = handle or fcm.Handle(params_for(fcm, systems[0], precision, max_n=max(ntot, 1)),
                             max_systems=max_systems or len(systems))
    try:
        h.batch_apply(off, pos, F, T, U, W, torch.cuda.current_stream().cuda_stream, stages=stages)
        assert h.check() == 0
    finally:
        if own:
            h.close()
    Un = U.double().cpu().numpy()
    Wn = W.double().cpu().numpy() if W is not None else None
    return off, Un, Wn


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_equals_each_system_alone(fcm, precision):
    from gpu_util import run_gpu
    prec = fcm.FCM_FP32 if precision == "fp32" else fcm.FCM_FP64
    tol = FP32_TOL if precision == "fp32" else FP64_TOL
    systems = _systems([700, 0, 1311, 1, 950], inputs.BASE_SEED + 60)
    off, U, W = _run_batch(fcm, systems, prec)
    for k, s in enumerate(systems):
        if s.n == 0:
            continue
        Us, Ws = U[off[k]:off[k + 1]], W[off[k]:off[k + 1]]
        Uo, Wo = s.oracle(prec)
        assert_parity(Us, Uo, tol, f"U system {k} of the batch")
        assert_parity(Ws, Wo, tol, f"W system {k} of the batch")
        Ua, Wa = run_gpu(s, prec)
        bar = 1e-6 if precision == "fp32" else 1e-13
        assert rel_l2(Us, Ua) < bar and rel_l2(Ws, Wa) < bar, (k, rel_l2(Us, Ua), rel_l2(Ws, Wa))


def test_batch_forces_only_and_each_stage(fcm):
    systems = _systems([500, 820, 333], inputs.BASE_SEED + 61, torques=False)
    for stages in (1, 2, 3):
        off, U, _ = _run_batch(fcm, systems, fcm.FCM_FP32, stages=stages)
        for k, s in enumerate(systems):
            Uo, _ = s.oracle(fcm.FCM_FP32, stages=stages)
            assert_parity(U[off[k]:off[k + 1]], Uo, FP32_TOL, f"U system {k}, stages {stages}")


def test_partial_bucket_repeated_passes_stay_exact(fcm):
    """A handle for 8 systems driven with 3, then 8, then 3 again: the bucket's unused grids
    must not leak into results over many passes. (Passes agree to rounding, not bit for bit:
    tiles add their halos into the grid with floating-point atomics in arrival order.)"""
    import torch
    systems = _systems([400, 600, 500, 450, 380, 700, 520, 610], inputs.BASE_SEED + 62)
    ntot = sum(s.n for s in systems)
    h = fcm.Handle(params_for(fcm, systems[0], fcm.FCM_FP32, max_n=ntot), max_systems=8)
    try:
        _, U3a, W3a = _run_batch(fcm, systems[:3], fcm.FCM_FP32, handle=h)
        for _ in range(12):
            _, U8, W8 = _run_batch(fcm, systems, fcm.FCM_FP32, handle=h)
            _, U3, W3 = _run_batch(fcm, systems[:3], fcm.FCM_FP32, handle=h)
        assert rel_l2(U3, U3a) < 1e-6 and rel_l2(W3, W3a) < 1e-6
        assert np.all(np.isfinite(U8)) and np.all(np.isfinite(W8))
        off = np.concatenate([[0], np.cumsum([s.n for s in systems])])
        for k in (0, 5, 7):
            Uo, Wo = systems[k].oracle(fcm.FCM_FP32)
            assert_parity(U8[off[k]:off[k + 1]], Uo, FP32_TOL, f"U system {k} of 8")
            assert_parity(W8[off[k]:off[k + 1]], Wo, FP32_TOL, f"W system {k} of 8")
    finally:
        h.close()


def test_batch_of_workload_sized_systems(fcm):
    """Four systems of 16,384 particles at 5% (the 128^3 workload's density and spacing)."""
    from oracle import params as op
    n, phi = 16384, 0.05
    L = inputs.box_edge(n, phi)
    M = 80
    Sigma = 2.0
    MG = op.support_points(Sigma, L / M, 4.8)
    rc = op.cutoff_radius(Sigma, 1e-6, torques=True)
    systems = [System(n, L, M, Sigma, MG, rc, inputs.BASE_SEED + 63 + k) for k in range(4)]
    off, U, W = _run_batch(fcm, systems, fcm.FCM_FP32)
    for k in (0, 3):
        Uo, Wo = systems[k].oracle(fcm.FCM_FP32)
        assert_parity(U[off[k]:off[k + 1]], Uo, FP32_TOL, f"U workload system {k}")
        assert_parity(W[off[k]:off[k + 1]], Wo, FP32_TOL, f"W workload system {k}")


@pytest.mark.parametrize("offsets, message", [
    ([1, 5, 9], "offsets[0]"),
    ([0, 9, 5], "nondecreasing"),
    ([0, 5, 5000], "max_n"),
    ([0, 1, 2, 3, 4, 5], "n_sys"),
])
def test_bad_offsets_are_rejected_before_any_work(fcm, offsets, message):
    import torch
    s = _systems([10], inputs.BASE_SEED + 64)[0]
    h = fcm.Handle(params_for(fcm, s, fcm.FCM_FP32, max_n=100), max_systems=4)
    try:
        z = torch.zeros((100, 3), dtype=torch.float32, device="cuda:0")
        with pytest.raises(fcm.FcmError) as e:
            h.batch_apply(offsets, z, z, z, z, z)
        assert e.value.code == fcm.FCM_ERR_ARG and message in str(e.value)
        assert h.check() == 0
    finally:
        h.close()
