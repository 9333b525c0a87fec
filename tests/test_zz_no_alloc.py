"""The pair correction through the entry point that allocates no device memory.

Callers that cannot allocate device memory (code whose memory pool owns the
whole device, so that a cudaMalloc beside it fails or fragments the pool, and
hosts that allocate everything at start-up and forbid cudaMalloc afterwards)
call fcm_pair_correction_noalloc, which keeps all its scratch in one fixed
device array. Its result must match the pair stage of the handle-based entry
point (fcm_apply_stages with FCM_STAGE_PAIR) and the FP64 oracle's pair
correction within the FP32 tolerance of the parity tests, on two calls in a row
with different loads (so a second call cannot pass on what the first left
behind). Further cases: forces only (T and W NULL), a box of three pair cells
per side (the unshifted cell sweep), and that calls after the first one take no
device memory. The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from gpu_util import FP32_TOL, System, assert_parity, ensure_built, rounded, suspension, torch_cuda
from oracle import grid_fcm as og
from paper_2310_12651_gb300 import inputs

pytestmark = pytest.mark.gpu


def _oracle_pair(s, F, T, fcm):
    Y, F, T = (rounded(x, fcm.FCM_FP32) for x in (s.Y, F, T))
    return og.pair_correction(Y, F, T, s.L, s.r_c, s.Sigma, s.Sigma)


def _both(fcm, torch, s, F, T, h, stream):
    """Handle path and no-alloc path on the same inputs; returns numpy (Uh, Wh, Un, Wn)."""
    dev = torch.device("cuda:0")
    p = fcm.make_params(s.L, s.M, s.Sigma, s.r_c, s.M_G, s.n, fcm.FCM_FP32)
    pos = torch.as_tensor(s.Y, dtype=torch.float32, device=dev)
    Ft = torch.as_tensor(F, dtype=torch.float32, device=dev)
    Tt = torch.as_tensor(T, dtype=torch.float32, device=dev) if T is not None else None
    Uh = torch.empty_like(Ft)
    Wh = torch.empty_like(Ft) if T is not None else None
    h.apply_stages(s.n, pos, Ft, Tt, Uh, Wh, fcm.STAGE_PAIR, stream)
    Un = torch.full_like(Ft, float("nan"))
    Wn = torch.full_like(Ft, float("nan")) if T is not None else None
    fcm.pair_correction_noalloc(p, s.n, pos, Ft, Tt, Un, Wn, stream)
    torch.cuda.synchronize()
    out = [Uh, Wh, Un, Wn]
    return [x.double().cpu().numpy() if x is not None else None for x in out]


def test_noalloc_pair_correction_matches_handle_path_and_oracle_twice():
    torch = torch_cuda()
    fcm = ensure_built()
    s = suspension(20000, 0.05, 64, 2.0, 1e-6, 71)
    p = fcm.make_params(s.L, s.M, s.Sigma, s.r_c, s.M_G, s.n, fcm.FCM_FP32)
    stream = torch.cuda.current_stream().cuda_stream
    loads = [inputs.random_loads(s.n, 72), inputs.random_loads(s.n, 73)]
    with fcm.Handle(p) as h:
        for k, (F, T) in enumerate(loads):
            Uh, Wh, Un, Wn = _both(fcm, torch, s, F, T, h, stream)
            for got, ref, name in ((Un, Uh, "U"), (Wn, Wh, "W")):
                assert np.all(np.isfinite(got))
                assert_parity(got, ref, FP32_TOL, f"{name} no-alloc call {k + 1} vs handle path")
            Uo, Wo = _oracle_pair(s, F, T, fcm)
            assert_parity(Un, Uo, FP32_TOL, f"U no-alloc call {k + 1} vs oracle")
            assert_parity(Wn, Wo, FP32_TOL, f"W no-alloc call {k + 1} vs oracle")


def test_noalloc_forces_only_and_three_cells_per_side():
    """T = W = NULL (forces-only kernels), and a box under 4 r_c per side (3 pair cells, unshifted sweep)."""
    torch = torch_cuda()
    fcm = ensure_built()
    stream = torch.cuda.current_stream().cuda_stream
    big = suspension(8000, 0.05, 48, 2.0, 1e-6, 81, torques=False)
    L = 40.0
    Y = inputs.random_suspension(600, L, 83, min_sep=2.2)
    small = System(600, L, 32, 2.0, 12, 14.3, 84, Y=Y)
    assert max(int(small.L / small.r_c), 3) == 3   # 3 pair cells per side: every cell neighbours every cell
    for s, T in ((big, None), (small, small.T), (small, None)):
        p = fcm.make_params(s.L, s.M, s.Sigma, s.r_c, s.M_G, s.n, fcm.FCM_FP32)
        with fcm.Handle(p) as h:
            Uh, Wh, Un, Wn = _both(fcm, torch, s, s.F, T, h, stream)
        assert np.all(np.isfinite(Un))
        assert_parity(Un, Uh, FP32_TOL, f"U no-alloc n={s.n} torques={T is not None} vs handle path")
        Uo, Wo = _oracle_pair(s, s.F, T, fcm)
        assert_parity(Un, Uo, FP32_TOL, f"U no-alloc n={s.n} torques={T is not None} vs oracle")
        if T is not None:
            assert_parity(Wn, Wh, FP32_TOL, "W no-alloc vs handle path")
            assert_parity(Wn, Wo, FP32_TOL, "W no-alloc vs oracle")


def test_noalloc_calls_take_no_device_memory():
    """After a first call (which, with lazy module loading, reserves the fixed array), further calls
    leave the device's free memory and torch's allocator unchanged."""
    torch = torch_cuda()
    fcm = ensure_built()
    s = suspension(20000, 0.05, 64, 2.0, 1e-6, 91)
    p = fcm.make_params(s.L, s.M, s.Sigma, s.r_c, s.M_G, s.n, fcm.FCM_FP32)
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    pos = torch.as_tensor(s.Y, dtype=torch.float32, device=dev)
    Ft = torch.as_tensor(s.F, dtype=torch.float32, device=dev)
    Tt = torch.as_tensor(s.T, dtype=torch.float32, device=dev)
    U, W = torch.empty_like(Ft), torch.empty_like(Ft)
    fcm.pair_correction_noalloc(p, s.n, pos, Ft, Tt, U, W, stream)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        fcm.pair_correction_noalloc(p, s.n, pos, Ft, Tt, U, W, stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == alloc0
    # any device allocation is at least a 2 MiB page; the scratch alone is 7.7 MB
    assert free0 - free1 < (1 << 20), (free0, free1)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    fcm = ensure_built()
    p = fcm.make_params(100.0, 64, 2.0, 14.0, 12, 10, fcm.FCM_FP32)
    with pytest.raises(fcm.FcmError) as e:
        fcm.pair_correction_noalloc(p, fcm.NOALLOC_MAX_N + 1, 0, 0, 0, 0, 0)
    assert e.value.code == fcm.FCM_ERR_ARG and "scratch" in str(e.value)
    p2 = fcm.make_params(1000.0, 64, 2.0, 10.0, 12, 10, fcm.FCM_FP32)  # 100^3 pair cells
    with pytest.raises(fcm.FcmError) as e:
        fcm.pair_correction_noalloc(p2, 10, 0, 0, 0, 0, 0)
    assert e.value.code == fcm.FCM_ERR_ARG and "cells" in str(e.value)
