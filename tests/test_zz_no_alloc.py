"""The pair correction through the entry point that allocates no device memory.

Callers that cannot allocate device memory (code whose memory pool owns the
whole device, so that a cudaMalloc beside it fails or fragments the pool, and
hosts that allocate everything at start-up and forbid cudaMalloc afterwards)
call fcm_pair_correction_noalloc, which keeps all its scratch in one fixed
device array. Its result must match the pair stage of
the handle-based entry point (fcm_apply_stages with FCM_STAGE_PAIR) within the
FP32 tolerance of the parity tests, on two calls in a row with different loads
(so a second call cannot pass on what the first left behind). The file is
named so that pytest collects it last.
"""
import numpy as np
import pytest

from gpu_util import FP32_TOL, assert_parity, ensure_built, suspension, torch_cuda
from paper_2310_12651_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_noalloc_pair_correction_matches_handle_path_twice():
    torch = torch_cuda()
    fcm = ensure_built()
    s = suspension(20000, 0.05, 64, 2.0, 1e-6, 71)
    p = fcm.make_params(s.L, s.M, s.Sigma, s.r_c, s.M_G, s.n, fcm.FCM_FP32)
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    pos = torch.as_tensor(s.Y, dtype=torch.float32, device=dev)
    loads = [inputs.random_loads(s.n, 72), inputs.random_loads(s.n, 73)]
    with fcm.Handle(p) as h:
        for k, (F, T) in enumerate(loads):
            Ft = torch.as_tensor(F, dtype=torch.float32, device=dev)
            Tt = torch.as_tensor(T, dtype=torch.float32, device=dev)
            Uh, Wh = (torch.empty_like(Ft) for _ in range(2))
            h.apply_stages(s.n, pos, Ft, Tt, Uh, Wh, fcm.STAGE_PAIR, stream)
            Un = torch.full_like(Ft, float("nan"))
            Wn = torch.full_like(Ft, float("nan"))
            fcm.pair_correction_noalloc(p, s.n, pos, Ft, Tt, Un, Wn, stream)
            torch.cuda.synchronize()
            for got, ref, name in ((Un, Uh, "U"), (Wn, Wh, "W")):
                g, r = got.double().cpu().numpy(), ref.double().cpu().numpy()
                assert np.all(np.isfinite(g))
                assert_parity(g, r, FP32_TOL, f"{name} no-alloc call {k + 1}")


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
