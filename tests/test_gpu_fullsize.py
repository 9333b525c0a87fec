"""Full-size checks of the CUDA path in the launch configuration bench.py times.

* The 128^3 workload (N = 65,536, phi = 5%, Sigma = 2a, M_G = 14, r_c from the
  1e-6 rule, forces + torques, FP32) against the full FP64 oracle, element by
  element.
* The N = 1,048,576, phi = 10%, 256^3 workload, too large for the full oracle:
  the FP32 path against the FP64 plain path on the same GPU (itself held to
  1e-10 against the oracle at smaller sizes), the pair stage on sampled
  particles against the oracle computed one particle at a time, and the
  symmetry of the discrete operator.
"""
import numpy as np
import pytest

from gpu_util import FP32_TOL, System, assert_parity, ensure_built, rel_l2, rounded, run_gpu, torch_cuda
from oracle import grid_fcm as og
from oracle import params as op
from paper_2310_12651_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def fcm():
    torch_cuda()
    return ensure_built()


def _workload(n, phi, M, Sigma, seed):
    L = inputs.box_edge(n, phi)
    MG = op.support_points(Sigma, L / M, 4.8)
    rc = op.cutoff_radius(Sigma, 1e-6, torques=True)
    return System(n, L, M, Sigma, MG, rc, seed)


def test_bench_workload_full_size_against_oracle(fcm):
    s = _workload(65536, 0.05, 128, 2.0, inputs.BASE_SEED + 1)
    assert s.M_G == 14
    U, W = run_gpu(s, fcm.FCM_FP32)
    Uo, Wo = s.oracle(fcm.FCM_FP32)
    assert_parity(U, Uo, FP32_TOL, "U 128^3 full size")
    assert_parity(W, Wo, FP32_TOL, "W 128^3 full size")


@pytest.fixture(scope="module")
def large(fcm):
    return _workload(1048576, 0.10, 256, 1.5, inputs.BASE_SEED + 3)


def test_large_fp32_matches_fp64_plain(fcm, large):
    U32, W32 = run_gpu(large, fcm.FCM_FP32)
    U64, W64 = run_gpu(large, fcm.FCM_FP64)
    assert_parity(U32, U64, FP32_TOL, "U 1M fp32 vs fp64")
    assert_parity(W32, W64, FP32_TOL, "W 1M fp32 vs fp64")


def test_large_pair_stage_on_sampled_particles(fcm, large):
    U, W = run_gpu(large, fcm.FCM_FP32, stages=fcm.STAGE_PAIR)
    idx = np.random.default_rng(74).choice(large.n, 300, replace=False)
    Y, F, T = (rounded(a, fcm.FCM_FP32) for a in (large.Y, large.F, large.T))
    Uo, Wo = og.pair_correction_subset(Y, F, T, large.L, large.r_c, large.Sigma, large.Sigma, idx)
    assert_parity(U[idx], Uo, FP32_TOL, "U 1M pair stage, sampled")
    assert_parity(W[idx], Wo, FP32_TOL, "W 1M pair stage, sampled")


def test_large_operator_symmetry(fcm, large):
    U1, W1 = run_gpu(large, fcm.FCM_FP32)
    F1, T1 = large.F.copy(), large.T.copy()
    large.F, large.T = inputs.random_loads(large.n, 75)
    try:
        U2, W2 = run_gpu(large, fcm.FCM_FP32)
        a = np.sum(F1 * U2) + np.sum(T1 * W2)
        b = np.sum(large.F * U1) + np.sum(large.T * W1)
    finally:
        large.F, large.T = F1, T1
    assert abs(a - b) < 1e-5 * (abs(a) + abs(b)), (a, b)
