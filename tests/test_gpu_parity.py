"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle, element by element.

FP64 plain path: relative L2 <= 1e-10 (same discretisation, FP64 throughout).
FP32 path: relative L2 <= 1e-4, the bar of the precision policy; the measured
errors (printed) are near 1e-6. Every element is also held to 10x the bar
relative to the rms of the reference.
"""
import math

import numpy as np
import pytest

from gpu_util import (FP32_TOL, FP64_TOL, SIGMA, SIGMA_D, System, assert_parity, ensure_built, rounded, run_gpu,
                      suspension, torch_cuda)
from oracle import grid_fcm as og
from oracle import params as op
from paper_2310_12651_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fcm():
    torch_cuda()
    return ensure_built()


# ---------------------------------------------------------------- small config (FP64 plain)

def test_fp64_forces_only_small_config(fcm):
    """N = 1000, L = 100a, 64^3, Sigma = 2a, window +-4 Sigma, r_c from the 1e-8 rule, forces only."""
    L, M, Sigma = 100.0, 64, 2.0
    MG = op.support_points(Sigma, L / M, 4.0)
    rc = op.cutoff_radius(Sigma, 1e-8)
    s = System(1000, L, M, Sigma, MG, rc, inputs.BASE_SEED + 0, torques=False)
    U, _ = run_gpu(s, fcm.FCM_FP64, want_W=False)
    Uo, _ = s.oracle(fcm.FCM_FP64)
    assert_parity(U, Uo, FP64_TOL, "U fp64 small config")


@pytest.mark.parametrize("Sigma", [1.5, 2.0])
def test_fp64_torques(fcm, Sigma):
    s = suspension(1500, 0.05, 36, Sigma, 1e-6, 41)
    U, W = run_gpu(s, fcm.FCM_FP64)
    Uo, Wo = s.oracle(fcm.FCM_FP64)
    assert_parity(U, Uo, FP64_TOL, "U fp64")
    assert_parity(W, Wo, FP64_TOL, "W fp64")


# ---------------------------------------------------------------- FP32 path

@pytest.mark.parametrize("Sigma, M", [(1.5, 48), (2.0, 44), (3.0, 48)])
def test_fp32_torques_several_tiles(fcm, Sigma, M):
    """5% suspension, grid spacing near the 128^3 workload's; M = 44 leaves a ragged last tile."""
    s = suspension(6000, 0.05, M, Sigma, 1e-6, 43)
    U, W = run_gpu(s, fcm.FCM_FP32)
    Uo, Wo = s.oracle(fcm.FCM_FP32)
    assert_parity(U, Uo, FP32_TOL, f"U fp32 Sigma={Sigma}")
    assert_parity(W, Wo, FP32_TOL, f"W fp32 Sigma={Sigma}")


@pytest.mark.parametrize("kernel", [0, 1, 2, 4])
def test_fp32_both_spread_kernels(fcm, kernel):
    """Pencil (0, the default), row-stationary per tile pair (1) and shared-atomic (2) spread kernels give
    the same product."""
    torch = torch_cuda()
    s = suspension(5000, 0.05, 48, 2.0, 1e-6, 66)
    p = fcm.make_params(s.L, s.M, s.Sigma, s.r_c, s.M_G, s.n, fcm.FCM_FP32, spread_kernel=kernel)
    with fcm.Handle(p) as h:
        U, W = run_gpu(s, fcm.FCM_FP32, handle=h)
    Uo, Wo = s.oracle(fcm.FCM_FP32)
    assert_parity(U, Uo, FP32_TOL, f"U spread kernel {kernel}")
    assert_parity(W, Wo, FP32_TOL, f"W spread kernel {kernel}")


def test_fp32_forces_only(fcm):
    s = suspension(4000, 0.05, 40, 2.0, 1e-6, 44, torques=False)
    U, _ = run_gpu(s, fcm.FCM_FP32, want_W=False)
    Uo, _ = s.oracle(fcm.FCM_FP32)
    assert_parity(U, Uo, FP32_TOL, "U fp32 forces only")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("stages", [1, 2])
def test_each_stage_alone(fcm, precision, stages):
    """The grid part (M~) and the pair part (M - M~) each match the oracle on their own."""
    prec = fcm.FCM_FP32 if precision == "fp32" else fcm.FCM_FP64
    s = suspension(3000, 0.08, 32, 1.6, 1e-6, 45)
    U, W = run_gpu(s, prec, stages=stages)
    Uo, Wo = s.oracle(prec, stages=stages)
    tol = FP32_TOL if precision == "fp32" else FP64_TOL
    assert_parity(U, Uo, tol, f"U stage {stages} {precision}")
    assert_parity(W, Wo, tol, f"W stage {stages} {precision}")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_spread_grid_matches_oracle(fcm, precision):
    """The spread force density itself, point by point (layout [c][z][y][x])."""
    torch = torch_cuda()
    prec = fcm.FCM_FP32 if precision == "fp32" else fcm.FCM_FP64
    s = suspension(2000, 0.05, 40, 2.0, 1e-6, 46)
    dt = torch.float32 if precision == "fp32" else torch.float64
    with fcm.Handle(fcm.make_params(s.L, s.M, s.Sigma, s.r_c, s.M_G, s.n, prec)) as h:
        pos = torch.as_tensor(s.Y, dtype=dt, device="cuda")
        F = torch.as_tensor(s.F, dtype=dt, device="cuda")
        T = torch.as_tensor(s.T, dtype=dt, device="cuda")
        h.spread(s.n, pos, F, T, torch.cuda.current_stream().cuda_stream)
        grid = torch.empty(3 * s.M ** 3, dtype=dt, device="cuda")
        h.copy_grid(grid, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
    got = grid.double().cpu().numpy().reshape(3, s.M, s.M, s.M).transpose(0, 3, 2, 1)  # -> [c][x][y][z]
    ref = og.spread(rounded(s.Y, prec), rounded(s.F, prec), rounded(s.T, prec), s.L, s.M, s.M_G, s.Sigma, s.Sigma)
    assert_parity(got, ref, FP32_TOL if precision == "fp32" else FP64_TOL, f"spread grid {precision}")


@pytest.mark.parametrize("kernel", [0, 4])
@pytest.mark.parametrize("M, Sigma, c_trunc, torques, sigma_d", [
    (42, 2.0, 4.7, True, 0.0),     # M_G = 14, M_x not a multiple of 4: scalar flushes; ragged last tile of 2 points
    (44, 1.5, 4.8, True, 0.0),     # M_G = 12, ragged last tile of 4 points
    (40, 2.0, 4.0, False, 0.0),    # forces only, M_G = 12
    (36, 2.0, 5.2, True, 0.0),     # M_G = 16: (8, 4, 4) tiles
    (32, 1.2, 4.8, True, 1.5),     # Sigma_D != Sigma, M_G = 10 at h = 1.1
    (16, 2.0, 4.8, True, 0.0),     # M_G = 14: the extended row (21 points) wraps past M_x = 16
])
def test_pencil_spread_grid_matches_oracle(fcm, M, Sigma, c_trunc, torques, sigma_d, kernel):
    """The pencil spreads' force density point by point (0: register rows, 4: tensor cores, which falls back
    to 0 for M_G = 16 and Sigma_D != Sigma): ragged and wrapping rows, the M_G variants, forces only and a
    torque width different from Sigma."""
    torch = torch_cuda()
    n = max(200, int(0.05 * (M * 1.37) ** 3 / 4.19))
    s = suspension(n, 0.05, M, Sigma, 1e-6, 460 + M, torques=torques, c_trunc=c_trunc)
    s.Sigma_D = sigma_d
    SD = sigma_d if sigma_d else Sigma
    p = fcm.make_params(s.L, s.M, s.Sigma, s.r_c, s.M_G, s.n, fcm.FCM_FP32, Sigma_D=sigma_d, spread_kernel=kernel)
    with fcm.Handle(p) as h:
        pos = torch.as_tensor(s.Y, dtype=torch.float32, device="cuda")
        F = torch.as_tensor(s.F, dtype=torch.float32, device="cuda")
        T = torch.as_tensor(s.T, dtype=torch.float32, device="cuda") if torques else None
        h.spread(s.n, pos, F, T, torch.cuda.current_stream().cuda_stream)
        grid = torch.empty(3 * s.M ** 3, dtype=torch.float32, device="cuda")
        h.copy_grid(grid, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
    got = grid.double().cpu().numpy().reshape(3, s.M, s.M, s.M).transpose(0, 3, 2, 1)
    T64 = rounded(s.T, fcm.FCM_FP32) if torques else None
    ref = og.spread(rounded(s.Y, fcm.FCM_FP32), rounded(s.F, fcm.FCM_FP32), T64, s.L, s.M, s.M_G, s.Sigma, SD,
                    fp32_windows=True)
    assert_parity(got, ref, FP32_TOL, f"pencil spread grid M={M} M_G={s.M_G}")


# ---------------------------------------------------------------- edge cases and degenerate cases

def test_empty_input_is_a_no_op(fcm):
    torch = torch_cuda()
    s = suspension(100, 0.05, 16, 1.2, 1e-4, 47)
    with fcm.Handle(fcm.make_params(s.L, s.M, s.Sigma, s.r_c, s.M_G, 100, fcm.FCM_FP32)) as h:
        z = torch.zeros((0, 3), device="cuda")
        h.apply(0, z, z, z, z, z)
        assert h.check() == 0


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_single_particle(fcm, precision):
    prec = fcm.FCM_FP32 if precision == "fp32" else fcm.FCM_FP64
    s = System(1, 30.0, 24, 1.5, 10, 10.0, 48, Y=np.array([[3.3, 29.9, 0.01]]))
    s.F, s.T = np.array([[0.3, -1.1, 0.7]]), np.array([[0.2, 0.5, -0.9]])
    U, W = run_gpu(s, prec)
    Uo, Wo = s.oracle(prec)
    tol = FP32_TOL if precision == "fp32" else FP64_TOL
    assert_parity(U, Uo, tol, "U single")
    assert_parity(W, Wo, tol, "W single")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_positions_outside_the_box_are_wrapped(fcm, precision):
    prec = fcm.FCM_FP32 if precision == "fp32" else fcm.FCM_FP64
    s = suspension(800, 0.05, 24, 1.5, 1e-6, 49)
    shift = np.random.default_rng(50).integers(-3, 4, size=s.Y.shape) * s.L
    U0, W0 = run_gpu(s, prec)
    U1, W1 = run_gpu(s, prec, Y=s.Y + shift)
    tol = 1e-5 if precision == "fp32" else 1e-11
    assert_parity(U1, U0, tol, "U shifted")
    assert_parity(W1, W0, tol, "W shifted")


def test_standard_fcm_mode(fcm):
    """Sigma = sigma, Sigma_D = sigma_D: standard FCM, no correction (Section 5, Sigma/sigma = 1)."""
    L = 16.0
    M = 40
    s = System(60, L, M, SIGMA, 16, 1.0, 51, Sigma_D=SIGMA_D)
    U, W = run_gpu(s, fcm.FCM_FP64)
    Uo, Wo = og.standard_fcm_apply(s.Y, s.F, s.T, L, M, 16)
    assert_parity(U, Uo, FP64_TOL, "U standard")
    assert_parity(W, Wo, FP64_TOL, "W standard")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_separate_torque_width(fcm, precision):
    prec = fcm.FCM_FP32 if precision == "fp32" else fcm.FCM_FP64
    L = inputs.box_edge(1200, 0.05)
    s = System(1200, L, 32, 2.0, 14, min(op.cutoff_radius(2.0, 1e-6, Sigma_D=1.4, torques=True), L / 2), 52,
               Sigma_D=1.4)
    U, W = run_gpu(s, prec)
    Uo, Wo = s.oracle(prec)
    tol = FP32_TOL if precision == "fp32" else FP64_TOL
    assert_parity(U, Uo, tol, "U Sigma_D")
    assert_parity(W, Wo, tol, "W Sigma_D")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_anisotropic_box_and_grid(fcm, precision):
    """L_x != L_y != L_z, odd and even M per dimension (Section 2.1 allows both)."""
    prec = fcm.FCM_FP32 if precision == "fp32" else fcm.FCM_FP64
    L = (40.0, 32.0, 24.0)
    s = System(700, L, (45, 36, 28), 1.4, 12, 10.0, 53, min_sep=0.0)
    U, W = run_gpu(s, prec)
    Uo, Wo = s.oracle(prec)
    tol = FP32_TOL if precision == "fp32" else FP64_TOL
    assert_parity(U, Uo, tol, "U aniso")
    assert_parity(W, Wo, tol, "W aniso")


def test_tiny_grid_window_wraps_onto_itself(fcm):
    """M = 16 with M_G = 14: the extended tile region wraps around the grid."""
    s = System(200, 20.0, 16, 1.6, 14, 8.0, 54, min_sep=1.0)
    for prec, tol in ((fcm.FCM_FP32, FP32_TOL), (fcm.FCM_FP64, FP64_TOL)):
        U, W = run_gpu(s, prec)
        Uo, Wo = s.oracle(prec)
        assert_parity(U, Uo, tol, "U tiny grid")
        assert_parity(W, Wo, tol, "W tiny grid")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_overlapping_pairs_use_the_small_r_branch(fcm, precision):
    """Pairs at r in [0.02, 0.5 sigma] go through the Taylor branch; the oracle uses the closed form."""
    prec = fcm.FCM_FP32 if precision == "fp32" else fcm.FCM_FP64
    rng = np.random.default_rng(55)
    L = 24.0
    base = inputs.random_suspension(150, L, 56, min_sep=3.0)
    d = rng.normal(size=(150, 3))
    d *= (rng.uniform(0.02, 0.5 * SIGMA, size=150) / np.linalg.norm(d, axis=1))[:, None]
    Y = np.concatenate([base, np.mod(base + d, L)])
    s = System(300, L, 24, 1.5, 10, 10.0, 57, Y=Y)
    U, W = run_gpu(s, prec)
    Uo, Wo = s.oracle(prec)
    tol = FP32_TOL if precision == "fp32" else 1e-9
    assert_parity(U, Uo, tol, "U overlapping")
    assert_parity(W, Wo, tol, "W overlapping")


def test_non_finite_position_is_flagged_not_faulted(fcm):
    torch = torch_cuda()
    s = suspension(300, 0.05, 24, 1.5, 1e-6, 58)
    Y = s.Y.copy()
    Y[17, 1] = np.nan
    Y[99, 0] = np.inf
    with fcm.Handle(fcm.make_params(s.L, s.M, s.Sigma, s.r_c, s.M_G, s.n, fcm.FCM_FP32)) as h:
        pos = torch.as_tensor(Y, dtype=torch.float32, device="cuda")
        F = torch.as_tensor(s.F, dtype=torch.float32, device="cuda")
        U = torch.empty_like(F)
        h.apply(s.n, pos, F, None, U, None, torch.cuda.current_stream().cuda_stream)
        assert h.check() & 1
        # the handle stays usable
        pos2 = torch.as_tensor(s.Y, dtype=torch.float32, device="cuda")
        h.apply(s.n, pos2, F, None, U, None, torch.cuda.current_stream().cuda_stream)
        assert h.check() == 0


def test_handle_reuse_with_smaller_n_and_repeat_calls(fcm):
    torch = torch_cuda()
    s = suspension(2000, 0.05, 32, 1.5, 1e-6, 59)
    with fcm.Handle(fcm.make_params(s.L, s.M, s.Sigma, s.r_c, s.M_G, 5000, fcm.FCM_FP32)) as h:
        U1, W1 = run_gpu(s, fcm.FCM_FP32, handle=h)
        U2, W2 = run_gpu(s, fcm.FCM_FP32, handle=h)
        sub = System(500, s.L, s.M, s.Sigma, s.M_G, s.r_c, 60, Y=s.Y[:500])
        U3, W3 = run_gpu(sub, fcm.FCM_FP32, handle=h)
    assert_parity(U2, U1, 1e-6, "U repeat")
    Uo, Wo = sub.oracle(fcm.FCM_FP32)
    assert_parity(U3, Uo, FP32_TOL, "U smaller n")
    assert_parity(W3, Wo, FP32_TOL, "W smaller n")


def test_rod_layout_clustered_pairs(fcm):
    """Rods of spheres at 2.2a spacing (Section 6.1 layouts): clustered, uneven pair load."""
    L = inputs.box_edge(128 * 16, 0.05)
    Y, _ = inputs.random_rods(128, 16, L, 61)
    n = Y.shape[0]
    s = System(n, L, 40, 1.8, 14, min(op.cutoff_radius(1.8, 1e-6, torques=True), L / 2), 62, Y=Y)
    s.F, s.T = inputs.random_loads(n, 63, mean_free=False, scale=0.1, bias=(0, 0, -1))
    U, W = run_gpu(s, fcm.FCM_FP32)
    Uo, Wo = s.oracle(fcm.FCM_FP32)
    assert_parity(U, Uo, FP32_TOL, "U rods")
    assert_parity(W, Wo, FP32_TOL, "W rods")


# ---------------------------------------------------------------- properties

def test_symmetry_linearity_positivity_fp32(fcm):
    """<(F1,T1), M (F2,T2)> = <(F2,T2), M (F1,T1)>, M linear, F.U + T.W > 0 (Section 3.3)."""
    s = suspension(5000, 0.05, 40, 2.0, 1e-6, 64)
    U1, W1 = run_gpu(s, fcm.FCM_FP32)
    F1, T1 = s.F.copy(), s.T.copy()
    s.F, s.T = inputs.random_loads(s.n, 65)
    U2, W2 = run_gpu(s, fcm.FCM_FP32)
    a = np.sum(F1 * U2) + np.sum(T1 * W2)
    b = np.sum(s.F * U1) + np.sum(s.T * W1)
    assert abs(a - b) < 1e-5 * (abs(a) + abs(b))
    assert np.sum(F1 * U1) + np.sum(T1 * W1) > 0
    F2, T2 = s.F.copy(), s.T.copy()
    s.F, s.T = 2.0 * F1 - 3.0 * F2, 2.0 * T1 - 3.0 * T2
    U3, W3 = run_gpu(s, fcm.FCM_FP32)
    assert_parity(U3, 2.0 * U1 - 3.0 * U2, 1e-5, "U linear")
    assert_parity(W3, 2.0 * W1 - 3.0 * W2, 1e-5, "W linear")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_dilute_system_with_widened_pair_cells(fcm, precision):
    """phi = 0.2%: an r_c cell would hold about one particle, so the library widens the pair cells
    (side (8/rho)^(1/3) > r_c, five cells per side here); every pair within r_c must still be found."""
    n, phi, M, Sigma = 1200, 0.002, 64, 2.5
    L = inputs.box_edge(n, phi)
    rc = op.cutoff_radius(Sigma, 1e-6, torques=True)
    rho = n / L ** 3
    assert (8.0 / rho) ** (1.0 / 3.0) > 1.3 * rc      # the widened side is what the kernels use
    s = System(n, L, M, Sigma, op.support_points(Sigma, L / M, 4.8), rc, inputs.BASE_SEED + 71)
    prec = fcm.FCM_FP32 if precision == "fp32" else fcm.FCM_FP64
    tol = FP32_TOL if precision == "fp32" else FP64_TOL
    U, W = run_gpu(s, prec, stages=fcm.STAGE_PAIR)
    Uo, Wo = s.oracle(prec, stages=2)
    assert_parity(U, Uo, tol, f"U pair stage, widened cells, {precision}")
    assert_parity(W, Wo, tol, f"W pair stage, widened cells, {precision}")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_flat_box_like_the_applications(fcm, precision):
    """A thin periodic slab on a 96 x 96 x 16 grid, the shape of the applications' 256^2 x 16 and
    512^2 x 8 grids (Section 6): M_G close to M_z, cells and tiles wrap in z."""
    prec = fcm.FCM_FP32 if precision == "fp32" else fcm.FCM_FP64
    L = (72.0, 72.0, 12.0)
    Sigma = 1.0
    rc = op.cutoff_radius(Sigma, 1e-4, torques=True)
    assert rc <= 6.0
    s = System(900, L, (96, 96, 16), Sigma, 12, rc, inputs.BASE_SEED + 72)
    U, W = run_gpu(s, prec)
    Uo, Wo = s.oracle(prec)
    tol = FP32_TOL if precision == "fp32" else FP64_TOL
    assert_parity(U, Uo, tol, f"U flat slab {precision}")
    assert_parity(W, Wo, tol, f"W flat slab {precision}")
