"""Full-size checks of the CUDA path in the launch configuration bench.py times.

* The 128^3 workload (N = 65,536, phi = 5%, Sigma = 2a, M_G = 14, r_c from the
  1e-6 rule, forces + torques, FP32) against the full FP64 oracle, element by
  element.
* The N = 1,048,576, phi = 10%, 256^3 workload, too large for the full oracle:
  the FP32 path against the FP64 plain path on the same GPU (itself held to
  1e-10 against the oracle at smaller sizes), the pair stage on sampled
  particles against the oracle computed one particle at a time, and the
  symmetry of the discrete operator.
* The exact batched launch bench.py times (32 systems of the 128^3 workload): sampled systems
  against their single-system applies, and the last one against the full oracle.
* Brownian increments on the 128^3 workload: the grid part at sampled particles against the
  oracle's noise velocity on the whole grid.
* The rigid-rod solve on the 7,744-rod suspension: the equations it solves, checked on the host,
  and the rod velocities against an FP64 solve.
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


def test_brownian_grid_part_full_size_on_sampled_particles(fcm):
    """fcm_brownian's grid part on the 128^3 workload (the configuration bench.py times): the
    noise through the square-root Stokes operator on the whole grid in the oracle, then
    interpolated at 300 sampled particles, element by element."""
    import torch
    from oracle import brownian as ob
    s = _workload(65536, 0.05, 128, 2.0, inputs.BASE_SEED + 1)
    kT = 1.0
    xi = np.random.default_rng(2310127400).standard_normal((3, 128, 128, 128))   # [c][z][y][x]
    dev = torch.device("cuda:0")
    pos = torch.as_tensor(s.Y, dtype=torch.float32, device=dev)
    U = torch.empty_like(pos)
    W = torch.empty_like(pos)
    xid = torch.as_tensor(xi.ravel(), dtype=torch.float32, device=dev)
    with fcm.Handle(fcm.make_params(s.L, s.M, s.Sigma, s.r_c, s.M_G, s.n, fcm.FCM_FP32)) as h:
        it = h.brownian(s.n, pos, kT, xid, None, U, W, max_iter=10, tol=1e-6,
                        stream=torch.cuda.current_stream().cuda_stream)
    assert it == 0
    idx = np.random.default_rng(75).choice(s.n, 300, replace=False)
    xir = rounded(xi, fcm.FCM_FP32).transpose(0, 3, 2, 1)   # oracle layout [c][x][y][z]
    h3 = (s.L / s.M) ** 3
    u = np.sqrt(2.0 * kT / h3) * ob.grid_noise_velocity(xir, s.L)
    Uo, Wo = og.interpolate(u, rounded(s.Y, fcm.FCM_FP32)[idx], s.L, s.M_G, s.Sigma, s.Sigma)
    assert_parity(U.double().cpu().numpy()[idx], Uo, FP32_TOL, "U Brownian grid part, 300 of 65,536")
    assert_parity(W.double().cpu().numpy()[idx], Wo, FP32_TOL, "W Brownian grid part, 300 of 65,536")


def test_rod_suspension_rigid_solve_full_size(fcm):
    """fcm_rigid_solve on the 7,744-rod suspension in the launch configuration bench.py times
    (FP32, Broyden tol 1e-4): the equations it solves hold on the host (rigid particle velocities
    under fcm_apply, rod force and torque sums), and the rod velocities agree with an FP64 solve at
    1e-8 on the same GPU (the FP64 solve is held to the dense oracle at small sizes); the solve from
    each rod's own mobility (body preconditioner) takes fewer steps to the same rod velocities."""
    import math
    import torch
    import bench
    n_rods, tol = 7744, 1e-4
    Lxy, Lz = 960.0 * math.sqrt(n_rods / 2304.0), 60.0
    Y, off, X = inputs.doublet_rods(n_rods, Lxy, Lz, 2310127500)
    ft = inputs.rod_loads(n_rods, 2310127501, gravity=(1.0, 0.0, 0.0))
    n = Y.shape[0]
    pr = bench.rod_suspension_params(Lxy, Lz, n, tol)
    dev = torch.device("cuda:0")
    st = torch.cuda.current_stream().cuda_stream
    out = {}
    for prec, t, pc in ((fcm.FCM_FP32, tol, 0), (fcm.FCM_FP64, 1e-8, 0), ("body", tol, 1)):
        pc = fcm.RIGID_PRECOND_BODY if pc else fcm.RIGID_PRECOND_DIAGONAL
        key = prec
        prec = fcm.FCM_FP32 if prec == "body" else prec
        dt = torch.float32 if prec == fcm.FCM_FP32 else torch.float64
        tens = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
        pos, Xd, ftd = tens(Y), tens(X), tens(ft)
        F = torch.zeros((n, 3), dtype=dt, device=dev)
        UG = torch.zeros((n_rods, 6), dtype=dt, device=dev)
        p = fcm.make_params((Lxy, Lxy, Lz), pr["M"], pr["Sigma"], pr["r_c"], pr["M_G"], n, prec)
        with fcm.Handle(p) as h:
            code, it, res = h.rigid_solve(n, pos, n_rods, torch.as_tensor(off, device=dev), Xd, ftd, F, UG,
                                          max_iter=256, tol=t, stream=st, precond=pc)
            V = torch.empty_like(F)
            h.apply(n, pos, F, None, V, None, st)
            torch.cuda.synchronize()
        assert code == fcm.FCM_OK and res <= t and it < 100, (key, it, res)
        out[key] = (F.double().cpu().numpy(), UG.double().cpu().numpy(), V.double().cpu().numpy(), it)
    assert out["body"][3] < out[fcm.FCM_FP32][3]   # fewer steps from each rod's own mobility
    assert rel_l2(out["body"][1], out[fcm.FCM_FP64][1]) <= 1e-4
    F, UG, V, _ = out[fcm.FCM_FP32]
    Lv = np.array([Lxy, Lxy, Lz])
    r = rounded(Y, fcm.FCM_FP32).reshape(n_rods, 22, 3) - rounded(X, fcm.FCM_FP32)[:, None, :]
    r -= Lv * np.round(r / Lv)
    F3, V3 = F.reshape(n_rods, 22, 3), V.reshape(n_rods, 22, 3)
    rigid = UG[:, None, :3] + np.cross(UG[:, None, 3:], r)
    sums = np.concatenate([F3.sum(axis=1), np.cross(r, F3).sum(axis=1)], axis=1)
    mu = 1.0 / (6.0 * math.pi)
    # ||R|| <= tol ||ft||: the rigid-motion block times mu bounds the velocity residual
    bound_v = tol * np.linalg.norm(ft) * mu / np.linalg.norm(V) * 1.01 + 3e-6
    rel_v = float(np.linalg.norm(V3 - rigid) / np.linalg.norm(V))
    rel_s = float(np.linalg.norm(sums - ft) / np.linalg.norm(ft))
    print(f"7,744 rods: rigid-motion residual {rel_v:.2e} (bound {bound_v:.2e}), sums {rel_s:.2e}")
    assert rel_v <= bound_v and rel_s <= tol * 1.01 + 3e-6
    # rod velocities: the FP32 solve at 1e-4 against the FP64 solve at 1e-8
    assert rel_l2(UG, out[fcm.FCM_FP64][1]) <= 1e-4


def test_bench_launch_configuration_32_systems(fcm):
    """The batched pass bench.py times (32 systems x N = 65,536 at 5%, 128^3, Sigma = 2a, the bench's
    seeds, one fcm_batch_apply): every sampled system equals its single-system apply (atomic rounding
    only, 1e-6), and the last system matches the full FP64 oracle element by element."""
    import torch
    import bench
    w = bench.workload("c2")
    n, B = w["n"], 32
    systems = [System(n, w["L"], w["M"], w["Sigma"], w["M_G"], w["r_c"], 0,
                      Y=inputs.random_suspension(n, w["L"], inputs.BASE_SEED + 1 + 100 * b)) for b in range(B)]
    for b, s in enumerate(systems):   # the bench's loads: seed + 1 of each system
        s.F, s.T = inputs.random_loads(n, inputs.BASE_SEED + 2 + 100 * b)
    dev = torch.device("cuda:0")
    st = torch.cuda.current_stream().cuda_stream
    cat = lambda attr: torch.as_tensor(np.concatenate([getattr(s, attr) for s in systems]), dtype=torch.float32,
                                       device=dev)
    pos, F, T = cat("Y"), cat("F"), cat("T")
    U = torch.empty_like(F)
    W = torch.empty_like(F)
    offsets = [b * n for b in range(B + 1)]
    p = fcm.make_params(w["L"], w["M"], w["Sigma"], w["r_c"], w["M_G"], n * B, fcm.FCM_FP32)
    with fcm.Handle(p, 0, max_systems=B) as h:
        h.batch_apply(offsets, pos, F, T, U, W, st)
        assert h.check() == 0
    Ub, Wb = U.double().cpu().numpy(), W.double().cpu().numpy()
    for b in (0, 13, 31):
        Us, Ws = run_gpu(systems[b], fcm.FCM_FP32)
        assert_parity(Ub[b * n:(b + 1) * n], Us, 1e-6, f"U system {b} of the batch vs alone")
        assert_parity(Wb[b * n:(b + 1) * n], Ws, 1e-6, f"W system {b} of the batch vs alone")
    Uo, Wo = systems[31].oracle(fcm.FCM_FP32)
    assert_parity(Ub[31 * n:], Uo, FP32_TOL, "U system 31 of the batch vs oracle")
    assert_parity(Wb[31 * n:], Wo, FP32_TOL, "W system 31 of the batch vs oracle")
