"""Rigid-body mobility solve on the GPU (fcm_rigid_solve) against the oracle of oracle/rigid.py.

* FP64: the solve at a tight tolerance equals the oracle's dense saddle-point solution (M built
  column by column from the fast-FCM oracle), and it takes as many Broyden steps as the
  oracle's Broyden on the same problem (same algorithm, same start, same tolerance);
* FP32 at the paper's tolerance: rod velocities within the FP32 bar of the dense solution;
* any size: the returned forces satisfy the equations they solve (rigid particle velocities
  under fcm_apply, rod force and torque sums), checked on the host with np.cross;
* ragged bodies, warm starts, ft = 0, invalid offsets, degenerate bodies, max_iter limits.
"""
import math

import numpy as np
import pytest

from gpu_util import FP32_TOL, FP64_TOL, assert_parity, ensure_built, rounded, torch_cuda
from oracle import params as op
from oracle import rigid as orr
from paper_2310_12651_gb300 import inputs

pytestmark = pytest.mark.gpu

L3 = (40.0, 40.0, 24.0)
M3 = (32, 32, 20)
SIGMA = 1.5


@pytest.fixture(scope="module")
def fcm():
    torch_cuda()
    return ensure_built()


def _geometry(L=L3, M=M3):
    MG = op.support_points(SIGMA, max(l / m for l, m in zip(L, M)), 4.8)
    rc = op.cutoff_radius(SIGMA, 1e-6)
    return MG, rc


def _rods(n_rods, seed):
    return inputs.doublet_rods(n_rods, L3[0], L3[2], inputs.BASE_SEED + seed, lattice=False)


def _ragged(seed, sizes):
    """Bodies of the given sizes: points within 4a of a random centre (not collinear)."""
    rng = np.random.default_rng(seed)
    Y, X = [], []
    for k in sizes:
        c = rng.random(3) * np.array(L3)
        pts = c + rng.uniform(-4.0, 4.0, size=(k, 3))
        Y.append(np.mod(pts, np.array(L3)))
        X.append(c)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    return np.concatenate(Y), off, np.array(X)


def _solve(fcm, prec, Y, off, X, ft, tol, max_iter=256, warm=None, check=True, handle=None, L=L3, M=M3, precond=0):
    import torch
    dt = torch.float32 if prec == fcm.FCM_FP32 else torch.float64
    dev = torch.device("cuda:0")
    n, nb = Y.shape[0], len(off) - 1
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    pos, Xd, ftd = t(Y), t(X), t(ft)
    offd = torch.as_tensor(np.asarray(off, dtype=np.int32), device=dev)
    F = torch.zeros((n, 3), dtype=dt, device=dev) if warm is None else t(warm[0])
    UG = torch.zeros((nb, 6), dtype=dt, device=dev) if warm is None else t(warm[1])
    MG, rc = _geometry(L, M)
    own = handle is None
    h = handle or fcm.Handle(fcm.make_params(L, M, SIGMA, rc, MG, n, prec))
    try:
        code, it, res = h.rigid_solve(n, pos, nb, offd, Xd, ftd, F, UG, max_iter=max_iter, tol=tol,
                                      warm=warm is not None, stream=torch.cuda.current_stream().cuda_stream,
                                      check=check, precond=precond)
        torch.cuda.synchronize()
        V = torch.empty_like(F)
        h.apply(n, pos, F, None, V, None, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
    finally:
        if own:
            h.close()
    return (code, it, res, F.double().cpu().numpy(), UG.double().cpu().numpy(), V.double().cpu().numpy())


def _oracle_dense(Y, off, X, ft):
    MG, rc = _geometry()
    Mvf = orr.mobility_matrix_vf(Y, L3, M3, MG, SIGMA, rc)
    return Mvf, orr.solve_saddle(Mvf, orr.constraint_matrix(Y, off, X, L3), ft)


def _check_equations(Y, off, X, ft, F, UG, V, tol_rigid, tol_sums, L=L3):
    """The equations of the problem, on the host: V_i = U_b + Gamma_b x r_i, sums of F and r x F."""
    Lv = np.array(L)
    mu = 1.0 / (6.0 * math.pi)
    vscale = np.linalg.norm(V)
    err_v = 0.0
    err_s = 0.0
    for b in range(len(off) - 1):
        sl = slice(off[b], off[b + 1])
        r = Y[sl] - X[b]
        r -= Lv * np.round(r / Lv)
        err_v += float(np.sum((V[sl] - UG[b, :3] - np.cross(UG[b, 3:], r)) ** 2))
        err_s += float(np.sum((F[sl].sum(axis=0) - ft[b, :3]) ** 2) +
                       np.sum((np.cross(r, F[sl]).sum(axis=0) - ft[b, 3:]) ** 2))
    rel_v = math.sqrt(err_v) / vscale
    rel_s = math.sqrt(err_s) / np.linalg.norm(ft)
    print(f"rigid-motion residual {rel_v:.2e}, force/torque-sum residual {rel_s:.2e} (mu = {mu:.4f})")
    assert rel_v <= tol_rigid, rel_v
    assert rel_s <= tol_sums, rel_s


def test_fp64_solve_equals_the_dense_oracle_solution(fcm):
    Y, off, X = _rods(3, 200)
    ft = inputs.rod_loads(3, inputs.BASE_SEED + 201, scale=1.0)
    Mvf, (F0, W0) = _oracle_dense(Y, off, X, ft)
    code, it, res, F, UG, V = _solve(fcm, fcm.FCM_FP64, Y, off, X, ft, 1e-12)
    assert code == fcm.FCM_OK and res <= 1e-12 and 10 < it < 200, (it, res)
    assert_parity(UG, W0, FP64_TOL, f"rod velocities FP64 ({it} Broyden steps)")
    assert_parity(F, F0, FP64_TOL, "particle forces FP64")
    # the same number of steps as the oracle's Broyden (same algorithm, start and tolerance)
    for tol in (1e-4, 1e-8):
        _, _, it_o, _ = orr.rigid_broyden(lambda f: (Mvf @ f.ravel()).reshape(-1, 3), Y, off, X, L3, ft, tol, 256)
        _, it_g, _, _, _, _ = _solve(fcm, fcm.FCM_FP64, Y, off, X, ft, tol)
        assert abs(it_g - it_o) <= 1, (tol, it_g, it_o)


def test_fp32_solve_at_the_paper_tolerance(fcm):
    Y, off, X = _rods(3, 202)
    ft = inputs.rod_loads(3, inputs.BASE_SEED + 203, scale=1.0)
    Yr, Xr, ftr = rounded(Y, fcm.FCM_FP32), rounded(X, fcm.FCM_FP32), rounded(ft, fcm.FCM_FP32)
    _, (F0, W0) = _oracle_dense(Yr, off, Xr, ftr)
    code, it, res, F, UG, V = _solve(fcm, fcm.FCM_FP32, Y, off, X, ft, 1e-5)
    assert code == fcm.FCM_OK and res <= 1e-5, (it, res)
    assert_parity(UG, W0, FP32_TOL, f"rod velocities FP32 at tol 1e-5 ({it} Broyden steps)")
    code, it4, res4, F4, UG4, _ = _solve(fcm, fcm.FCM_FP32, Y, off, X, ft, 1e-4)
    assert code == fcm.FCM_OK and it4 < it
    assert_parity(UG4, W0, 1e-3, f"rod velocities FP32 at the paper's tol 1e-4 ({it4} Broyden steps)")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_ragged_bodies_match_the_oracle(fcm, precision):
    prec = fcm.FCM_FP32 if precision == "fp32" else fcm.FCM_FP64
    sizes = [3, 17, 5, 33, 4, 9, 26, 3]
    Y, off, X = _ragged(204, sizes)
    ft = inputs.rod_loads(len(sizes), inputs.BASE_SEED + 205, scale=1.0, per_rod=1)
    Yr, Xr, ftr = rounded(Y, prec), rounded(X, prec), rounded(ft, prec)
    _, (F0, W0) = _oracle_dense(Yr, off, Xr, ftr)
    tol = 1e-12 if precision == "fp64" else 1e-5
    code, it, res, F, UG, V = _solve(fcm, prec, Y, off, X, ft, tol)
    assert code == fcm.FCM_OK
    assert_parity(UG, W0, FP64_TOL if precision == "fp64" else FP32_TOL, f"ragged bodies {precision} ({it} steps)")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_equations_hold_for_a_rod_lattice(fcm, precision):
    """16 rods on a 4 x 4 lattice of spacing 16a (352 particles, rods apart as in the paper's
    suspensions): the equations checked on the host. (Rods that cross each other, e.g. 64 rods
    at spacing 5a, make Broyden from the diagonal-mobility Jacobian diverge; the oracle shows
    the same.)"""
    prec = fcm.FCM_FP32 if precision == "fp32" else fcm.FCM_FP64
    L, M = (64.0, 64.0, 24.0), (52, 52, 20)
    Y, off, X = inputs.doublet_rods(16, L[0], L[2], inputs.BASE_SEED + 206)
    ft = inputs.rod_loads(16, inputs.BASE_SEED + 207, scale=0.5)
    tol = 1e-4 if precision == "fp32" else 1e-9
    code, it, res, F, UG, V = _solve(fcm, prec, Y, off, X, ft, tol, L=L, M=M)
    assert code == fcm.FCM_OK and res <= tol
    # ||R|| <= tol ||ft|| bounds both blocks: the rigid-motion one in velocity units (times mu)
    mu = 1.0 / (6.0 * math.pi)
    slack = 3e-6 if precision == "fp32" else 1e-12
    bound_v = tol * np.linalg.norm(ft) * mu / np.linalg.norm(V) * 1.01 + slack
    _check_equations(rounded(Y, prec), off, rounded(X, prec), rounded(ft, prec), F, UG, V, bound_v,
                     tol * 1.01 + slack, L=L)


def test_warm_start_and_zero_loads(fcm):
    Y, off, X = _rods(4, 208)
    ft = inputs.rod_loads(4, inputs.BASE_SEED + 209, scale=1.0)
    code, it, res, F, UG, _ = _solve(fcm, fcm.FCM_FP64, Y, off, X, ft, 1e-8)
    assert code == fcm.FCM_OK and it > 5
    # restart from the solution: converged at the first residual
    code2, it2, res2, F2, UG2, _ = _solve(fcm, fcm.FCM_FP64, Y, off, X, ft, 1e-8, warm=(F, UG))
    assert code2 == fcm.FCM_OK and it2 == 0 and res2 <= 1e-8
    assert np.array_equal(F2, F) and np.allclose(UG2, UG, rtol=1e-15, atol=0)   # UG went through / mu, * mu
    # restart from a perturbed solution: fewer steps than from zero
    rng = np.random.default_rng(3)
    code3, it3, _, _, UG3, _ = _solve(fcm, fcm.FCM_FP64, Y, off, X, ft, 1e-8,
                                      warm=(F * (1 + 1e-3 * rng.standard_normal(F.shape)), UG))
    assert code3 == fcm.FCM_OK and it3 < it
    assert np.abs(UG3 - UG).max() < 1e-6 * np.abs(UG).max()
    # no load: zero forces and velocities without a product
    code4, it4, res4, F4, UG4, _ = _solve(fcm, fcm.FCM_FP64, Y, off, X, np.zeros_like(ft), 1e-8)
    assert code4 == fcm.FCM_OK and it4 == 0 and not F4.any() and not UG4.any()


def test_iteration_limit_reports_not_converged(fcm):
    Y, off, X = _rods(3, 210)
    ft = inputs.rod_loads(3, inputs.BASE_SEED + 211, scale=1.0)
    code, it, res, F, UG, _ = _solve(fcm, fcm.FCM_FP64, Y, off, X, ft, 1e-12, max_iter=3, check=False)
    assert code == fcm.FCM_ERR_NOT_CONVERGED and it == 3 and res > 1e-12
    assert np.isfinite(F).all() and np.abs(UG).max() > 0
    with pytest.raises(fcm.FcmError) as e:
        _solve(fcm, fcm.FCM_FP64, Y, off, X, ft, 1e-12, max_iter=3)
    assert e.value.code == fcm.FCM_ERR_NOT_CONVERGED and "after 3 iterations" in str(e.value)


@pytest.mark.parametrize("case", ["decreasing", "short", "long", "collinear"])
def test_invalid_bodies_are_flagged_before_any_product(fcm, case):
    Y, off, X = _rods(3, 212)
    ft = inputs.rod_loads(3, inputs.BASE_SEED + 213, scale=1.0)
    off = off.copy()
    if case == "decreasing":
        off[1], off[2] = off[2], off[1]
    elif case == "short":
        off[-1] -= 1          # the last body ends before n
    elif case == "long":
        off[-1] += 5          # beyond n
    else:
        Y = Y.copy()
        Y[22:44] = X[1] + np.outer(np.arange(22) - 10.5, [0.3, 0.4, 0.0])   # body 1 on one line
    with pytest.raises(fcm.FcmError) as e:
        _solve(fcm, fcm.FCM_FP64, Y, off, X, ft, 1e-6)
    assert e.value.code == fcm.FCM_ERR_INPUT
    assert ("degenerate" if case == "collinear" else "body_off invalid") in str(e.value)


def test_bad_arguments_are_rejected(fcm):
    import torch
    Y, off, X = _rods(2, 214)
    n = Y.shape[0]
    MG, rc = _geometry()
    with fcm.Handle(fcm.make_params(L3, M3, SIGMA, rc, MG, n, fcm.FCM_FP32)) as h:
        d = lambda a: torch.as_tensor(a, dtype=torch.float32, device="cuda")
        pos, Xd, ft = d(Y), d(X), d(np.ones((2, 6)))
        offd = torch.as_tensor(off, device="cuda")
        F, UG = torch.zeros((n, 3), device="cuda"), torch.zeros((2, 6), device="cuda")
        for kw, msg in ((dict(max_iter=0), "max_iter"), (dict(max_iter=257), "max_iter"), (dict(tol=0.0), "tol"),
                        (dict(nb=0), "n_bodies"), (dict(nb=n + 1), "n_bodies"), (dict(n=n + 1), "max_n"),
                        (dict(X=None), "non-NULL")):
            a = dict(n=n, nb=2, max_iter=10, tol=1e-4, X=Xd)
            a.update(kw)
            with pytest.raises(fcm.FcmError) as e:
                h.rigid_solve(a["n"], pos, a["nb"], offd, a["X"], ft, F, UG, max_iter=a["max_iter"], tol=a["tol"])
            assert e.value.code == fcm.FCM_ERR_ARG and msg in str(e.value), (kw, str(e.value))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_body_preconditioner_matches_the_oracle(fcm, precision):
    """Broyden from each body's own free-space FCM mobility (FCM_RIGID_PRECOND_BODY): the same dense
    oracle solution, the oracle's step count for that start (+-1), and fewer steps than from mu I."""
    prec = fcm.FCM_FP32 if precision == "fp32" else fcm.FCM_FP64
    Y, off, X = _rods(3, 200)
    ft = inputs.rod_loads(3, inputs.BASE_SEED + 201, scale=1.0)
    Yr, Xr, ftr = rounded(Y, prec), rounded(X, prec), rounded(ft, prec)
    Mvf, (F0, W0) = _oracle_dense(Yr, off, Xr, ftr)
    tol = 1e-12 if precision == "fp64" else 1e-5
    code, itb, res, F, UG, V = _solve(fcm, prec, Y, off, X, ft, tol, precond=fcm.RIGID_PRECOND_BODY)
    _, itd, _, _, _, _ = _solve(fcm, prec, Y, off, X, ft, tol)
    assert code == fcm.FCM_OK and res <= tol and itb < itd, (itb, itd)
    assert_parity(UG, W0, FP64_TOL if precision == "fp64" else FP32_TOL, f"rod velocities, body start ({itb} steps)")
    if precision == "fp64":
        assert_parity(F, F0, FP64_TOL, "particle forces, body start")
        for t in (1e-4, 1e-8):
            _, _, it_o, _ = orr.rigid_broyden(lambda f: (Mvf @ f.ravel()).reshape(-1, 3), Y, off, X, L3, ft, t, 256,
                                              precond="body")
            _, it_g, _, _, _, _ = _solve(fcm, prec, Y, off, X, ft, t, precond=fcm.RIGID_PRECOND_BODY)
            assert abs(it_g - it_o) <= 1, (t, it_g, it_o)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_body_preconditioner_on_a_rod_lattice_and_ragged_bodies(fcm, precision):
    prec = fcm.FCM_FP32 if precision == "fp32" else fcm.FCM_FP64
    L, M = (64.0, 64.0, 24.0), (52, 52, 20)
    Y, off, X = inputs.doublet_rods(16, L[0], L[2], inputs.BASE_SEED + 206)
    ft = inputs.rod_loads(16, inputs.BASE_SEED + 207, scale=0.5)
    tol = 1e-4 if precision == "fp32" else 1e-9
    code, itb, res, F, UG, V = _solve(fcm, prec, Y, off, X, ft, tol, L=L, M=M, precond=fcm.RIGID_PRECOND_BODY)
    _, itd, _, _, UGd, _ = _solve(fcm, prec, Y, off, X, ft, tol, L=L, M=M)
    assert code == fcm.FCM_OK and res <= tol and itb < itd, (itb, itd)
    mu = 1.0 / (6.0 * math.pi)
    slack = 3e-6 if precision == "fp32" else 1e-12
    _check_equations(rounded(Y, prec), off, rounded(X, prec), rounded(ft, prec), F, UG, V,
                     tol * np.linalg.norm(ft) * mu / np.linalg.norm(V) * 1.01 + slack, tol * 1.01 + slack, L=L)
    # ragged bodies of 3..32 particles (the limit)
    sizes = [3, 17, 5, 32, 4, 9, 26, 3]
    Y, off, X = _ragged(204, sizes)
    ft = inputs.rod_loads(len(sizes), inputs.BASE_SEED + 205, scale=1.0, per_rod=1)
    _, (F0, W0) = _oracle_dense(rounded(Y, prec), off, rounded(X, prec), rounded(ft, prec))
    code, it, res, F, UG, V = _solve(fcm, prec, Y, off, X, ft, 1e-12 if precision == "fp64" else 1e-5,
                                     precond=fcm.RIGID_PRECOND_BODY)
    assert code == fcm.FCM_OK
    assert_parity(UG, W0, FP64_TOL if precision == "fp64" else FP32_TOL, f"ragged bodies, body start ({it} steps)")


def test_body_preconditioner_limits(fcm):
    """Bodies beyond FCM_RIGID_BODY_MAX particles and an unknown precond are rejected."""
    Y, off, X = _ragged(215, [33, 4])
    ft = inputs.rod_loads(2, inputs.BASE_SEED + 216, scale=1.0, per_rod=1)
    with pytest.raises(fcm.FcmError) as e:
        _solve(fcm, fcm.FCM_FP32, Y, off, X, ft, 1e-4, precond=fcm.RIGID_PRECOND_BODY)
    assert e.value.code == fcm.FCM_ERR_INPUT and "at most 32" in str(e.value)
    with pytest.raises(fcm.FcmError) as e:
        _solve(fcm, fcm.FCM_FP32, Y, off, X, ft, 1e-4, precond=7)
    assert e.value.code == fcm.FCM_ERR_ARG and "precond" in str(e.value)
    # the same bodies with the diagonal start are fine
    code, it, res, _, _, _ = _solve(fcm, fcm.FCM_FP32, Y, off, X, ft, 1e-4)
    assert code == fcm.FCM_OK
