"""Pins of the rigid-body mobility oracle (rod suspensions, Section 6.1).

* the saddle-point solution agrees with the Schur-complement route;
* with a diagonal mobility mu I and X_b at the centroid, U_b = mu f_b / n_b and
  Gamma_b = mu I_b^-1 tau_b (I_b the particles' second-moment tensor), which checks K's
  sign conventions; Broyden started from that Jacobian then needs one step;
* with the fast-FCM mobility the particles move rigidly and carry the rod force and torque
  (checked with np.cross, not with K);
* Broyden's product-form steps equal the textbook rank-one inverse update, satisfy the
  secant condition, and end within 2m steps on an m-dimensional linear system (Gay 1979);
* symmetry: a doublet rod pushed along its axis translates along it without rotating,
  and faster than when pushed across it (slender body).
"""
import math

import numpy as np
import pytest

from oracle import params as op
from oracle import rigid as orr
from paper_2310_12651_gb300 import inputs

L3 = (40.0, 40.0, 24.0)
M3 = (32, 32, 20)
SIGMA = 1.5


def _fcm_setup(n_rods=3, seed=100):
    MG = op.support_points(SIGMA, 1.25, 4.8)
    rc = op.cutoff_radius(SIGMA, 1e-6)
    pos, off, X = inputs.doublet_rods(n_rods, L3[0], L3[2], inputs.BASE_SEED + seed, lattice=False)
    return pos, off, X, MG, rc


@pytest.fixture(scope="module")
def fcm_system():
    pos, off, X, MG, rc = _fcm_setup()
    Mvf = orr.mobility_matrix_vf(pos, L3, M3, MG, SIGMA, rc)
    ft = inputs.rod_loads(3, inputs.BASE_SEED + 101, scale=1.0)
    return pos, off, X, MG, rc, Mvf, ft


def test_saddle_point_and_schur_complement_agree(fcm_system):
    pos, off, X, MG, rc, Mvf, ft = fcm_system
    K = orr.constraint_matrix(pos, off, X, L3)
    F1, W1 = orr.solve_saddle(Mvf, K, ft)
    F2, W2 = orr.solve_schur(Mvf, K, ft)
    assert np.abs(F1 - F2).max() < 1e-10 * np.abs(F1).max()
    assert np.abs(W1 - W2).max() < 1e-10 * np.abs(W1).max()
    # on a random SPD matrix as well
    rng = np.random.default_rng(7)
    A = rng.standard_normal(Mvf.shape)
    A = A @ A.T / Mvf.shape[0] + 0.1 * np.eye(Mvf.shape[0])
    F1, W1 = orr.solve_saddle(A, K, ft)
    F2, W2 = orr.solve_schur(A, K, ft)
    assert np.abs(W1 - W2).max() < 1e-10 * np.abs(W1).max()


def test_diagonal_mobility_closed_form():
    eta, a = 1.3, 1.0
    mu = 1.0 / (6.0 * math.pi * eta * a)
    pos, off, X = inputs.doublet_rods(4, 60.0, 30.0, inputs.BASE_SEED + 102, lattice=False)
    ft = inputs.rod_loads(4, inputs.BASE_SEED + 103, scale=2.0)
    n = pos.shape[0]
    K = orr.constraint_matrix(pos, off, X, 60.0 * np.array([1, 1, 0.5]))
    F, W = orr.solve_saddle(mu * np.eye(3 * n), K, ft)
    for b in range(4):
        rb = pos[off[b]:off[b + 1]] - X[b]
        rb -= np.array([60.0, 60.0, 30.0]) * np.round(rb / np.array([60.0, 60.0, 30.0]))
        inertia = sum(np.dot(r, r) * np.eye(3) - np.outer(r, r) for r in rb)
        assert np.allclose(W[b, :3], mu * ft[b, :3] / len(rb), rtol=1e-12, atol=0)
        assert np.allclose(W[b, 3:], mu * np.linalg.solve(inertia, ft[b, 3:]), rtol=1e-10, atol=1e-15)
    # Broyden from the diagonal-mobility Jacobian is exact in one step for this mobility
    Fb, Wb, it, rel = orr.rigid_broyden(lambda f: mu * f, pos, off, X, np.array([60.0, 60.0, 30.0]), ft,
                                        1e-12, 10, eta=eta)
    assert it == 1 and rel[-1] < 1e-13
    assert np.allclose(Wb, W, rtol=1e-12, atol=1e-16)


def test_fcm_solution_moves_rigidly(fcm_system):
    pos, off, X, MG, rc, Mvf, ft = fcm_system
    F, W = orr.solve_saddle(Mvf, orr.constraint_matrix(pos, off, X, L3), ft)
    V = (Mvf @ F.ravel()).reshape(-1, 3)
    Lv = np.array(L3)
    scale = np.abs(V).max()
    for b in range(len(off) - 1):
        sl = slice(off[b], off[b + 1])
        r = pos[sl] - X[b]
        r -= Lv * np.round(r / Lv)
        rigid = W[b, :3][None, :] + np.cross(W[b, 3:][None, :], r)
        assert np.abs(V[sl] - rigid).max() < 1e-11 * scale
        assert np.allclose(F[sl].sum(axis=0), ft[b, :3], rtol=0, atol=1e-11 * np.abs(ft).max())
        assert np.allclose(np.cross(r, F[sl]).sum(axis=0), ft[b, 3:], rtol=0, atol=1e-10 * np.abs(ft).max())


def test_broyden_steps_follow_the_rank_one_update():
    """Product-form steps == textbook inverse update; secant condition; end within 2m steps."""
    m = 7
    rng = np.random.default_rng(11)
    A = np.eye(m) + 0.4 * rng.standard_normal((m, m))
    b = rng.standard_normal(m)
    H0 = np.linalg.inv(np.diag(np.diag(A)))
    xs = []

    def residual(x):
        xs.append(x.copy())
        return A @ x - b

    x, it, norms = orr.broyden(residual, lambda v: H0 @ v, np.zeros(m), 1e-11 * np.linalg.norm(b), 4 * m)
    assert it <= 2 * m and norms[-1] <= 1e-11 * np.linalg.norm(b)
    assert np.allclose(x, np.linalg.solve(A, b), rtol=0, atol=1e-9)
    # replay with the dense update H+ = H + (s - H y) s^T H / (s^T H y)
    H = H0.copy()
    x = np.zeros(m)
    Rx = A @ x - b
    for k in range(1, len(xs)):
        s = -H @ Rx
        assert np.allclose(x + s, xs[k], rtol=0, atol=1e-9 * (1 + np.abs(xs[k]).max())), k
        Rn = A @ (x + s) - b
        y = Rn - Rx
        H = H + np.outer(s - H @ y, s @ H) / (s @ H @ y)
        assert np.allclose(H @ y, s, rtol=0, atol=1e-9 * np.abs(s).max())   # secant condition
        x, Rx = x + s, Rn


def test_broyden_converges_to_the_saddle_point_solution(fcm_system):
    pos, off, X, MG, rc, Mvf, ft = fcm_system
    F0, W0 = orr.solve_saddle(Mvf, orr.constraint_matrix(pos, off, X, L3), ft)
    F, W, it, rel = orr.rigid_broyden(lambda f: (Mvf @ f.ravel()).reshape(-1, 3), pos, off, X, L3, ft, 1e-11, 200)
    assert 5 < it < 120 and rel[-1] <= 1e-11
    assert np.abs(W - W0).max() < 1e-9 * np.abs(W0).max()
    assert np.abs(F - F0).max() < 1e-7 * np.abs(F0).max()
    # at the paper's tolerance the rod velocities are already close
    F4, W4, it4, _ = orr.rigid_broyden(lambda f: (Mvf @ f.ravel()).reshape(-1, 3), pos, off, X, L3, ft, 1e-4, 200)
    assert it4 < it and np.abs(W4 - W0).max() < 1e-3 * np.abs(W0).max()


def test_rod_pushed_along_its_axis_translates_without_rotating():
    MG = op.support_points(SIGMA, 1.25, 4.8)
    rc = op.cutoff_radius(SIGMA, 1e-6)
    # one rod through the box centre (a grid point), turned about z so that its axis is x
    pos, off, X = inputs.doublet_rods(1, L3[0], L3[2], inputs.BASE_SEED + 104, lattice=True)
    d = pos[20] + pos[21] - pos[0] - pos[1]
    ang = math.atan2(d[1], d[0])
    c, s = math.cos(-ang), math.sin(-ang)
    Rz = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
    pos = X[0] + (pos - X[0]) @ Rz.T
    Mvf = orr.mobility_matrix_vf(pos, L3, M3, MG, SIGMA, rc)
    K = orr.constraint_matrix(pos, off, X, L3)
    axis = pos[20] + pos[21] - pos[0] - pos[1]
    axis /= np.linalg.norm(axis)
    assert abs(abs(axis[0]) - 1.0) < 1e-12
    _, Wpar = orr.solve_saddle(Mvf, K, np.array([[22.0, 0, 0, 0, 0, 0]]))
    _, Wperp = orr.solve_saddle(Mvf, K, np.array([[0, 22.0, 0, 0, 0, 0]]))
    # the reflections x, y, z -> -x, -y, -z about the rod centre map the rod, the grid and the
    # windows onto themselves up to the kernel truncation (M_G points, ~1e-5 of the kernel)
    assert np.abs(Wpar[0, 1:]).max() < 1e-4 * abs(Wpar[0, 0])
    assert abs(Wperp[0, 0]) < 1e-4 * abs(Wperp[0, 1]) and np.abs(Wperp[0, 3:]).max() < 1e-4 * abs(Wperp[0, 1])
    assert Wpar[0, 0] > Wperp[0, 1] > 0.0


def test_body_preconditioner_is_exact_for_isolated_bodies():
    """With the mobility of bodies that do not interact (each body's own free-space FCM block), the
    body preconditioner is the exact inverse Jacobian: Broyden ends after one step, at the dense
    solution. The blocks themselves are the free-space FCM pair mobility (checked against S(x; sigma
    sqrt 2) of the closed forms and symmetric)."""
    from oracle import closed_forms as cf
    L = np.array([80.0, 80.0, 40.0])
    pos, off, X = inputs.doublet_rods(4, L[0], L[2], inputs.BASE_SEED + 105, lattice=False)
    ft = inputs.rod_loads(4, inputs.BASE_SEED + 106, scale=1.0)
    n = pos.shape[0]
    Mbd = np.zeros((3 * n, 3 * n))
    for b in range(4):
        sl = slice(3 * off[b], 3 * off[b + 1])
        Mbd[sl, sl] = orr.body_mobility(pos[off[b]:off[b + 1]], L)
    assert np.allclose(Mbd, Mbd.T, rtol=0, atol=1e-15)
    d = pos[1] - pos[0]
    assert np.allclose(Mbd[0:3, 3:6], cf.S(d[None, :], cf.fcm_sigma() * math.sqrt(2.0))[0], rtol=1e-14, atol=0)
    F0, W0 = orr.solve_saddle(Mbd, orr.constraint_matrix(pos, off, X, L), ft)
    F, W, it, rel = orr.rigid_broyden(lambda f: (Mbd @ f.ravel()).reshape(-1, 3), pos, off, X, L, ft, 1e-12, 10,
                                      precond="body")
    assert it == 1 and rel[-1] < 1e-12
    assert np.allclose(W, W0, rtol=1e-10, atol=0) and np.allclose(F, F0, rtol=1e-9, atol=1e-12)


def test_body_preconditioner_converges_to_the_same_solution(fcm_system):
    pos, off, X, MG, rc, Mvf, ft = fcm_system
    F0, W0 = orr.solve_saddle(Mvf, orr.constraint_matrix(pos, off, X, L3), ft)
    av = lambda f: (Mvf @ f.ravel()).reshape(-1, 3)
    F, W, itb, rel = orr.rigid_broyden(av, pos, off, X, L3, ft, 1e-11, 200, precond="body")
    _, _, itd, _ = orr.rigid_broyden(av, pos, off, X, L3, ft, 1e-11, 200)
    assert rel[-1] <= 1e-11 and itb < itd
    assert np.abs(W - W0).max() < 1e-9 * np.abs(W0).max()
