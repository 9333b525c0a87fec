"""Mobility problem of rigid bodies built from FCM particles, FP64 numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The rod suspensions of Section 6.1 make the FCM particles of each rod move as one
rigid body. With rod b's reference point X_b and lever arms r_i = Y_i - X_b
(minimum image), the particle forces F and rod velocities (U_b, Gamma_b) solve,
for given rod forces f_b and torques tau_b,
    V = M^VF F                                 (particle velocities, eq. U)
    V_i = U_b + Gamma_b x r_i     (i in b)     (rigid motion, eq. ui)
    sum_{i in b} F_i = f_b,  sum_{i in b} r_i x F_i = tau_b    (eqs. Fn, Tn)
With K the (3N x 6B) map from rod velocities to particle velocities
(K_i = [I, -[r_i]x] for i in b, so Gamma x r = -[r]x Gamma), K^T F collects each
rod's force and torque and the problem is the saddle-point system
    [ M   -K ] [F]   [0 ]
    [ K^T  0 ] [W] = [ft]
Its exact solution (dense LU, or the Schur complement) is the oracle for the GPU
solve. The paper solves it with Broyden's method started from the Jacobian of a
diagonal mobility M = mu I, mu = 1/(6 pi eta a) (Section 6.1); ``broyden`` and
``rigid_broyden`` take those steps (inverse "good" Broyden update, full steps). ``rigid_broyden``
can also start from the Jacobian of each body's own free-space FCM mobility (not in the paper).

Scaling used by ``rigid_broyden`` (a reading: the paper gives neither the norm nor
the scaling): the unknowns are x = (F, W/mu) and the residual is
R = ((M F - K W)/mu, K^T F - ft), both in force units, so that the diagonal
mobility Jacobian is J0 = [[I, -K], [K^T, 0]]. Convergence: ||R||_2 <= tol ||ft||_2
(||ft|| is the residual of x = 0).
"""
from __future__ import annotations

import math

import numpy as np

from . import closed_forms as cf
from .grid_fcm import _as3, fast_fcm_apply


def lever_arms(Y, body_off, X, L):
    """r_i = Y_i - X_b under the minimum image, particles of body b in [body_off[b], body_off[b+1])."""
    L = _as3(L)
    Y = np.asarray(Y, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    r = np.empty_like(Y)
    for b in range(len(body_off) - 1):
        d = Y[body_off[b]:body_off[b + 1]] - X[b]
        r[body_off[b]:body_off[b + 1]] = d - L * np.round(d / L)
    return r


def constraint_matrix(Y, body_off, X, L):
    """K (3N x 6B): particle velocities from rod velocities (U_b, Gamma_b)."""
    r = lever_arms(Y, body_off, X, L)
    nb = len(body_off) - 1
    K = np.zeros((3 * r.shape[0], 6 * nb))
    for b in range(nb):
        for i in range(body_off[b], body_off[b + 1]):
            rx, ry, rz = r[i]
            K[3 * i:3 * i + 3, 6 * b:6 * b + 3] = np.eye(3)
            K[3 * i:3 * i + 3, 6 * b + 3:6 * b + 6] = -np.array([[0.0, -rz, ry], [rz, 0.0, -rx], [-ry, rx, 0.0]])
    return K


def mobility_matrix_vf(Y, L, M, M_G, Sigma, R_c, a=1.0, eta=1.0):
    """The force-velocity block of the fast-FCM mobility (3N x 3N), one column per unit force."""
    n = Y.shape[0]
    cols = []
    for k in range(3 * n):
        F = np.zeros(3 * n)
        F[k] = 1.0
        U, _ = fast_fcm_apply(Y, F.reshape(n, 3), None, L, M, M_G, Sigma, R_c, a=a, eta=eta)
        cols.append(U.ravel())
    return np.array(cols).T


def solve_saddle(Mvf, K, ft):
    """(F, W) of the saddle-point system by dense LU; W rows are (U_b, Gamma_b)."""
    n3, b6 = K.shape
    A = np.block([[Mvf, -K], [K.T, np.zeros((b6, b6))]])
    rhs = np.concatenate([np.zeros(n3), np.asarray(ft, dtype=np.float64).ravel()])
    x = np.linalg.solve(A, rhs)
    return x[:n3].reshape(-1, 3), x[n3:].reshape(-1, 6)


def solve_schur(Mvf, K, ft):
    """The same problem by the Schur complement: W = (K^T M^-1 K)^-1 ft, F = M^-1 K W."""
    MinvK = np.linalg.solve(Mvf, K)
    W = np.linalg.solve(K.T @ MinvK, np.asarray(ft, dtype=np.float64).ravel())
    return (MinvK @ W).reshape(-1, 3), W.reshape(-1, 6)


def broyden(residual, precond, x0, tol_abs, max_iter):
    """Broyden's "good" method with an inverse-Jacobian update and full steps.

    ``residual(x)`` gives R(x); ``precond(v)`` applies H0, the inverse of the initial
    Jacobian. With H_{k+1} = H_k + (s_k - H_k y_k) s_k^T H_k / (s_k^T H_k y_k) and full
    steps s_k = -H_k R(x_k), y_k = R(x_{k+1}) - R(x_k), the update reduces to
    H_{k+1} = (I + s_{k+1} s_k^T / |s_k|^2) H_k, so H_k R is H0 R followed by one rank-one
    factor per earlier step, and the next step is z / (1 - s_k^T z / |s_k|^2) with
    z = -H_k R(x_{k+1}). Returns (x, iterations, residual norms); iterations counts the
    residual evaluations after the one at x0.
    """
    x = np.array(x0, dtype=np.float64)
    R = residual(x)
    norms = [float(np.linalg.norm(R))]
    if norms[-1] <= tol_abs:
        return x, 0, norms
    steps = [-precond(R)]
    for it in range(max_iter):
        x = x + steps[-1]
        R = residual(x)
        norms.append(float(np.linalg.norm(R)))
        if norms[-1] <= tol_abs:
            return x, it + 1, norms
        z = -precond(R)
        for j in range(len(steps) - 1):
            z = z + steps[j + 1] * (steps[j] @ z) / (steps[j] @ steps[j])
        sn = steps[-1]
        steps.append(z / (1.0 - (sn @ z) / (sn @ sn)))
    return x, max_iter, norms


def body_mobility(Yb, L, a=1.0, eta=1.0):
    """The free-space FCM force-velocity mobility of one body's particles (3k x 3k): pair blocks
    S(x; sigma sqrt 2) (eq. M_VF) for the minimum-image separations, 1/(6 pi eta a) I on the diagonal."""
    L = _as3(L)
    k = Yb.shape[0]
    Mb = np.zeros((3 * k, 3 * k))
    for i in range(k):
        for j in range(k):
            if i == j:
                Mb[3 * i:3 * i + 3, 3 * j:3 * j + 3] = np.eye(3) / (6.0 * math.pi * eta * a)
            else:
                d = Yb[i] - Yb[j]
                d = d - L * np.round(d / L)
                Mb[3 * i:3 * i + 3, 3 * j:3 * j + 3] = cf.fcm_pair_mobility(d[None, :], a, eta)[0][0]
    return Mb


def rigid_broyden(apply_vf, Y, body_off, X, L, ft, tol, max_iter, a=1.0, eta=1.0, x0=None, precond="diagonal"):
    """The rigid-body mobility problem by ``broyden``.

    ``apply_vf(F)`` returns V = M^VF F for F of shape (N, 3). Returns (F, W, iterations,
    relative residual norms), W rows (U_b, Gamma_b). precond: "diagonal" starts from the Jacobian
    of the diagonal mobility mu I (the paper's choice); "body" from the Jacobian of the
    block-diagonal mobility that keeps each body's own free-space FCM interactions
    (``body_mobility``) and drops those between bodies, J0 = [[M_bb / mu, -K], [K^T, 0]] per body.
    """
    r = lever_arms(Y, body_off, X, L)
    n = r.shape[0]
    nb = len(body_off) - 1
    mu = 1.0 / (6.0 * math.pi * eta * a)
    ft = np.asarray(ft, dtype=np.float64).reshape(nb, 6)
    # K^T K per body: [[n I, -[S]x], [[S]x, sum(|r|^2 I - r r^T)]], S = sum r
    G = []
    for b in range(nb):
        rb = r[body_off[b]:body_off[b + 1]]
        S = rb.sum(axis=0)
        Sx = np.array([[0.0, -S[2], S[1]], [S[2], 0.0, -S[0]], [-S[1], S[0], 0.0]])
        inertia = (rb * rb).sum() * np.eye(3) - rb.T @ rb
        G.append(np.block([[len(rb) * np.eye(3), -Sx], [Sx, inertia]]))

    def rigid_velocity(What, b, rb):
        return What[b, :3][None, :] + np.cross(What[b, 3:][None, :], rb)

    def residual(x):
        F = x[:3 * n].reshape(n, 3)
        What = x[3 * n:].reshape(nb, 6)
        V = apply_vf(F)
        R1 = np.empty((n, 3))
        R2 = np.empty((nb, 6))
        for b in range(nb):
            sl = slice(body_off[b], body_off[b + 1])
            rb = r[sl]
            R1[sl] = V[sl] / mu - rigid_velocity(What, b, rb)
            R2[b, :3] = F[sl].sum(axis=0) - ft[b, :3]
            R2[b, 3:] = np.cross(rb, F[sl]).sum(axis=0) - ft[b, 3:]
        return np.concatenate([R1.ravel(), R2.ravel()])

    if precond == "body":
        blocks = []
        for b in range(nb):
            sl = slice(body_off[b], body_off[b + 1])
            Kb = constraint_matrix(Y[sl], np.array([0, body_off[b + 1] - body_off[b]]), X[b:b + 1], L)
            Ab = np.block([[body_mobility(Y[sl], L, a, eta) / mu, -Kb], [Kb.T, np.zeros((6, 6))]])
            blocks.append(np.linalg.inv(Ab))

    def precond_body(v):
        r1 = v[:3 * n].reshape(n, 3)
        r2 = v[3 * n:].reshape(nb, 6)
        F = np.empty((n, 3))
        What = np.empty((nb, 6))
        for b in range(nb):
            sl = slice(body_off[b], body_off[b + 1])
            sol = blocks[b] @ np.concatenate([r1[sl].ravel(), r2[b]])
            F[sl] = sol[:-6].reshape(-1, 3)
            What[b] = sol[-6:]
        return np.concatenate([F.ravel(), What.ravel()])

    def precond_diag(v):
        # J0^-1 (r1, r2): W = (K^T K)^-1 (r2 - K^T r1), F = r1 + K W
        r1 = v[:3 * n].reshape(n, 3)
        r2 = v[3 * n:].reshape(nb, 6)
        F = np.empty((n, 3))
        What = np.empty((nb, 6))
        for b in range(nb):
            sl = slice(body_off[b], body_off[b + 1])
            rb = r[sl]
            kt = np.concatenate([r1[sl].sum(axis=0), np.cross(rb, r1[sl]).sum(axis=0)])
            What[b] = np.linalg.solve(G[b], r2[b] - kt)
            F[sl] = r1[sl] + rigid_velocity(What, b, rb)
        return np.concatenate([F.ravel(), What.ravel()])

    scale = float(np.linalg.norm(ft))
    if x0 is None:
        x0 = np.zeros(3 * n + 6 * nb)
    x, it, norms = broyden(residual, precond_body if precond == "body" else precond_diag, x0, tol * scale, max_iter)
    F = x[:3 * n].reshape(n, 3)
    W = mu * x[3 * n:].reshape(nb, 6)
    rel = [v / scale for v in norms] if scale > 0 else norms
    return F, W, it, rel


def fast_fcm_rigid_broyden(Y, body_off, X, ft, L, M, M_G, Sigma, R_c, tol, max_iter, a=1.0, eta=1.0,
                           precond="diagonal"):
    """``rigid_broyden`` with the fast-FCM oracle product (forces only) as M^VF."""
    def apply_vf(F):
        return fast_fcm_apply(Y, F, None, L, M, M_G, Sigma, R_c, a=a, eta=eta)[0]
    return rigid_broyden(apply_vf, Y, body_off, X, L, ft, tol, max_iter, a=a, eta=eta, precond=precond)
