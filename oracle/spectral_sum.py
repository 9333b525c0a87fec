"""Direct periodic Fourier sum of the FCM mobility product, FP64 numpy (tiny N).

TEST INFRASTRUCTURE ONLY (see the package docstring).

For a periodic box of edges L the FCM flow is a Fourier series over the
reciprocal lattice k = 2 pi (n_x/L_x, n_y/L_y, n_z/L_z). With the spreading of
Section 2 and Section 3.4 (force kernel g_F(k) = exp(-sigma^2 k^2/2), torque
kernel g_T(k) = exp(-sigma_D^2 k^2/2), the torque spread as (1/2) curl(T Delta)),
the inverse Stokes operator (I - k k^T/k^2)/(eta k^2) of Appendix A and the
volume averages of eq. avg_particle_vel / avg_particle_rot:

    u_k  = (I - k^ k^)/(eta k^2) sum_m e^{-i k.Y_m} [g_F F_m + g_T (i/2) k x T_m]
    U_n  = (1/V) sum_{k != 0} g_F e^{i k.Y_n} u_k
    W_n  = (1/V) sum_{k != 0} g_T e^{i k.Y_n} (i/2) k x u_k

The k = 0 mode is left out (zero mean flow). With ``Sigma`` given the kernels are
the modified ones, g_F = (1 - dd k^2/2) exp(-Sigma^2 k^2/2) and
g_T = exp(-Sigma_D^2 k^2/2) (Section 3.3), which gives the grid part M~ alone.
"""
from __future__ import annotations

import math

import numpy as np

from .closed_forms import fcm_sigma, fcm_sigma_D


def _kernels(a, Sigma, Sigma_D):
    sg, sd = fcm_sigma(a), fcm_sigma_D(a)
    if Sigma is None:
        return (lambda k2: np.exp(-0.5 * sg * sg * k2)), (lambda k2: np.exp(-0.5 * sd * sd * k2)), sd
    Sigma_D = Sigma if Sigma_D is None else Sigma_D
    dd = sg * sg - Sigma * Sigma
    gF = lambda k2: (1.0 - 0.5 * dd * k2) * np.exp(-0.5 * Sigma * Sigma * k2)
    gT = lambda k2: np.exp(-0.5 * Sigma_D * Sigma_D * k2)
    return gF, gT, Sigma_D


def lattice(L, kmax):
    """All reciprocal lattice vectors with 0 < |k| <= kmax, as (nk, 3)."""
    L = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,))
    nmax = [int(math.floor(kmax * L[d] / (2 * math.pi))) for d in range(3)]
    axes = [np.arange(-nmax[d], nmax[d] + 1) * (2 * math.pi / L[d]) for d in range(3)]
    kx, ky, kz = np.meshgrid(*axes, indexing="ij")
    k = np.stack([kx.ravel(), ky.ravel(), kz.ravel()], axis=1)
    k2 = np.einsum("ij,ij->i", k, k)
    keep = (k2 > 0) & (k2 <= kmax * kmax)
    return k[keep]


def apply(Y, F, T, L, a=1.0, eta=1.0, Sigma=None, Sigma_D=None, tol=1e-16, chunk=20000):
    """(U, W) = M (F, T) by the direct reciprocal-lattice sum.

    ``T`` may be None (forces only; W is then returned for the force part alone).
    The lattice is cut where the product of the two kernels falls below ``tol``.
    """
    Y = np.asarray(Y, dtype=np.float64)
    F = np.asarray(F, dtype=np.float64)
    n = Y.shape[0]
    Tm = np.zeros_like(F) if T is None else np.asarray(T, dtype=np.float64)
    L = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,))
    V = float(np.prod(L))
    gF, gT, sD = _kernels(a, Sigma, Sigma_D)
    smallest = min(fcm_sigma(a) if Sigma is None else Sigma, sD)
    kmax = math.sqrt(-math.log(tol)) / smallest + 1e-9
    if Sigma is not None:  # the polynomial factor widens the support a little
        kmax *= 1.25
    ks = lattice(L, kmax)
    U = np.zeros((n, 3))
    W = np.zeros((n, 3))
    for s in range(0, ks.shape[0], chunk):
        k = ks[s:s + chunk]
        k2 = np.einsum("ij,ij->i", k, k)
        f_, t_ = gF(k2), gT(k2)
        phase = np.exp(-1j * (k @ Y.T))                      # (nk, n): e^{-i k.Y_m}
        src = phase @ F * f_[:, None]                          # sum_m e^{-ik.Y_m} g_F F_m
        src = src + 0.5j * np.cross(k, phase @ Tm) * t_[:, None]
        khat = k / np.sqrt(k2)[:, None]
        uk = (src - khat * np.einsum("ij,ij->i", khat, src)[:, None]) / (eta * k2)[:, None]
        back = np.conj(phase).T                               # (n, nk): e^{+i k.Y_n}
        U += np.real(back @ (uk * f_[:, None]))
        W += np.real(back @ (0.5j * np.cross(k, uk) * t_[:, None]))
    return U / V, W / V


def mobility_matrix(Y, L, a=1.0, eta=1.0, Sigma=None, Sigma_D=None, tol=1e-16, torques=True):
    """The 6N x 6N (or 3N x 3N) matrix of :func:`apply`, one column per unit load."""
    Y = np.asarray(Y, dtype=np.float64)
    n = Y.shape[0]
    dof = 6 * n if torques else 3 * n
    Mx = np.zeros((dof, dof))
    for j in range(dof):
        F = np.zeros((n, 3))
        T = np.zeros((n, 3))
        if j < 3 * n:
            F[j // 3, j % 3] = 1.0
        else:
            T[(j - 3 * n) // 3, (j - 3 * n) % 3] = 1.0
        U, W = apply(Y, F, T if torques else None, L, a, eta, Sigma, Sigma_D, tol)
        Mx[:, j] = np.concatenate([U.ravel(), W.ravel()])[:dof]
    return Mx
