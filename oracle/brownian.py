"""Brownian increments of fast FCM by positive splitting, FP64 numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 3.3 shows that the modified kernel splits the mobility positively: both
M~ (the grid part) and M - M~ (the pairwise correction) are symmetric positive
definite, which is what makes Brownian displacements cheap; the conclusion
(Section 7) proposes fluctuating FCM for the grid part and a Lanczos square root
for the pairwise part. A Brownian velocity with covariance 2 kT M is then the sum
of two independent parts:

1. grid part, covariance 2 kT M~. With K the (grid x particle) kernel matrix
   (spread f = K F, interpolation U = h^3 K^T u) and G the discrete inverse
   Stokes operator of ``grid_fcm.stokes_solve``, M~ = h^3 K^T G K. A velocity
   field u_B = sqrt(2 kT / h^3) G^{1/2} xi, with xi white noise on the grid
   (unit variance per point and component), interpolated as in the deterministic
   product, has covariance h^6 K^T (2 kT / h^3) G K = 2 kT M~. G is diagonal in
   Fourier space with the projector (I - k^ k^)/(eta k^2), so its square root is
   (I - k^ k^)/(sqrt(eta) |k|) (the projector is idempotent), with the same zero
   modes (k = 0 and Nyquist planes). The interpolation also yields the rotational
   part, so the grid part covers forces and torques.
2. pair part, covariance 2 kT (M - M~): sqrt(2 kT) (M - M~)^{1/2} z with z
   standard normal, the square root taken exactly here (symmetric eigen-
   decomposition of the dense matrix). Only the force-velocity block: the paper
   proves positive splitting for it and leaves the torque blocks open (Section 7).
"""
from __future__ import annotations

import math

import numpy as np

from . import closed_forms as cf
from . import fft as offt
from .grid_fcm import _as3, interpolate, neighbour_pairs, solve_keep_mask, wavevectors, wrap


def grid_noise_velocity(xi, L, eta=1.0):
    """G^{1/2} xi on the periodic grid: xi (3, M_x, M_y, M_z) real; zero k = 0 and Nyquist modes."""
    M = np.array(xi.shape[1:], dtype=np.int64)
    kx, ky, kz = wavevectors(L, M)
    k2 = kx * kx + ky * ky + kz * kz
    keep = solve_keep_mask(M)
    xh = offt.dftn(xi)
    inv_k2 = np.where(keep, 1.0 / np.where(keep, k2, 1.0), 0.0)
    kdotx = (kx * xh[0] + ky * xh[1] + kz * xh[2]) * inv_k2
    inv_k = np.sqrt(inv_k2)
    uh = np.stack([xh[0] - kx * kdotx, xh[1] - ky * kdotx, xh[2] - kz * kdotx]) * (inv_k / math.sqrt(eta))
    return np.real(offt.idftn(uh))


def brownian_grid(Y, xi, L, M_G, Sigma, Sigma_D, kT, a=1.0, eta=1.0):
    """(U, W) of the grid part for grid noise xi (3, M_x, M_y, M_z): covariance 2 kT M~ over xi."""
    M = np.array(xi.shape[1:], dtype=np.int64)
    h3 = float(np.prod(_as3(L) / M))
    u = math.sqrt(2.0 * kT / h3) * grid_noise_velocity(xi, L, eta)
    return interpolate(u, Y, L, M_G, Sigma, Sigma_D, a)


def pair_correction_matrix(Y, L, R_c, Sigma, a=1.0, eta=1.0):
    """The dense (3n x 3n) force-velocity block of M - M~: self terms (Appendix B) plus the
    correction_VF block of every pair closer than R_c (minimum image)."""
    Yw = wrap(Y, L)
    n = Yw.shape[0]
    A = np.zeros((3 * n, 3 * n))
    for i in range(n):
        A[3 * i:3 * i + 3, 3 * i:3 * i + 3] = cf.self_correction_VF(Sigma, a, eta) * np.eye(3)
    pairs, xs = neighbour_pairs(Yw, L, R_c)
    for (i, j), x in zip(pairs, xs):
        if np.linalg.norm(x) == 0.0:
            blk = cf.self_correction_VF(Sigma, a, eta) * np.eye(3)
        else:
            blk = cf.correction_VF(x[None, :], Sigma, a, eta)[0]
        A[3 * i:3 * i + 3, 3 * j:3 * j + 3] += blk
        A[3 * j:3 * j + 3, 3 * i:3 * i + 3] += blk      # the block is even in x and symmetric
    return A


def matrix_sqrt_spd(A):
    """A^{1/2} of a symmetric positive definite matrix by eigendecomposition; raises otherwise."""
    w, Q = np.linalg.eigh(0.5 * (A + A.T))
    if w.min() <= 0.0:
        raise ValueError(f"matrix not positive definite (smallest eigenvalue {w.min():.3e})")
    return (Q * np.sqrt(w)) @ Q.T


def brownian_pair(Y, z, L, R_c, Sigma, kT, a=1.0, eta=1.0):
    """U of the pair part for standard normal z (n, 3): sqrt(2 kT) (M - M~)^{1/2} z."""
    A = pair_correction_matrix(Y, L, R_c, Sigma, a, eta)
    return math.sqrt(2.0 * kT) * (matrix_sqrt_spd(A) @ np.asarray(z, dtype=np.float64).ravel()).reshape(-1, 3)
