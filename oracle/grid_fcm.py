"""Grid-based FCM and fast FCM mobility product, FP64 numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Standard FCM (Section 2.1) and the grid part of fast FCM (Section 3.1, Section
3.4 and the algorithm of Section 4) share the same three steps:

1. spread (J~^dagger + N~^dagger): on grid points x_g = (i h_x, j h_y, k h_z),
       f(x_g) = sum_n F_n Delta~(x_g - Y_n; Sigma) - (1/2) T_n x grad Delta(x_g - Y_n; Sigma_D)
   over each particle's M_G^3 window (params.window_start), with the modified
   kernel Delta~ = (1 + dd/2 nabla^2) Delta(.; Sigma) (Section 3); for standard
   FCM Sigma = sigma, Sigma_D = sigma_D and Delta~ = Delta;
2. inverse Stokes operator L^-1 (Section 2.1 step 2): unnormalised FFT,
   u_k = (I - k^ k^) f_k / (eta k^2), inverse FFT divided by M; the k = 0 mode
   and every mode on a Nyquist plane (index M_i/2 of an even M_i) are set to 0;
   the transforms are the oracle's own mixed-radix Cooley-Tukey DFT (``fft``);
3. interpolate (J~ + N~) with the trapezoidal rule (Section 2.1 step 3):
       U_n = h^3 sum_g u(x_g) Delta~(x_g - Y_n; Sigma)
       W_n = h^3 sum_g Delta(x_g - Y_n; Sigma_D) (d_g x u(x_g)) / (2 Sigma_D^2),  d_g = x_g - Y_n
   the second line is (1/2) int (curl u) Delta after one integration by parts,
   which makes it the exact adjoint of the torque spread in step 1.

Fast FCM then adds the pairwise correction of Section 4 (step 6): for every pair
with minimum-image separation r < R_c the correction blocks of
``closed_forms``, plus the Appendix B self correction for every particle.
"""
from __future__ import annotations

import math

import numpy as np

from . import closed_forms as cf
from . import fft as offt
from .params import window_start

try:
    from scipy.spatial import cKDTree
except Exception:  # pragma: no cover
    cKDTree = None


def _as3(v, dtype=np.float64):
    return np.broadcast_to(np.asarray(v, dtype=dtype), (3,)).copy()


def wrap(Y, L):
    """Positions wrapped into [0, L) per dimension."""
    L = _as3(L)
    Yw = np.asarray(Y, dtype=np.float64) - L * np.floor(np.asarray(Y, dtype=np.float64) / L)
    return np.where(Yw >= L, Yw - L, Yw)


def _windows(Yc, L, M, M_G, fp32_windows=False):
    """Per dimension: wrapped indices (P, M_G) and displacements x_g - Y (P, M_G). With fp32_windows
    the window start is decided in FP32 (params.window_start), as an FP32 path decides it."""
    h = L / M
    idx, dsp = [], []
    for d in range(3):
        inv = np.float32(M[d] / L[d]) if fp32_windows else None
        i0 = window_start(Yc[:, d], h[d], M_G, inv)
        ii = i0[:, None] + np.arange(M_G)[None, :]
        dsp.append(ii * h[d] - Yc[:, d][:, None])
        idx.append(np.mod(ii, M[d]))
    return idx, dsp


def _kernel_values(dsp, Sigma, Sigma_D, sigma):
    """Delta~(d; Sigma) and Delta(d; Sigma_D) on the (P, M_G, M_G, M_G) window."""
    dx, dy, dz = dsp
    r2 = dx[:, :, None, None] ** 2 + dy[:, None, :, None] ** 2 + dz[:, None, None, :] ** 2
    dd = sigma * sigma - Sigma * Sigma
    g = (2 * math.pi * Sigma ** 2) ** -1.5 * np.exp(-r2 / (2 * Sigma ** 2))
    lap_g = (r2 / Sigma ** 4 - 3.0 / Sigma ** 2) * g        # nabla^2 Delta(.; Sigma)
    g_mod = g + 0.5 * dd * lap_g
    gD = (2 * math.pi * Sigma_D ** 2) ** -1.5 * np.exp(-r2 / (2 * Sigma_D ** 2))
    return g_mod, gD


def _flat(idx, M):
    ix, iy, iz = idx
    return ((ix[:, :, None, None] * M[1] + iy[:, None, :, None]) * M[2] + iz[:, None, None, :])


def spread(Y, F, T, L, M, M_G, Sigma, Sigma_D, a=1.0, chunk=512, fp32_windows=False):
    """Force density on the grid, shape (3, M_x, M_y, M_z). fp32_windows: window starts decided in
    FP32 (for checking an FP32 path on particles that sit on grid points)."""
    L, M = _as3(L), _as3(M, np.int64)
    Yw = wrap(Y, L)
    n = Yw.shape[0]
    sigma = cf.fcm_sigma(a)
    size = int(np.prod(M))
    f = np.zeros((3, size))
    for s in range(0, n, chunk):
        Yc = Yw[s:s + chunk]
        idx, dsp = _windows(Yc, L, M, M_G, fp32_windows)
        g_mod, gD = _kernel_values(dsp, Sigma, Sigma_D, sigma)
        flat = _flat(idx, M).ravel()
        Fc = np.asarray(F[s:s + chunk], dtype=np.float64)
        vals = [Fc[:, c, None, None, None] * g_mod for c in range(3)]
        if T is not None:
            Tc = np.asarray(T[s:s + chunk], dtype=np.float64)
            dx = dsp[0][:, :, None, None]
            dy = dsp[1][:, None, :, None]
            dz = dsp[2][:, None, None, :]
            # -(1/2) T x grad Delta_D with grad Delta_D = -d Delta_D / Sigma_D^2
            w = gD / (2.0 * Sigma_D ** 2)
            tx, ty, tz = (Tc[:, c, None, None, None] for c in range(3))
            vals[0] = vals[0] + w * (ty * dz - tz * dy)
            vals[1] = vals[1] + w * (tz * dx - tx * dz)
            vals[2] = vals[2] + w * (tx * dy - ty * dx)
        for c in range(3):
            f[c] += np.bincount(flat, weights=np.broadcast_to(vals[c], g_mod.shape).ravel(), minlength=size)
    return f.reshape(3, *M)


def wavevectors(L, M):
    """Spectral k per grid mode; index i maps to i if i <= M/2 else i - M."""
    L, M = _as3(L), _as3(M, np.int64)
    ks = [2 * math.pi * offt.mode_numbers(int(M[d])) / L[d] for d in range(3)]
    return np.meshgrid(*ks, indexing="ij")


def solve_keep_mask(M):
    """Modes kept by the Stokes solve: every mode but k = 0 and those on a Nyquist plane (index M_i/2
    of an even M_i)."""
    M = _as3(M, np.int64)
    n = [offt.mode_numbers(int(M[d])) for d in range(3)]
    nx, ny, nz = np.meshgrid(*n, indexing="ij")
    keep = (nx != 0) | (ny != 0) | (nz != 0)
    for d, nd in enumerate((nx, ny, nz)):
        if M[d] % 2 == 0:
            keep &= np.abs(nd) != M[d] // 2
    return keep


def stokes_solve(f, L, eta=1.0):
    """u = L^-1 f on the periodic grid (Section 2.1 step 2), zero k = 0 and Nyquist modes."""
    M = np.array(f.shape[1:], dtype=np.int64)
    kx, ky, kz = wavevectors(L, M)
    k2 = kx * kx + ky * ky + kz * kz
    keep = solve_keep_mask(M)
    fh = offt.dftn(f)
    inv_k2 = np.where(keep, 1.0 / np.where(keep, k2, 1.0), 0.0)
    kdotf = (kx * fh[0] + ky * fh[1] + kz * fh[2]) * inv_k2
    uh = np.stack([fh[0] - kx * kdotf, fh[1] - ky * kdotf, fh[2] - kz * kdotf]) * (inv_k2 / eta)
    return np.real(offt.idftn(uh))


def interpolate(u, Y, L, M_G, Sigma, Sigma_D, a=1.0, chunk=512):
    """Particle (U, W) from the grid velocity (Section 2.1 step 3, with N~ as in the module doc)."""
    M = np.array(u.shape[1:], dtype=np.int64)
    L = _as3(L)
    h3 = float(np.prod(L / M))
    Yw = wrap(Y, L)
    n = Yw.shape[0]
    sigma = cf.fcm_sigma(a)
    uf = u.reshape(3, -1)
    U = np.zeros((n, 3))
    W = np.zeros((n, 3))
    for s in range(0, n, chunk):
        Yc = Yw[s:s + chunk]
        idx, dsp = _windows(Yc, L, M, M_G)
        g_mod, gD = _kernel_values(dsp, Sigma, Sigma_D, sigma)
        flat = _flat(idx, M)
        ux, uy, uz = uf[0][flat], uf[1][flat], uf[2][flat]
        ax = (1, 2, 3)
        U[s:s + chunk, 0] = h3 * np.sum(g_mod * ux, axis=ax)
        U[s:s + chunk, 1] = h3 * np.sum(g_mod * uy, axis=ax)
        U[s:s + chunk, 2] = h3 * np.sum(g_mod * uz, axis=ax)
        dx = dsp[0][:, :, None, None]
        dy = dsp[1][:, None, :, None]
        dz = dsp[2][:, None, None, :]
        w = gD / (2.0 * Sigma_D ** 2)
        W[s:s + chunk, 0] = h3 * np.sum(w * (dy * uz - dz * uy), axis=ax)
        W[s:s + chunk, 1] = h3 * np.sum(w * (dz * ux - dx * uz), axis=ax)
        W[s:s + chunk, 2] = h3 * np.sum(w * (dx * uy - dy * ux), axis=ax)
    return U, W


def neighbour_pairs(Yw, L, R_c):
    """All unordered pairs (i < j) with minimum-image distance < R_c, and their x_ij = Y_i - Y_j."""
    L = _as3(L)
    n = Yw.shape[0]
    if n < 2:
        return np.zeros((0, 2), dtype=np.int64), np.zeros((0, 3))
    if cKDTree is not None:
        tree = cKDTree(Yw, boxsize=L)
        pairs = tree.query_pairs(R_c, output_type="ndarray").astype(np.int64)
    else:  # brute force
        ii, jj = np.triu_indices(n, 1)
        pairs = np.stack([ii, jj], axis=1)
    if pairs.size == 0:
        return np.zeros((0, 2), dtype=np.int64), np.zeros((0, 3))
    x = Yw[pairs[:, 0]] - Yw[pairs[:, 1]]
    x = x - L * np.round(x / L)
    r = np.linalg.norm(x, axis=1)
    keep = r < R_c
    return pairs[keep], x[keep]


def pair_correction(Y, F, T, L, R_c, Sigma, Sigma_D, a=1.0, eta=1.0, chunk=200000):
    """Sum over pairs r < R_c of (M - M~)(F, T), plus the self correction (Section 4 step 6, Appendix B)."""
    L = _as3(L)
    Yw = wrap(Y, L)
    n = Yw.shape[0]
    F = np.asarray(F, dtype=np.float64)
    U = np.zeros((n, 3))
    W = np.zeros((n, 3))
    U += cf.self_correction_VF(Sigma, a, eta) * F
    if T is not None:
        T = np.asarray(T, dtype=np.float64)
        W += cf.self_correction_WT(Sigma_D, a, eta) * T
    pairs, xs = neighbour_pairs(Yw, L, R_c)
    for s in range(0, pairs.shape[0], chunk):
        p = pairs[s:s + chunk]
        x = xs[s:s + chunk]
        i, j = p[:, 0], p[:, 1]
        r = np.linalg.norm(x, axis=1)
        coincident = r == 0.0
        xs_ = np.where(coincident[:, None], np.array([1.0, 0.0, 0.0]), x)
        vf = cf.correction_VF(xs_, Sigma, a, eta)
        vf[coincident] = cf.self_correction_VF(Sigma, a, eta) * np.eye(3)
        # x_ji = -x_ij: the VF block is even in x
        np.add.at(U, i, np.einsum("pab,pb->pa", vf, F[j]))
        np.add.at(U, j, np.einsum("pab,pb->pa", vf, F[i]))
        if T is not None:
            wf = cf.correction_WF(xs_, Sigma, Sigma_D, a, eta)
            wf[coincident] = 0.0
            wt = cf.correction_WT(xs_, Sigma, Sigma_D, a, eta)
            wt[coincident] = cf.self_correction_WT(Sigma_D, a, eta) * np.eye(3)
            wf_m = -wf                                    # WF block at -x (odd in x)
            vt = np.swapaxes(wf_m, -1, -2)                # VT_ij = (WF_ji)^T, WF_ji = WF(-x)
            vt_m = np.swapaxes(wf, -1, -2)                # VT_ji = (WF_ij)^T
            np.add.at(U, i, np.einsum("pab,pb->pa", vt, T[j]))
            np.add.at(U, j, np.einsum("pab,pb->pa", vt_m, T[i]))
            np.add.at(W, i, np.einsum("pab,pb->pa", wf, F[j]) + np.einsum("pab,pb->pa", wt, T[j]))
            np.add.at(W, j, np.einsum("pab,pb->pa", wf_m, F[i]) + np.einsum("pab,pb->pa", wt, T[i]))
    return U, W


def grid_apply(Y, F, T, L, M, M_G, Sigma, Sigma_D, a=1.0, eta=1.0):
    """The grid part M~ (F, T): spread, Stokes solve, interpolate."""
    f = spread(Y, F, T, L, M, M_G, Sigma, Sigma_D, a)
    u = stokes_solve(f, L, eta)
    return interpolate(u, Y, L, M_G, Sigma, Sigma_D, a)


def standard_fcm_apply(Y, F, T, L, M, M_G, a=1.0, eta=1.0):
    """Standard FCM (Section 2.1): the grid algorithm with sigma, sigma_D and no correction."""
    return grid_apply(Y, F, T, L, M, M_G, cf.fcm_sigma(a), cf.fcm_sigma_D(a), a, eta)


def fast_fcm_apply(Y, F, T, L, M, M_G, Sigma, R_c, Sigma_D=None, a=1.0, eta=1.0):
    """Fast FCM (Section 4): grid part with the modified kernels plus the pairwise correction.

    Requires R_c <= min(L)/2 so that each pair is met once under the minimum image.
    """
    Sigma_D = Sigma if Sigma_D is None else Sigma_D
    if R_c > 0.5 * float(np.min(_as3(L))) + 1e-12:
        raise ValueError("R_c must not exceed half the box")
    Ug, Wg = grid_apply(Y, F, T, L, M, M_G, Sigma, Sigma_D, a, eta)
    Up, Wp = pair_correction(Y, F, T, L, R_c, Sigma, Sigma_D, a, eta)
    return Ug + Up, Wg + Wp


def pair_correction_subset(Y, F, T, L, R_c, Sigma, Sigma_D, idx, a=1.0, eta=1.0):
    """Rows ``idx`` of :func:`pair_correction`, each computed on its own from the
    particles within R_c of it (used to check large systems on sampled particles)."""
    L = _as3(L)
    Yw = wrap(Y, L)
    F = np.asarray(F, dtype=np.float64)
    idx = np.asarray(idx, dtype=np.int64)
    U = cf.self_correction_VF(Sigma, a, eta) * F[idx]
    W = np.zeros((idx.size, 3))
    if T is not None:
        T = np.asarray(T, dtype=np.float64)
        W = W + cf.self_correction_WT(Sigma_D, a, eta) * T[idx]
    tree = cKDTree(Yw, boxsize=L)
    for row, i in enumerate(idx):
        nb = np.array(tree.query_ball_point(Yw[i], R_c), dtype=np.int64)
        nb = nb[nb != i]
        if nb.size == 0:
            continue
        x = Yw[i][None, :] - Yw[nb]
        x = x - L * np.round(x / L)
        r = np.linalg.norm(x, axis=1)
        keep = r < R_c
        nb, x, r = nb[keep], x[keep], r[keep]
        if nb.size == 0:
            continue
        coincident = r == 0.0
        xs_ = np.where(coincident[:, None], np.array([1.0, 0.0, 0.0]), x)
        vf = cf.correction_VF(xs_, Sigma, a, eta)
        vf[coincident] = cf.self_correction_VF(Sigma, a, eta) * np.eye(3)
        U[row] += np.einsum("pab,pb->a", vf, F[nb])
        if T is not None:
            wf = cf.correction_WF(xs_, Sigma, Sigma_D, a, eta)
            wf[coincident] = 0.0
            wt = cf.correction_WT(xs_, Sigma, Sigma_D, a, eta)
            wt[coincident] = cf.self_correction_WT(Sigma_D, a, eta) * np.eye(3)
            vt = np.swapaxes(-wf, -1, -2)
            U[row] += np.einsum("pab,pb->a", vt, T[nb])
            W[row] += np.einsum("pab,pb->a", wf, F[nb]) + np.einsum("pab,pb->a", wt, T[nb])
    return U, W
