"""Parameter rules of the oracle: grid window, grid support, cutoff radius. FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* Window (Section 2.1: each kernel occupies M_G x M_G x M_G grid points): the
  M_G consecutive points i_start .. i_start + M_G - 1 per dimension, with
  i_start = floor(Y/h - M_G/2) + 1, i.e. the M_G points nearest to Y.
* Grid support read from a truncation radius: M_G = 2 ceil(c Sigma / h) for a
  kernel truncated at +-c Sigma.
* Cutoff radius (Section 4, "tolerance-related" R_c): the smallest r such that
  for every r' >= r the correction blocks are below ``tol`` relative to the
  single-particle mobilities (VF relative to 1/(6 pi eta a); with torques also
  WT relative to 1/(8 pi eta a^3) and WF relative to their geometric mean).
"""
from __future__ import annotations

import math

import numpy as np

from . import closed_forms as cf


def window_start(Y, h, M_G, inv_h32=None):
    """First grid index of the M_G-point window around coordinate Y (unwrapped, may be < 0):
    floor(Y/h - M_G/2) + 1 (Section 4 places the window; it does not fix a precision).

    The window start is an integer decided by floating point, so a check of an FP32 path takes the
    decision in FP32 like that path: with inv_h32 = fl32(M/L) given, s = fl32(fl32(Y) * inv_h32) and
    the floor of fl32(s - M_G/2). Away from the points where Y/h - M_G/2 is an integer (a particle on
    a grid point, for even M_G) both readings give the same index."""
    if inv_h32 is None:
        return np.floor(np.asarray(Y, dtype=np.float64) / h - 0.5 * M_G).astype(np.int64) + 1
    s = np.asarray(Y, dtype=np.float32) * np.float32(inv_h32)
    return np.floor(s - np.float32(0.5 * M_G)).astype(np.int64) + 1


def support_points(Sigma, h, c=4.0):
    """M_G = 2 ceil(c Sigma / h): the window covering +-c Sigma."""
    return int(2 * math.ceil(c * Sigma / h - 1e-12))


def _block_norms(r, Sigma, Sigma_D, a, eta, torques):
    x = np.zeros((r.size, 3))
    x[:, 0] = r
    vf = np.linalg.norm(cf.correction_VF(x, Sigma, a, eta), ord=2, axis=(-2, -1)) * 6 * math.pi * eta * a
    out = vf
    if torques:
        wt = np.linalg.norm(cf.correction_WT(x, Sigma, Sigma_D, a, eta), ord=2, axis=(-2, -1)) * 8 * math.pi * eta * a ** 3
        wf = np.linalg.norm(cf.correction_WF(x, Sigma, Sigma_D, a, eta), ord=2, axis=(-2, -1))
        wf = wf * math.sqrt(6 * math.pi * eta * a * 8 * math.pi * eta * a ** 3)
        out = np.maximum(out, np.maximum(wt, wf))
    return out


def cutoff_radius(Sigma, tol, Sigma_D=None, a=1.0, eta=1.0, torques=False, r_max=None):
    """Smallest R_c with every normalised correction block < tol for all r >= R_c."""
    Sigma_D = Sigma if Sigma_D is None else Sigma_D
    r_max = 40.0 * max(Sigma, Sigma_D) if r_max is None else r_max
    rs = np.linspace(r_max, 1e-3, 40000)
    vals = _block_norms(rs, Sigma, Sigma_D, a, eta, torques)
    above = np.nonzero(vals >= tol)[0]
    if above.size == 0:
        return 0.0
    i = above[0]
    if i == 0:
        raise ValueError("correction still above tolerance at r_max")
    lo, hi = rs[i], rs[i - 1]   # vals(lo) >= tol > vals(r) for r in (lo, hi]
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if _block_norms(np.array([mid]), Sigma, Sigma_D, a, eta, torques)[0] >= tol:
            lo = mid
        else:
            hi = mid
    return hi
