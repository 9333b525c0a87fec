"""Parameter rules for a fast-FCM system (the autotuner's rule layer).

The paper sets four parameters per error tolerance (Section 5): the grid
resolution Sigma/dx and support M_G (Section 5.1), and the split Sigma/sigma
with the cutoff R_c (Section 5.2). Here:

* ``support_points``: M_G = 2 ceil(c Sigma / h), a cube window covering
  +-c Sigma. The modified kernel's polynomial factor fattens its tail, so c is
  chosen from the tolerance (measured relative errors of the grid part against
  a converged window: c = 4.2 -> 3e-4, 4.7 -> 4e-5, 5.0 -> 1e-5, 5.5 -> 6e-7,
  6.3 -> 8e-9).
* ``cutoff``: the library's host rule fcm_cutoff_radius (smallest r beyond
  which every correction block is below the tolerance).
* ``grid_for``: the smallest FFT-friendly M (2^a 3^b 5^c) with Sigma/h >= ratio.
"""
from __future__ import annotations

import math

from . import fcm

TRUNCATION = {1e-3: 3.8, 1e-4: 4.5, 1e-5: 5.0, 1e-6: 5.4, 1e-8: 6.3}


def support_points(Sigma: float, h: float, c: float = 4.8) -> int:
    return int(2 * math.ceil(c * Sigma / h - 1e-12))


def truncation_for(tol: float) -> float:
    """Window half-width in units of Sigma whose truncation error stays below tol."""
    for key in sorted(TRUNCATION, reverse=True):   # 1e-3, 1e-4, ...
        if key <= tol:
            return TRUNCATION[key]
    return TRUNCATION[min(TRUNCATION)]


def cutoff(Sigma: float, tol: float, torques: bool = True, Sigma_D: float = 0.0) -> float:
    return fcm.cutoff_radius(Sigma, tol, Sigma_D=Sigma_D, torques=torques)


def _smooth(m: int) -> bool:
    for p in (2, 3, 5):
        while m % p == 0:
            m //= p
    return m == 1


def grid_for(L: float, Sigma: float, ratio: float) -> int:
    m = max(8, int(math.ceil(L * ratio / Sigma)))
    while not _smooth(m) or m % 2:
        m += 1
    return m
