"""Parameter selection for a fast-FCM system: the autotuner.

The paper sets four parameters per error tolerance (Section 5): the grid
resolution Sigma/dx and the grid support M_G (Section 5.1, Table 1), and the
split Sigma/sigma with the cutoff R_c (Section 5.2, Table 2); Sigma plays the
role of the Ewald splitting parameter and its best value depends on the volume
fraction and on the machine (Section 5.2, Table 3). Here:

* ``support_points``: M_G = 2 ceil(c Sigma / h), a cube window covering
  +-c Sigma. The modified kernel's polynomial factor fattens its tail, so c
  follows the tolerance (measured relative errors of the grid part against a
  converged window: c = 4.2 -> 3e-4, 4.7 -> 4e-5, 5.0 -> 1e-5, 5.5 -> 6e-7,
  6.3 -> 8e-9).
* ``resolution_for``: the smallest Sigma/h for a tolerance (Table 1 rows,
  interpolated in log10 of the tolerance).
* ``cutoff``: the library's host rule fcm_cutoff_radius (one pair's neglected
  block below tol); ``pair_cutoff`` tightens it for the number of neighbours
  whose neglected terms add up.
* ``grid_for``: the smallest FFT-friendly M (2^a 3^b 5^c, even) with Sigma/h >= ratio.
* ``candidates`` / ``choose``: for a system (N, box, tolerance) enumerate
  Sigma/sigma on a ladder, derive (M, M_G, r_c) for each, and rank them with a
  cost model of this library's kernels (per window point, per candidate pair
  test, per grid point); ``choose(measure=...)`` then times the best few on
  the GPU and keeps the fastest. ``TunedCache`` persists choices as JSON.
"""
from __future__ import annotations

import json
import math
import os
import threading

from . import fcm

SQRT_PI = math.sqrt(math.pi)
TRUNCATION = {1e-3: 3.8, 1e-4: 4.5, 1e-5: 5.0, 1e-6: 5.4, 1e-8: 6.3}
# Table 1 of the paper: tolerance -> minimum Sigma/dx, and the grid support printed beside it
RESOLUTION = {1e-2: 0.71, 1e-3: 0.87, 1e-4: 0.99, 1e-6: 1.20, 1e-8: 1.39}
TABLE1_SUPPORT = {1e-2: 8, 1e-3: 9, 1e-4: 10, 1e-6: 12, 1e-8: 14}
# Cost model coefficients (seconds) measured on GB300 with this library's FP32 kernels:
# spread + gather per (particle, window point), pair test per candidate, FFT solve per grid point,
# and a fixed cost per apply (launches and small kernels).
COST = {"point": 3.5e-12, "candidate": 4.8e-12, "grid": 4.8e-11, "fixed": 6.0e-5}
SIGMA_D_STANDARD = 1.0 / (6.0 * SQRT_PI) ** (1.0 / 3.0)   # sigma_D / a
# The tolerance is split evenly: the grid part (resolution and window truncation) gets tol/2 and
# the neglected pair terms tol/2. Against the direct Fourier sum (N = 250, phi = 5% and 20%,
# tol = 1e-3..1e-5, the four cheapest candidates) the worst mean relative error was 0.82 tol.
GRID_SHARE = 0.5
SIGMA_LADDER = (1.0, 1.25, 1.5, 1.75, 2.0, 2.5, 3.0, 3.5, 4.0, 5.0, 6.0)


def support_points(Sigma: float, h: float, c: float = 4.8) -> int:
    return int(2 * math.ceil(c * Sigma / h - 1e-12))


def truncation_for(tol: float) -> float:
    """Window half-width in units of Sigma whose truncation error stays below tol."""
    for key in sorted(TRUNCATION, reverse=True):   # 1e-3, 1e-4, ...
        if key <= tol:
            return TRUNCATION[key]
    return TRUNCATION[min(TRUNCATION)]


def standard_support(tol: float, width_over_h: float) -> int:
    """M_G for standard FCM (Sigma = sigma: the plain Gaussian, no modified-kernel tail) at tol: the
    half-width c = M_G dx / (2 Sigma) of Table 1's row for the tolerance (the row with the largest
    error at or below tol), kept for the kernel width the grid resolves. The printed pairs reach the
    printed error with the plain Gaussian down to the 1e-6 row (they floor near 4e-7 at the 1e-8
    row), and the pair-free standard method gives the whole tolerance to the grid."""
    keys = sorted(TABLE1_SUPPORT, reverse=True)           # 1e-2, 1e-3, ...
    row = next((k for k in keys if k <= tol), keys[-1])
    c = TABLE1_SUPPORT[row] / (2.0 * RESOLUTION[row])
    return int(2 * math.ceil(c * width_over_h - 1e-12))


def resolution_for(tol: float) -> float:
    """Smallest Sigma/h reaching tol, interpolated in log10(tol) between the Table 1 rows."""
    keys = sorted(RESOLUTION)
    if tol <= keys[0]:
        return RESOLUTION[keys[0]]
    if tol >= keys[-1]:
        return RESOLUTION[keys[-1]]
    lt = math.log10(tol)
    for lo, hi in zip(keys, keys[1:]):
        if lo <= tol <= hi:
            f = (lt - math.log10(lo)) / (math.log10(hi) - math.log10(lo))
            return RESOLUTION[lo] + f * (RESOLUTION[hi] - RESOLUTION[lo])
    return RESOLUTION[keys[-1]]


def cutoff(Sigma: float, tol: float, torques: bool = True, Sigma_D: float = 0.0) -> float:
    return fcm.cutoff_radius(Sigma, tol, Sigma_D=Sigma_D, torques=torques)


def pair_cutoff(Sigma: float, tol: float, rho: float, torques: bool = True) -> float:
    """r_c for a system of number density rho such that the neglected pair terms stay below tol/2
    in the paper's mean relative particle error.

    ``cutoff`` bounds a single pair's neglected block relative to the self mobility; the
    neglected terms of the nb ~ (4 pi/3) rho r_c^3 neighbours near the cutoff add with random
    signs. Measured against the direct Fourier sum (random suspensions, phi = 2-20%,
    Sigma/sigma = 1.5-4) the mean error was at most 0.6 sqrt(nb) times the per-pair
    tolerance, so the per-pair tolerance is tol / (2 max(1, 0.6 sqrt(nb))), iterated because
    nb grows with r_c."""
    tol_c = 0.5 * tol
    rc = cutoff(Sigma, tol_c, torques)
    for _ in range(4):
        nb = rho * 4.0 * math.pi / 3.0 * rc ** 3
        tol_c = 0.5 * tol / max(1.0, 0.6 * math.sqrt(nb))
        rc_new = cutoff(Sigma, tol_c, torques)
        if abs(rc_new - rc) < 1e-3 * rc:
            return rc_new
        rc = rc_new
    return rc


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


def candidates(n: int, L: float, tol: float, torques: bool = True, a: float = 1.0, max_grid: int = 512,
               min_grid: int = 8, grid: int | None = None):
    """Every admissible parameter set on the Sigma/sigma ladder, with its modelled cost (seconds).
    ``grid`` fixes M (then only Sigma values the grid resolves at tol are admissible)."""
    sg = a / SQRT_PI
    ratio = resolution_for(GRID_SHARE * tol)
    c = truncation_for(GRID_SHARE * tol)
    # standard FCM has no pair error: with forces only the grid takes all of tol (the rotation's
    # derivative kernel needs the finer split resolution when torques act)
    ratio_std = resolution_for(tol if not torques else GRID_SHARE * tol)
    rho = n / L ** 3
    out = []
    for s in SIGMA_LADDER:
        Sigma = s * sg
        standard = s == 1.0
        # standard FCM resolves the narrower rotlet width sigma_D when torques act
        width = min(Sigma, SIGMA_D_STANDARD * a) if (standard and torques) else Sigma
        need = ratio_std if standard else ratio
        if grid is not None:
            M = int(grid)
            if width / (L / M) < need:
                continue
        else:
            M = max(grid_for(L, width, need), grid_for(L, L, min_grid))
        if M > max_grid:
            continue
        h = L / M
        MG = min(standard_support(tol, Sigma / h) if standard else support_points(Sigma, h, c), M)
        if MG > 24:
            continue
        rc = 0.0 if standard else pair_cutoff(Sigma, tol, rho, torques)
        if rc > 0.5 * L:
            continue
        # pair cells as the library builds them: side max(r_c, (8 / rho)^(1/3)), at least 3 per side
        m = max(int(L / max(rc, (8.0 / rho) ** (1.0 / 3.0))), 3) if rc > 0 else 0
        cand = 27.0 * rho * (L / m) ** 3 if m else 0.0
        cost = (COST["point"] * n * MG ** 3 + COST["candidate"] * n * cand + COST["grid"] * M ** 3
                + COST["fixed"])
        out.append({"Sigma": Sigma, "Sigma_over_sigma": s, "M": M, "M_G": MG, "r_c": rc, "h": h,
                    "cost_model_s": cost})
    out.sort(key=lambda d: d["cost_model_s"])
    return out


def choose(n: int, L: float, tol: float = 1e-5, torques: bool = True, measure=None, top: int = 3,
           max_grid: int = 512, min_grid: int = 8, grid: int | None = None):
    """Best parameter set for a system. ``measure(params) -> seconds`` (optional) times the ``top``
    candidates of the cost model and keeps the fastest."""
    cands = candidates(n, L, tol, torques, max_grid=max_grid, min_grid=min_grid, grid=grid)
    if not cands:
        raise ValueError("no admissible fast-FCM parameters for this system")
    if measure is None:
        return dict(cands[0], measured_s=None)
    best = None
    for c in cands[:top]:
        t = measure(c)
        if best is None or t < best["measured_s"]:
            best = dict(c, measured_s=t)
    return best


def make_params(choice, L, n_max, precision=fcm.FCM_FP32, a=1.0):
    """libfcm parameters for a choice returned by ``choose``/``candidates`` (fast FCM: Sigma_D = Sigma;
    standard FCM: Sigma_D = sigma_D and no pair correction)."""
    standard = choice["Sigma_over_sigma"] == 1.0
    return fcm.make_params(L, choice["M"], choice["Sigma"], choice["r_c"] or 1.0, choice["M_G"], n_max,
                           precision, a=a, Sigma_D=SIGMA_D_STANDARD * a if standard else 0.0)


class TunedCache:
    """Tuned parameter sets persisted as JSON, keyed by (N bucket, box, tolerance, torques)."""

    def __init__(self, path: str):
        self.path = path
        self._lock = threading.Lock()
        self._data = {}
        if os.path.exists(path):
            with open(path) as f:
                self._data = json.load(f)

    @staticmethod
    def key(n, L, tol, torques):
        nb = 1 << max(0, int(math.ceil(math.log2(max(n, 1)))))
        return f"n{nb}_L{L:.3f}_tol{tol:.0e}_t{int(bool(torques))}"

    def get(self, n, L, tol, torques):
        with self._lock:
            return self._data.get(self.key(n, L, tol, torques))

    def put(self, n, L, tol, torques, params):
        with self._lock:
            self._data[self.key(n, L, tol, torques)] = params
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self._data, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)


def gpu_timer(pos, F, T, L, device=0, reps=5, warmup=2, precision=fcm.FCM_FP32):
    """``measure`` callback for ``choose``: the mean time of one fcm_apply (seconds) for a
    candidate, on torch CUDA tensors pos, F, T of shape (n, 3), timed with CUDA events on the
    launching stream after ``warmup`` untimed applies."""
    import torch

    n = pos.shape[0]
    U = torch.empty_like(F)
    W = torch.empty_like(F) if T is not None else None
    stream = torch.cuda.current_stream(device)

    def measure(choice):
        with fcm.Handle(make_params(choice, L, n, precision), device) as h:
            for _ in range(warmup):
                h.apply(n, pos, F, T, U, W, stream.cuda_stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                h.apply(n, pos, F, T, U, W, stream.cuda_stream)
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1) * 1e-3 / reps

    return measure
