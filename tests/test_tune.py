"""The autotuner: its rules against the paper's tables, and its choices against the oracle.

A tuned parameter set must reach the requested tolerance: the fast-FCM oracle
run with the chosen (Sigma, M, M_G, r_c) is compared with the direct Fourier
sum of the exact FCM mobility (no grid, no cutoff), with the paper's error
measure (mean relative particle error, Section 5).
"""
import math

import numpy as np
import pytest

from oracle import grid_fcm as g
from oracle import params as pr
from oracle import spectral_sum as ss
from paper_2310_12651_gb300 import inputs, tune


def _golden_rows(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    rows = []
    for line in open(path):
        line = line.split("#")[0].strip()
        if line:
            rows.append(line.split())
    return rows


def test_resolution_rule_reproduces_table1_rows():
    for eps, ratio, _ in _golden_rows("table1_grid_resolution.txt"):
        assert tune.resolution_for(float(eps)) == pytest.approx(float(ratio), abs=1e-12)
    # monotone between the rows, clamped outside them
    tols = np.logspace(-9, -1, 40)
    vals = [tune.resolution_for(t) for t in tols]
    assert all(a >= b for a, b in zip(vals, vals[1:]))
    assert tune.resolution_for(1e-12) == tune.resolution_for(1e-8)
    assert tune.resolution_for(0.5) == tune.resolution_for(1e-2)


def test_cutoff_rule_is_the_oracle_rule():
    for Sigma in (1.2, 2.0, 3.0):
        for tol in (1e-4, 1e-6):
            assert tune.cutoff(Sigma, tol) == pytest.approx(pr.cutoff_radius(Sigma, tol, torques=True), rel=1e-6)


def test_grid_sizes_are_fft_friendly_and_resolve_sigma():
    for L in (20.0, 57.3, 176.4):
        for Sigma in (0.6, 1.1, 2.3):
            for ratio in (0.9, 1.1, 1.3):
                M = tune.grid_for(L, Sigma, ratio)
                assert M % 2 == 0 and Sigma / (L / M) >= ratio - 1e-12
                m = M
                for p in (2, 3, 5):
                    while m % p == 0:
                        m //= p
                assert m == 1


@pytest.mark.parametrize("n,phi,tol", [(65536, 0.05, 1e-5), (2000, 0.2, 1e-4), (200000, 0.01, 1e-6)])
def test_candidates_are_admissible_and_ranked(n, phi, tol):
    L = inputs.box_edge(n, phi)
    cands = tune.candidates(n, L, tol)
    assert cands
    costs = [c["cost_model_s"] for c in cands]
    assert costs == sorted(costs)
    for c in cands:
        standard = c["Sigma_over_sigma"] == 1.0
        width = c["Sigma"] if not standard else tune.SIGMA_D_STANDARD
        assert min(c["Sigma"], width) / c["h"] >= tune.resolution_for(tune.GRID_SHARE * tol) - 1e-12
        assert c["M_G"] % 2 == 0 and c["M_G"] <= min(24, c["M"])
        if standard:
            # standard FCM keeps the truncation of Table 1's row for the tolerance (plain Gaussian)
            assert c["r_c"] == 0.0
            assert c["M_G"] == tune.standard_support(tol, c["Sigma"] / c["h"])
        else:
            assert c["M_G"] * c["h"] >= 2 * tune.truncation_for(tol) * c["Sigma"] - 1e-9
            assert 0 < c["r_c"] <= L / 2
    # a dilute system prefers a wider Sigma than a dense one (Section 5.2, Table 3)
    if phi <= 0.01:
        assert tune.choose(n, L, tol)["Sigma_over_sigma"] >= 3.0


def test_standard_support_follows_table1():
    """At Table 1's own resolution the standard-FCM support is the printed M_G (odd rows rounded up to
    an even window), and it grows with the resolved width's points per h."""
    for eps, ratio, MG in _golden_rows("table1_grid_resolution.txt"):
        got = tune.standard_support(float(eps), float(ratio))
        assert got == int(MG) + (int(MG) % 2)
    assert tune.standard_support(1e-4, 2.0) > tune.standard_support(1e-4, 0.99)
    assert tune.standard_support(3e-5, 1.0) == tune.standard_support(1e-6, 1.0)   # the next tighter row


def test_choose_with_measurement_keeps_the_fastest():
    L = inputs.box_edge(65536, 0.05)
    cands = tune.candidates(65536, L, 1e-5)
    def measure(c):
        return 1.0 / c["Sigma"]  # pretend wider kernels are faster
    best = tune.choose(65536, L, 1e-5, measure=measure, top=3)
    assert best["Sigma"] == max(c["Sigma"] for c in cands[:3])
    assert best["measured_s"] == pytest.approx(1.0 / best["Sigma"])
    assert tune.choose(65536, L, 1e-5)["measured_s"] is None


@pytest.fixture(scope="module", params=[0.2, 0.05])
def suspension(request):
    n, phi = 250, request.param
    L = inputs.box_edge(n, phi)
    Y = inputs.random_suspension(n, L, inputs.BASE_SEED + 40)
    F, T = inputs.random_loads(n, inputs.BASE_SEED + 41)
    Ub, Wb = ss.apply(Y, F, T, L)
    return n, L, Y, F, T, Ub, Wb


@pytest.mark.slow
@pytest.mark.parametrize("tol", [1e-3, 1e-4])
def test_chosen_parameters_reach_the_tolerance(suspension, tol):
    """The three cheapest candidates (and standard FCM) reach tol in U and W."""
    n, L, Y, F, T, Ub, Wb = suspension
    cands = tune.candidates(n, L, tol, max_grid=96)
    picked = cands[:3] + [c for c in cands[3:] if c["Sigma_over_sigma"] == 1.0]
    for c in picked:
        if c["Sigma_over_sigma"] == 1.0:
            U, W = g.standard_fcm_apply(Y, F, T, L, c["M"], c["M_G"])
        else:
            U, W = g.fast_fcm_apply(Y, F, T, L, c["M"], c["M_G"], c["Sigma"], c["r_c"])
        eu = np.mean(np.linalg.norm(U - Ub, axis=1) / np.linalg.norm(Ub, axis=1))
        ew = np.mean(np.linalg.norm(W - Wb, axis=1) / np.linalg.norm(Wb, axis=1))
        assert eu < tol and ew < tol, (c, eu, ew)


@pytest.mark.slow
@pytest.mark.parametrize("tol", [1e-3, 1e-4, 1e-6])
def test_standard_forces_only_reaches_the_tolerance(suspension, tol):
    """Forces only (the crossover study's setting): standard FCM at Table 1's resolution and support
    for the whole tolerance reaches it against the direct Fourier sum."""
    n, L, Y, F, T, Ub, Wb = suspension
    Ub, _ = ss.apply(Y, F, None, L)
    std = [c for c in tune.candidates(n, L, tol, torques=False, max_grid=160) if c["Sigma_over_sigma"] == 1.0]
    assert std
    U, _ = g.standard_fcm_apply(Y, F, None, L, std[0]["M"], std[0]["M_G"])
    eu = np.mean(np.linalg.norm(U - Ub, axis=1) / np.linalg.norm(Ub, axis=1))
    assert eu < tol, (std[0], eu)


def test_tuned_cache_round_trip(tmp_path):
    path = str(tmp_path / "tuned.json")
    c = tune.TunedCache(path)
    L = inputs.box_edge(65536, 0.05)
    best = tune.choose(65536, L, 1e-5)
    c.put(65536, L, 1e-5, True, best)
    # same N bucket, same key; a fresh cache reads it back from disk
    c2 = tune.TunedCache(path)
    assert c2.get(40000, L, 1e-5, True) == best
    assert c2.get(65536, L, 1e-6, True) is None
    assert c2.get(65536, L, 1e-5, False) is None
    assert tune.TunedCache.key(65536, L, 1e-5, True) != tune.TunedCache.key(65537, L, 1e-5, True)
    assert not math.isnan(best["cost_model_s"])
