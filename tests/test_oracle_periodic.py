"""Pins of the periodic oracles (direct Fourier sum, standard and fast FCM grids).

What fixes each expected value:
* Hasimoto's periodic drag constant (tests/golden/hasimoto_constant.txt) and
  the O((a/L)^3) terms that follow from the reciprocal-lattice sum with the k = 0
  mode removed (the sum minus the integral of a smooth kernel is minus the k = 0
  term alone);
* Cholesky of the mobility matrix (positive definiteness, Section 3.3 and 6);
* plane-wave solutions of the Stokes equations for the solver;
* the zeroth and first moments of the spread force density;
* exact equality of the fast and standard algorithms when Sigma = sigma;
* brute-force pair search;
* the paper's printed error tables, as soft pins.
"""
import math
import os

import numpy as np
import pytest

from oracle import closed_forms as cf
from oracle import grid_fcm as g
from oracle import params as pr
from oracle import spectral_sum as ss
from paper_2310_12651_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SG = cf.fcm_sigma()
SD = cf.fcm_sigma_D()


def _golden(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].strip()
        if line:
            rows.append(line.split())
    return rows


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


XI = float(dict(_golden("hasimoto_constant.txt"))["xi"])


@pytest.mark.parametrize("L", [8.0, 12.0, 20.0])
def test_spectral_sum_single_particle_hasimoto(L):
    U, W = ss.apply(np.array([[1.0, 2.0, 3.0]]), np.array([[1.0, 0.0, 0.0]]), np.array([[0.0, 0.0, 1.0]]), L)
    drag = 6 * math.pi * U[0, 0]
    assert abs(drag - (1 - XI / L + 4.0 / L ** 3)) < 5e-7 / L + 1e-11
    assert abs(U[0, 1]) < 1e-14 and abs(U[0, 2]) < 1e-14
    rot = 8 * math.pi * W[0, 2]
    assert abs(rot - (1 - 4 * math.pi / 3 / L ** 3)) < 1e-12


def test_spectral_sum_matrix_spd_and_symmetric():
    Y = inputs.random_suspension(8, 10.0, 11)
    Mx = ss.mobility_matrix(Y, 10.0, torques=True)
    np.testing.assert_allclose(Mx, Mx.T, atol=1e-14)
    np.linalg.cholesky(Mx)


def test_spectral_sum_close_pair_is_free_space_plus_periodic_shift():
    """At separation s << L the periodic pair block is the free-space closed form shifted by the
    periodic self correction, up to O(s^2/L^3)."""
    L = 40.0
    x = np.array([2.3, -1.1, 0.9])
    Y = np.array([[10.0, 10.0, 10.0], [10.0, 10.0, 10.0] + x])
    F = np.array([[0.0, 0.0, 0.0], [0.3, -0.5, 0.8]])
    T = np.array([[0.0, 0.0, 0.0], [0.2, 0.7, -0.4]])
    U, W = ss.apply(Y, F, T, L)
    m = cf.fcm_pair_mobility((Y[0] - Y[1])[None])
    shift_vf = -XI / (6 * math.pi * L)
    expect_U = m[0][0] @ F[1] + m[2][0] @ T[1] + shift_vf * F[1]
    expect_W = m[1][0] @ F[1] + m[3][0] @ T[1]
    s2 = float(x @ x)
    assert np.max(np.abs(U[0] - expect_U)) < 0.2 * s2 / L ** 3
    assert np.max(np.abs(W[0] - expect_W)) < 0.2 * s2 / L ** 3


def _grid(L, width, ratio):
    M = int(math.ceil(L / (width / ratio)))
    return M + (M % 2)


def test_standard_grid_single_particle_hasimoto():
    L = 12.0
    M = _grid(L, SD, 1.6)
    U, W = g.standard_fcm_apply(np.array([[3.3, 7.1, 0.4]]), np.array([[0.0, 1.0, 0.0]]),
                                np.array([[1.0, 0.0, 0.0]]), L, M, 26)
    assert abs(6 * math.pi * U[0, 1] - (1 - XI / L + 4.0 / L ** 3)) < 1e-6
    assert abs(8 * math.pi * W[0, 0] - (1 - 4 * math.pi / 3 / L ** 3)) < 1e-6


def test_standard_grid_matches_spectral_sum():
    L, n = 16.0, 12
    Y = inputs.random_suspension(n, L, 1)
    F, T = inputs.random_loads(n, 2)
    Ub, Wb = ss.apply(Y, F, T, L)
    M = _grid(L, SG, 2.0)
    Ua, Wa = g.standard_fcm_apply(Y, F, T, L, M, 24)
    assert _rel(Ua, Ub) < 2e-8 and _rel(Wa, Wb) < 2e-8


def test_fast_grid_matches_spectral_sum():
    L, n = 16.0, 12
    Y = inputs.random_suspension(n, L, 1)
    F, T = inputs.random_loads(n, 2)
    Ub, Wb = ss.apply(Y, F, T, L)
    Sigma = 0.8
    rc = pr.cutoff_radius(Sigma, 1e-10, torques=True)
    M = _grid(L, Sigma, 2.0)
    Uc, Wc = g.fast_fcm_apply(Y, F, T, L, M, 24, Sigma, rc)
    assert _rel(Uc, Ub) < 5e-8 and _rel(Wc, Wb) < 5e-8


def test_fast_grid_part_matches_modified_spectral_sum():
    """The grid part alone equals the Fourier sum with the modified kernels (Section 3.3)."""
    L, n = 14.0, 10
    Y = inputs.random_suspension(n, L, 5)
    F, T = inputs.random_loads(n, 6)
    Sigma = 1.3
    Ub, Wb = ss.apply(Y, F, T, L, Sigma=Sigma)
    M = _grid(L, Sigma, 2.0)
    Ug, Wg = g.grid_apply(Y, F, T, L, M, 26, Sigma, Sigma)
    assert _rel(Ug, Ub) < 1e-8 and _rel(Wg, Wb) < 1e-8


def test_fast_with_sigma_equal_standard_is_identical():
    L, n = 12.0, 9
    Y = inputs.random_suspension(n, L, 7)
    F, T = inputs.random_loads(n, 8)
    M = 24
    Ua, Wa = g.standard_fcm_apply(Y, F, T, L, M, 12)
    Uc, Wc = g.fast_fcm_apply(Y, F, T, L, M, 12, SG, 1e-9, Sigma_D=SD)
    np.testing.assert_allclose(Uc, Ua, rtol=0, atol=1e-15)
    np.testing.assert_allclose(Wc, Wa, rtol=0, atol=1e-15)


@pytest.mark.parametrize("transverse", [True, False])
def test_stokes_solve_plane_wave(transverse):
    """f = e_x cos(k y) is divergence free: u = f/(eta k^2). f = e_x cos(k x) is a pure gradient: u = 0."""
    L, M, eta = 10.0, 20, 0.7
    x = np.arange(M) * (L / M)
    X, Yg, Z = np.meshgrid(x, x, x, indexing="ij")
    k = 2 * math.pi * 3 / L
    f = np.zeros((3, M, M, M))
    f[0] = np.cos(k * (Yg if transverse else X))
    u = g.stokes_solve(f, L, eta)
    expect = f / (eta * k * k) if transverse else np.zeros_like(f)
    np.testing.assert_allclose(u, expect, atol=1e-12)


@pytest.mark.parametrize("Sigma", [SG, 2.0])
def test_spread_moments(Sigma):
    """h^3 sum f = F and h^3 sum (x_g - Y) x f = T: force and torque transferred to the fluid."""
    L, M = 30.0, 64          # h = 0.47: both widths resolved (Sigma/h >= 1.2)
    h = L / M
    Y = np.array([[13.37, 17.21, 9.05]])
    F = np.array([[0.3, -1.2, 0.5]])
    T = np.array([[0.7, 0.1, -0.9]])
    MG = pr.support_points(Sigma, h, 6.5)
    f = g.spread(Y, F, T, L, M, MG, Sigma, Sigma)
    tot = f.reshape(3, -1).sum(axis=1) * h ** 3
    np.testing.assert_allclose(tot, F[0], atol=1e-8)
    xs = np.arange(M) * h
    X, Yg, Z = np.meshgrid(xs, xs, xs, indexing="ij")
    d = np.stack([X - Y[0, 0], Yg - Y[0, 1], Z - Y[0, 2]])
    d = d - L * np.round(d / L)
    torque = np.cross(d.reshape(3, -1).T, f.reshape(3, -1).T).sum(axis=0) * h ** 3
    np.testing.assert_allclose(torque, T[0], atol=1e-8)


def test_rotation_interpolation_equals_spectral_curl():
    """W = (1/2) h^3 sum (curl u) Delta_D: the integrated-by-parts form equals a spectral curl."""
    L, n = 16.0, 6
    Y = inputs.random_suspension(n, L, 9)
    F, T = inputs.random_loads(n, 10)
    Sigma = 1.2
    M = _grid(L, Sigma, 2.2)
    MG = 26
    f = g.spread(Y, F, T, L, M, MG, Sigma, Sigma)
    u = g.stokes_solve(f, L)
    _, W = g.interpolate(u, Y, L, MG, Sigma, Sigma)
    kx, ky, kz = g.wavevectors(L, M)
    uh = [np.fft.fftn(u[c]) for c in range(3)]
    curl = [np.real(np.fft.ifftn(1j * (ky * uh[2] - kz * uh[1]))),
            np.real(np.fft.ifftn(1j * (kz * uh[0] - kx * uh[2]))),
            np.real(np.fft.ifftn(1j * (kx * uh[1] - ky * uh[0])))]
    h = L / M
    Wc = np.zeros((n, 3))
    xs = np.arange(M) * h
    X, Yg, Z = np.meshgrid(xs, xs, xs, indexing="ij")
    for i in range(n):
        d = np.stack([X - Y[i, 0], Yg - Y[i, 1], Z - Y[i, 2]])
        d = d - L * np.round(d / L)
        D = (2 * math.pi * Sigma ** 2) ** -1.5 * np.exp(-np.sum(d * d, axis=0) / (2 * Sigma ** 2))
        Wc[i] = [0.5 * h ** 3 * np.sum(curl[c] * D) for c in range(3)]
    assert _rel(W, Wc) < 1e-7


def test_fast_operator_symmetric_and_positive():
    L, n = 20.0, 40
    Y = inputs.random_suspension(n, L, 12)
    F1, T1 = inputs.random_loads(n, 13)
    F2, T2 = inputs.random_loads(n, 14)
    Sigma, M, MG = 1.2, 24, 14
    rc = pr.cutoff_radius(Sigma, 1e-6, torques=True)
    U1, W1 = g.fast_fcm_apply(Y, F1, T1, L, M, MG, Sigma, rc)
    U2, W2 = g.fast_fcm_apply(Y, F2, T2, L, M, MG, Sigma, rc)
    a = np.sum(F1 * U2) + np.sum(T1 * W2)
    b = np.sum(F2 * U1) + np.sum(T2 * W1)
    assert abs(a - b) < 1e-13 * (abs(a) + abs(b))
    assert np.sum(F1 * U1) + np.sum(T1 * W1) > 0


def test_neighbour_pairs_brute_force():
    L, n = 15.0, 120
    Yw = g.wrap(inputs.random_suspension(n, L, 15, min_sep=0.5), L)
    pairs, x = g.neighbour_pairs(Yw, L, 5.3)
    got = set(map(tuple, pairs.tolist()))
    want = set()
    for i in range(n):
        for j in range(i + 1, n):
            d = Yw[i] - Yw[j]
            d -= L * np.round(d / L)
            if np.linalg.norm(d) < 5.3:
                want.add((i, j))
    assert got == want
    for (i, j), xv in zip(pairs, x):
        d = Yw[i] - Yw[j]
        d -= L * np.round(d / L)
        np.testing.assert_allclose(xv, d, atol=1e-14)


@pytest.mark.parametrize("MG", [6, 7, 12])
def test_window_is_the_nearest_points(MG):
    rng = np.random.default_rng(16)
    Y = rng.random(2000) * 37.0
    h = 1.3
    i0 = pr.window_start(Y, h, MG)
    d = (i0[:, None] + np.arange(MG)[None, :]) * h - Y[:, None]
    assert np.all(np.abs(d) <= 0.5 * MG * h + 1e-12)
    before = (i0 - 1) * h - Y
    after = (i0 + MG) * h - Y
    # every point outside the window is at least as far as every point inside
    assert np.all(np.minimum(np.abs(before), np.abs(after)) >= np.max(np.abs(d), axis=1) - 1e-12)


@pytest.mark.parametrize("MG", [10, 12, 14])
def test_fp32_window_decision(MG):
    """Window starts decided in FP32 (params.window_start with inv_h32, as an FP32 path decides them)
    equal the FP64 decision away from ties; for a particle on a grid point k (a tie for even M_G)
    either decision is one of the two nearest-point windows, so it holds k at position M_G/2 - 1 or
    M_G/2; and without ties the FP32-decided spread is the FP64-decided one."""
    L, M = 48.0, 40
    h = L / M
    inv = np.float32(M / L)
    rng = np.random.default_rng(17)
    Y = rng.random(20000).astype(np.float32).astype(np.float64) * np.float32(L)
    a, b = pr.window_start(Y, h, MG), pr.window_start(Y, h, MG, inv)
    s = Y / h - 0.5 * MG
    away = np.abs(s - np.round(s)) > 1e-5
    assert np.array_equal(a[away], b[away])
    k = np.arange(4 * M)
    Yk = (k * h).astype(np.float32).astype(np.float64)
    b = pr.window_start(Yk, h, MG, inv)
    assert set(np.unique(b - (k - MG // 2))) <= {0, 1}
    Y3 = np.array([[5.1, 7.7, 30.3], [17.3, 44.9, 2.2], [47.9, 0.05, 23.3]])
    F = np.array([[0.3, -1.1, 0.7], [1.0, 0.2, -0.4], [-0.6, 0.5, 0.9]])
    T = np.array([[0.2, 0.1, -0.3], [-0.5, 0.4, 0.6], [0.7, -0.2, 0.1]])
    f32 = g.spread(Y3, F, T, L, M, MG, 2.0, 1.7, fp32_windows=True)
    f64 = g.spread(Y3, F, T, L, M, MG, 2.0, 1.7)
    assert np.array_equal(f32, f64)


def test_cutoff_rule_against_table2():
    """Our pointwise R_c rule lands on the paper's empirical slopes lambda (Table 2) within 8%."""
    rows = {float(r[0]): [float(v) for v in r[1:]] for r in _golden("table2_cutoff_slope.txt")}
    for eps, lams in rows.items():
        lam = pr.cutoff_radius(2.0, eps) / 2.0
        assert min(lams) * 0.92 <= lam <= max(lams) * 1.08, (eps, lam, lams)


@pytest.mark.slow
def test_grid_error_against_table1():
    """Table 1 (Section 5.1) against the direct Fourier sum, with every pair corrected (R_c = L/2).

    The error is the paper's mean relative particle error. Two readings are pinned:
    * the printed (Sigma/dx, M_G) pairs, M_G consecutive points per direction: the first three rows
      reach the printed error within a factor 2; the 1e-6 and 1e-8 rows cannot, because every printed
      pair truncates the kernel near +-5 Sigma (c = M_G dx / (2 Sigma) = 5.0 ... 5.6), where the
      modified kernel's tail floors the error near 1e-5;
    * the printed Sigma/dx with a window wide enough not to truncate (+-7 Sigma): all five rows
      reach the printed error within a factor 2, so the Sigma/dx column is the resolution the
      tolerance needs, and the M_G column is not a truncation that reaches 1e-6 or 1e-8.
    """
    rows = _golden("table1_grid_resolution.txt")
    n = 200
    L = inputs.box_edge(n, 0.08)
    Y = inputs.random_suspension(n, L, 3)
    F, _ = inputs.random_loads(n, 4, torques=False)
    Ub, _ = ss.apply(Y, F, None, L)
    Sigma = 1.1
    rc = min(pr.cutoff_radius(Sigma, 1e-12), 0.5 * L)

    def err_at(M, MG):
        U, _ = g.fast_fcm_apply(Y, F, None, L, M, MG, Sigma, rc)
        return np.mean(np.linalg.norm(U - Ub, axis=1) / np.linalg.norm(Ub, axis=1))

    for k, (eps, ratio, MG) in enumerate(rows):
        eps, ratio, MG = float(eps), float(ratio), int(MG)
        M = int(round(L / (Sigma / ratio)))
        literal = err_at(M, MG)
        if k < 3:
            assert eps / 2 <= literal <= 2 * eps, (eps, literal)
        else:
            assert literal > 10 * eps, (eps, literal)   # the printed M_G truncates above the row's error
        wide = err_at(M, min(M, 2 * int(math.ceil(7.0 * ratio))))
        assert eps / 2 <= wide <= 2 * eps, (eps, wide)


def test_pair_correction_subset_equals_full_rows():
    L, n = 24.0, 150
    Y = inputs.random_suspension(n, L, 17)
    F, T = inputs.random_loads(n, 18)
    Sigma, rc = 1.4, 9.5
    Uf, Wf = g.pair_correction(Y, F, T, L, rc, Sigma, Sigma)
    idx = np.array([0, 7, 33, 149])
    Us, Ws = g.pair_correction_subset(Y, F, T, L, rc, Sigma, Sigma, idx)
    np.testing.assert_allclose(Us, Uf[idx], rtol=1e-12, atol=1e-16)
    np.testing.assert_allclose(Ws, Wf[idx], rtol=1e-12, atol=1e-16)
