"""Pins of the oracle's closed forms against routes that do not use them.

Each pair mobility of the paper is the inverse Fourier transform of a radial
kernel (Appendix A for VF; the same steps give WF and WT). For an isotropic
kernel the 3-D transform reduces to 1-D radial integrals with spherical Bessel
functions, evaluated here by adaptive quadrature. A dropped term, a wrong sign,
a wrong width (sigma vs sigma sqrt 2) or a missing factor 1/2 in any closed form
breaks one of these checks.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import spherical_jn

from oracle import closed_forms as cf

A, ETA = 1.0, 1.0
SG = A / math.sqrt(math.pi)
SD = A / (6.0 * math.sqrt(math.pi)) ** (1.0 / 3.0)


def _radial(fn, kmax):
    val, _ = quad(fn, 0.0, kmax, limit=4000, epsabs=1e-16, epsrel=1e-13)
    return val


def vf_quadrature(phi, r, kmax):
    """(1/(2 pi^2 eta)) int phi(k) [(j0 - j1/(kr)) I + j2 nn] dk -> (alpha, beta) of alpha I + beta nn."""
    al = _radial(lambda k: phi(k) * (spherical_jn(0, k * r) - spherical_jn(1, k * r) / (k * r)), kmax)
    be = _radial(lambda k: phi(k) * spherical_jn(2, k * r), kmax)
    c = 1.0 / (2 * math.pi ** 2 * ETA)
    return c * al, c * be


def wf_quadrature(psi, r, kmax):
    """c(r) with M_WF = c(r) (-x cross): c = (1/(4 pi^2 eta r)) int psi(k) k j1(kr) dk."""
    return _radial(lambda k: psi(k) * k * spherical_jn(1, k * r), kmax) / (4 * math.pi ** 2 * ETA * r)


def wt_quadrature(chi, r, kmax):
    """(1/(8 pi^2 eta)) int chi(k) k^2 [(j0 - j1/(kr)) I + j2 nn] dk -> (alpha, beta)."""
    al = _radial(lambda k: chi(k) * k * k * (spherical_jn(0, k * r) - spherical_jn(1, k * r) / (k * r)), kmax)
    be = _radial(lambda k: chi(k) * k * k * spherical_jn(2, k * r), kmax)
    c = 1.0 / (8 * math.pi ** 2 * ETA)
    return c * al, c * be


def _split(tensor, x):
    """alpha, beta of a tensor alpha I + beta nn at direction x."""
    n = x / np.linalg.norm(x)
    perp = np.cross(n, [0.3, -0.7, 0.2])
    perp /= np.linalg.norm(perp)
    alpha = perp @ tensor @ perp
    beta = n @ tensor @ n - alpha
    return alpha, beta


def _wf_coeff(tensor, x):
    """c of a tensor c (-x cross)."""
    mx = cf.minus_x_cross(x)
    return float(np.sum(tensor * mx) / np.sum(mx * mx))


SIGMAS = [1.0, 2.0, 3.0]
RADII = [0.35, 1.1, 2.2, 4.0, 7.5]
X_DIR = np.array([0.48, -0.64, 0.6])


def _x(r):
    return X_DIR / np.linalg.norm(X_DIR) * r


@pytest.mark.parametrize("r", RADII)
def test_fcm_vf_matches_fourier(r):
    """M_VF = S(x; sigma sqrt 2) is the transform of exp(-sigma^2 k^2) (Appendix A)."""
    x = _x(r)
    al, be = vf_quadrature(lambda k: math.exp(-SG * SG * k * k), r, 12.0 / SG)
    t = cf.fcm_pair_mobility(x[None], A, ETA)[0][0]
    a2, b2 = _split(t, x)
    scale = 1.0 / (6 * math.pi)
    assert abs(a2 - al) < 1e-12 * scale and abs(b2 - be) < 1e-12 * scale


@pytest.mark.parametrize("Sigma", SIGMAS)
@pytest.mark.parametrize("r", RADII)
def test_modified_and_correction_vf_match_fourier(Sigma, r):
    """M~_VF (Section 3.2) is the transform of (1 - dd k^2/2)^2 exp(-Sigma^2 k^2); the correction is their difference."""
    x = _x(r)
    dd = SG * SG - Sigma * Sigma
    phi_mod = lambda k: (1 - 0.5 * dd * k * k) ** 2 * math.exp(-Sigma * Sigma * k * k)
    phi_cor = lambda k: math.exp(-SG * SG * k * k) - phi_mod(k)
    kmax = 14.0 / SG
    scale = 1.0 / (6 * math.pi)
    al, be = vf_quadrature(phi_mod, r, kmax)
    a2, b2 = _split(cf.modified_pair_mobility(x[None], Sigma, None, A, ETA)[0][0], x)
    assert abs(a2 - al) < 1e-12 * scale and abs(b2 - be) < 1e-12 * scale
    al, be = vf_quadrature(phi_cor, r, kmax)
    a2, b2 = _split(cf.correction_VF(x[None], Sigma, A, ETA)[0], x)
    assert abs(a2 - al) < 1e-12 * scale and abs(b2 - be) < 1e-12 * scale


@pytest.mark.parametrize("Sigma", SIGMAS)
@pytest.mark.parametrize("r", RADII)
def test_wf_blocks_match_fourier(Sigma, r):
    """M_WF = R(x; sqrt(sigma^2 + sigma_D^2)); M~_WF adds dd/2 K; their difference is correction_WF."""
    x = _x(r)
    dd = SG * SG - Sigma * Sigma
    psi = lambda k: math.exp(-0.5 * (SG * SG + SD * SD) * k * k)
    psi_mod = lambda k: (1 - 0.5 * dd * k * k) * math.exp(-0.5 * (2 * Sigma * Sigma) * k * k)
    kmax = 16.0 / SD
    scale = 1.0 / (6 * math.pi)
    c_std = wf_quadrature(psi, r, kmax)
    c_mod = wf_quadrature(psi_mod, r, kmax)
    m = cf.fcm_pair_mobility(x[None], A, ETA)
    mt = cf.modified_pair_mobility(x[None], Sigma, None, A, ETA)
    assert abs(_wf_coeff(m[1][0], x) - c_std) < 1e-12 * scale
    assert abs(_wf_coeff(mt[1][0], x) - c_mod) < 1e-12 * scale
    assert abs(_wf_coeff(cf.correction_WF(x[None], Sigma, None, A, ETA)[0], x) - (c_std - c_mod)) < 1e-12 * scale
    # VT_nm = (WF_mn)^T: the same block (the matrix is antisymmetric and odd in x)
    np.testing.assert_allclose(m[2][0], m[1][0], atol=1e-16)
    np.testing.assert_allclose(mt[2][0], mt[1][0], atol=1e-16)


@pytest.mark.parametrize("Sigma_D", SIGMAS)
@pytest.mark.parametrize("r", RADII)
def test_wt_blocks_match_fourier(Sigma_D, r):
    """M_WT = P(x; sigma_D sqrt 2)/2 is the transform of k^2 exp(-sigma_D^2 k^2)/(4 eta) (I - k^k^)."""
    x = _x(r)
    chi = lambda k: math.exp(-SD * SD * k * k)
    chi_mod = lambda k: math.exp(-Sigma_D * Sigma_D * k * k)
    kmax = 18.0 / SD
    scale = 1.0 / (8 * math.pi)
    al, be = wt_quadrature(chi, r, kmax)
    a2, b2 = _split(cf.fcm_pair_mobility(x[None], A, ETA)[3][0], x)
    assert abs(a2 - al) < 1e-12 * scale and abs(b2 - be) < 1e-12 * scale
    al2, be2 = wt_quadrature(chi_mod, r, kmax)
    a3, b3 = _split(cf.correction_WT(x[None], 2.0, Sigma_D, A, ETA)[0], x)
    assert abs(a3 - (al - al2)) < 1e-12 * scale and abs(b3 - (be - be2)) < 1e-12 * scale


@pytest.mark.parametrize("Sigma", SIGMAS)
def test_self_corrections_match_fourier_at_r0(Sigma):
    """Appendix B limits equal the r = 0 Fourier integrals (2/3 of the trace kernel)."""
    dd = SG * SG - Sigma * Sigma
    vf0 = _radial(lambda k: (2.0 / 3.0) * (math.exp(-SG * SG * k * k)
                                            - (1 - 0.5 * dd * k * k) ** 2 * math.exp(-Sigma * Sigma * k * k)), 14 / SG)
    vf0 /= 2 * math.pi ** 2 * ETA
    assert abs(cf.self_correction_VF(Sigma, A, ETA) - vf0) < 1e-13
    wt0 = _radial(lambda k: (2.0 / 3.0) * k * k * (math.exp(-SD * SD * k * k) - math.exp(-Sigma * Sigma * k * k)), 18 / SD)
    wt0 /= 8 * math.pi ** 2 * ETA
    assert abs(cf.self_correction_WT(Sigma, A, ETA) - wt0) < 1e-13


@pytest.mark.parametrize("Sigma", SIGMAS)
def test_closed_forms_approach_self_limit(Sigma):
    """The correction closed forms tend to the Appendix B constants as r -> 0 (O(r^2))."""
    for r in (1e-2, 3e-3):
        x = _x(r)[None]
        vf = cf.correction_VF(x, Sigma, A, ETA)[0]
        wt = cf.correction_WT(x, Sigma, None, A, ETA)[0]
        wf = cf.correction_WF(x, Sigma, None, A, ETA)[0]
        np.testing.assert_allclose(vf, cf.self_correction_VF(Sigma) * np.eye(3), atol=2e-4 * r / 1e-2 * 0.05 + 1e-9)
        np.testing.assert_allclose(wt, cf.self_correction_WT(Sigma) * np.eye(3), atol=2e-3 * (r / 1e-2) ** 2 + 1e-8)
        assert np.max(np.abs(wf)) < 0.1 * r


def test_unbounded_drag_laws():
    """Single-particle FCM mobilities: 1/(6 pi eta a) (Section 2) and 1/(8 pi eta a^3) (Section 3.4)."""
    tiny = _x(1e-4)[None]
    s = cf.fcm_pair_mobility(tiny, A, ETA)
    np.testing.assert_allclose(np.diag(s[0][0]), 1 / (6 * math.pi), rtol=1e-6)
    np.testing.assert_allclose(np.diag(s[3][0]), 1 / (8 * math.pi), rtol=1e-6)
    # a = 2: the drag laws scale as 1/a and 1/a^3
    s2 = cf.fcm_pair_mobility(_x(1e-4)[None] * 2, 2.0, ETA)
    np.testing.assert_allclose(np.diag(s2[0][0]), 1 / (12 * math.pi), rtol=1e-6)
    np.testing.assert_allclose(np.diag(s2[3][0]), 1 / (64 * math.pi), rtol=1e-6)


def test_far_field_is_oseen_and_corrections_decay():
    """At r >> sigma the FCM VF block is G + sigma^2 nabla^2 G (the erf factors of S1, S2 tend to 1 and
    S3 decays like a Gaussian) and every correction is exponentially small."""
    x = _x(30.0)[None]
    far = cf.oseen(x)[0] + SG * SG * cf.laplacian_oseen(x)[0]
    np.testing.assert_allclose(cf.fcm_pair_mobility(x)[0][0], far, rtol=1e-12, atol=1e-18)
    for Sigma in SIGMAS:
        x = _x(12.0 * Sigma)[None]
        assert np.max(np.abs(cf.correction_VF(x, Sigma)[0])) < 1e-12
        assert np.max(np.abs(cf.correction_WF(x, Sigma)[0])) < 1e-12
        assert np.max(np.abs(cf.correction_WT(x, Sigma)[0])) < 1e-12


@pytest.mark.parametrize("Sigma", [0.7, 1.5, 4.0])
def test_positive_splitting_function(Sigma):
    """H_FCM in (0, 1], equal to 1 at k = 0, monotone decreasing (Section 3.3)."""
    k = np.linspace(0, 20.0 / Sigma, 20001)   # H stays above the FP64 underflow here
    H = cf.splitting_function(k, Sigma)
    assert H[0] == pytest.approx(1.0, abs=1e-15)
    assert np.all(H[1:] > 0) and np.all(H <= 1.0 + 1e-15) and np.all(np.diff(H) <= 1e-15)
    # it is the ratio of the squared kernel transforms
    dd = SG * SG - Sigma * Sigma
    ratio = (1 - 0.5 * dd * k * k) ** 2 * np.exp(-Sigma * Sigma * k * k) / np.exp(-SG * SG * k * k)
    mask = k < 6.0 / Sigma
    np.testing.assert_allclose(H[mask], ratio[mask], rtol=1e-10)


def test_sigma_equal_Sigma_gives_zero_correction():
    """With Sigma = sigma the modified kernel is the FCM kernel and every correction vanishes (Section 5)."""
    x = np.array([[0.7, 0.2, -0.4], [2.0, 1.0, 3.0]])
    assert np.max(np.abs(cf.correction_VF(x, SG))) < 1e-16
    assert np.max(np.abs(cf.correction_WT(x, SG, SD))) < 1e-16
    assert np.max(np.abs(cf.correction_WF(x, SG, SD))) < 1e-16
    assert abs(cf.self_correction_VF(SG)) < 1e-16 and abs(cf.self_correction_WT(SD)) < 1e-16


def _ball_points(n, seed, radius=6.0, min_sep=2.2):
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < n:
        p = (rng.random(3) * 2 - 1) * radius
        if np.linalg.norm(p) <= radius and all(np.linalg.norm(p - q) >= min_sep for q in pts):
            pts.append(p)
    return np.array(pts)


def _free_matrix(Y, block, diag):
    n = Y.shape[0]
    Mx = np.zeros((3 * n, 3 * n))
    for i in range(n):
        Mx[3 * i:3 * i + 3, 3 * i:3 * i + 3] = diag * np.eye(3)
        for j in range(n):
            if i != j:
                Mx[3 * i:3 * i + 3, 3 * j:3 * j + 3] = block((Y[i] - Y[j])[None])[0]
    return Mx


@pytest.mark.parametrize("Sigma", [1.0, 2.0])
def test_positive_splitting_matrices_are_spd(Sigma):
    """M_VF, M~_VF and M_VF - M~_VF are symmetric positive definite (Section 3.3), by Cholesky."""
    Y = _ball_points(24, 7)
    m_full = _free_matrix(Y, lambda x: cf.fcm_pair_mobility(x)[0], 1 / (6 * math.pi))
    m_cor = _free_matrix(Y, lambda x: cf.correction_VF(x, Sigma), cf.self_correction_VF(Sigma))
    m_mod = m_full - m_cor
    for Mx in (m_full, m_cor, m_mod):
        np.testing.assert_allclose(Mx, Mx.T, atol=1e-15)
        np.linalg.cholesky(Mx)
