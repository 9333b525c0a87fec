"""Closed-form FCM pair mobilities and fast-FCM corrections, FP64 numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Every tensor function takes displacements ``x`` of shape (..., 3) with r > 0
and returns (..., 3, 3). ``eta`` is the viscosity. Notation follows the paper:
sigma = a/sqrt(pi) (Section 2), sigma_D = a/(6 sqrt(pi))^(1/3) (Section 3.4),
Sigma / Sigma_D the modified widths, and dd = sigma^2 - Sigma^2.

Readings of the printed formulas (each checked by the Fourier-quadrature tests):
* correction VF: the erf difference is erf(r/(2 sigma)) - erf(r/(2 Sigma)),
  the arguments that S(x; sigma sqrt 2) and S(x; Sigma sqrt 2) carry;
* correction WT: the factor 1/2 of the M^WT pair mobility is kept;
* the torque-Gaussian self correction uses Sigma_D (Sigma_D = Sigma in the paper).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf, erfc

PI = math.pi


def fcm_sigma(a: float = 1.0) -> float:
    """Force Gaussian width, a = sigma sqrt(pi) (Section 2)."""
    return a / math.sqrt(PI)


def fcm_sigma_D(a: float = 1.0) -> float:
    """Torque (dipole) Gaussian width sigma_D = a / (6 sqrt(pi))^(1/3) (Section 3.4)."""
    return a / (6.0 * math.sqrt(PI)) ** (1.0 / 3.0)


def gaussian(r, s):
    """Delta(x; s) = (2 pi s^2)^(-3/2) exp(-r^2 / (2 s^2)) (Section 2, first equation)."""
    r = np.asarray(r, dtype=np.float64)
    return (2.0 * PI * s * s) ** -1.5 * np.exp(-r * r / (2.0 * s * s))


def _geometry(x):
    x = np.asarray(x, dtype=np.float64)
    r = np.linalg.norm(x, axis=-1)
    n = x / r[..., None]
    nn = n[..., :, None] * n[..., None, :]
    eye = np.broadcast_to(np.eye(3), nn.shape)
    return x, r, nn, eye


def minus_x_cross(x):
    """The matrix (-x cross) printed in Section 3.4: (-x cross) v = -x cross v."""
    x = np.asarray(x, dtype=np.float64)
    z = np.zeros(x.shape[:-1])
    x1, x2, x3 = x[..., 0], x[..., 1], x[..., 2]
    rows = [np.stack([z, x3, -x2], -1), np.stack([-x3, z, x1], -1), np.stack([x2, -x1, z], -1)]
    return np.stack(rows, axis=-2)


def _b(v):  # broadcast a (...,) scalar field against (..., 3, 3)
    return np.asarray(v)[..., None, None]


# --- flows of Gaussian force distributions (Section 2.2) -------------------

def oseen(x, eta=1.0):
    """G(x) = (I + x x^T / r^2) / (8 pi eta r)."""
    x, r, nn, eye = _geometry(x)
    return (eye + nn) / _b(8.0 * PI * eta * r)


def laplacian_oseen(x, eta=1.0):
    """nabla^2 G = (I - 3 x x^T / r^2) / (4 pi eta r^3)."""
    x, r, nn, eye = _geometry(x)
    return (eye - 3.0 * nn) / _b(4.0 * PI * eta * r ** 3)


def S1(x, s, eta=1.0):
    x, r, nn, eye = _geometry(x)
    return _b(erf(r / (s * math.sqrt(2.0))) / (8.0 * PI * eta * r)) * (eye + nn)


def S2(x, s, eta=1.0):
    x, r, nn, eye = _geometry(x)
    return _b(s * s * erf(r / (s * math.sqrt(2.0))) / (8.0 * PI * eta * r ** 3)) * (eye - 3.0 * nn)


def S3(x, s, eta=1.0):
    x, r, nn, eye = _geometry(x)
    return _b(-(s * s / (2.0 * eta)) * (s * s / r ** 2) * gaussian(r, s)) * (eye - 3.0 * nn)


def S(x, s, eta=1.0):
    """Flow of F Delta(x; s): u = S(x; s) F, S = S1 + S2 + S3 (Section 2.2)."""
    return S1(x, s, eta) + S2(x, s, eta) + S3(x, s, eta)


def Q1(x, s, eta=1.0):
    x, r, nn, eye = _geometry(x)
    return _b(erf(r / (s * math.sqrt(2.0))) / (4.0 * PI * eta * r ** 3)) * (eye - 3.0 * nn)


def Q2(x, s, eta=1.0):
    x, r, nn, eye = _geometry(x)
    g = gaussian(r, s)
    return -(_b((1.0 + s * s / r ** 2) * g) * eye - _b((1.0 + 3.0 * s * s / r ** 2) * g) * nn) / eta


def Q(x, s, eta=1.0):
    """Flow of H nabla^2 Delta(x; s): u = Q(x; s) H, Q = Q1 + Q2 (Section 2.2)."""
    return Q1(x, s, eta) + Q2(x, s, eta)


def T_tensor(x, s, eta=1.0):
    """T(x; s) = (1/(eta s^2)) (2 I + (x x^T - r^2 I)/s^2) Delta(x; s) (Section 3.2)."""
    x, r, nn, eye = _geometry(x)
    g = gaussian(r, s)
    return (_b(2.0 * g) * eye + _b(r * r * g / (s * s)) * (nn - eye)) / (eta * s * s)


def R_tensor(x, s, eta=1.0):
    """R(x; s) = [erf(r/(s sqrt 2)) - 4 pi r s^2 Delta] / (8 pi eta r^3) (-x cross) (Section 3.4)."""
    x, r, nn, eye = _geometry(x)
    c = (erf(r / (s * math.sqrt(2.0))) - 4.0 * PI * r * s * s * gaussian(r, s)) / (8.0 * PI * eta * r ** 3)
    return _b(c) * minus_x_cross(x)


def P_tensor(x, s, eta=1.0):
    """P = P1 + P2, the vorticity of a Gaussian torque distribution (Section 3.4)."""
    x, r, nn, eye = _geometry(x)
    p1 = _b(erf(r / (s * math.sqrt(2.0))) / (8.0 * PI * eta * r ** 3)) * (-eye + 3.0 * nn)
    g = gaussian(r, s)
    p2 = (_b((s * s + r * r) * g) * eye - _b((3.0 * s * s + r * r) * g) * nn) / _b(2.0 * eta * r * r)
    return p1 + p2


def K_tensor(x, s, eta=1.0):
    """K(x; s) = -Delta(x; s) / (2 s^2 eta) (-x cross) (Section 3.4)."""
    x, r, nn, eye = _geometry(x)
    return _b(-gaussian(r, s) / (2.0 * s * s * eta)) * minus_x_cross(x)


# --- pair mobilities --------------------------------------------------------

def fcm_pair_mobility(x, a=1.0, eta=1.0):
    """Standard FCM pair blocks (M_VF, M_WF, M_VT, M_WT) for x = Y_n - Y_m.

    M_VF = S(x; sigma sqrt 2) (eq. M_VF), M_WF = R(x; sqrt(sigma^2 + sigma_D^2)),
    M_WT = P(x; sigma_D sqrt 2) / 2 and M_VT_nm = (M_WF_mn)^T (Section 3.4).
    """
    sg, sd = fcm_sigma(a), fcm_sigma_D(a)
    x = np.asarray(x, dtype=np.float64)
    m_vf = S(x, sg * math.sqrt(2.0), eta)
    m_wf = R_tensor(x, math.sqrt(sg * sg + sd * sd), eta)
    m_vt = np.swapaxes(R_tensor(-x, math.sqrt(sg * sg + sd * sd), eta), -1, -2)
    m_wt = 0.5 * P_tensor(x, sd * math.sqrt(2.0), eta)
    return m_vf, m_wf, m_vt, m_wt


def modified_pair_mobility(x, Sigma, Sigma_D=None, a=1.0, eta=1.0):
    """Pair blocks of the grid operator with the modified kernels (Sections 3.2 and 3.4).

    M~_VF = S(x; sqrt2 Sigma) + dd Q(x; sqrt2 Sigma) + dd^2/4 T(x; sqrt2 Sigma);
    M~_WF = R(x; St) + dd/2 K(x; St) with St = sqrt(Sigma^2 + Sigma_D^2);
    M~_WT = P(x; Sigma_D sqrt 2) / 2; M~_VT_nm = (M~_WF_mn)^T.
    """
    Sigma_D = Sigma if Sigma_D is None else Sigma_D
    sg = fcm_sigma(a)
    dd = sg * sg - Sigma * Sigma
    x = np.asarray(x, dtype=np.float64)
    s2 = Sigma * math.sqrt(2.0)
    m_vf = S(x, s2, eta) + dd * Q(x, s2, eta) + 0.25 * dd * dd * T_tensor(x, s2, eta)
    st = math.sqrt(Sigma * Sigma + Sigma_D * Sigma_D)
    m_wf = R_tensor(x, st, eta) + 0.5 * dd * K_tensor(x, st, eta)
    m_vt = np.swapaxes(R_tensor(-x, st, eta) + 0.5 * dd * K_tensor(-x, st, eta), -1, -2)
    m_wt = 0.5 * P_tensor(x, Sigma_D * math.sqrt(2.0), eta)
    return m_vf, m_wf, m_vt, m_wt


# --- pairwise corrections M - M~ (Section 3.2 and 3.4) ----------------------

def correction_VF(x, Sigma, a=1.0, eta=1.0):
    """M_VF - M~_VF, the correction_VF equation (Section 3.2).

    (G + sigma^2 nabla^2 G)(erf(r/2sigma) - erf(r/2Sigma)) + S3(x; sigma sqrt2)
    - S3(x; Sigma sqrt2) - dd Q2(x; Sigma sqrt2) - dd^2/4 T(x; Sigma sqrt2).
    The erf difference is evaluated as erfc(r/2Sigma) - erfc(r/2sigma).
    """
    sg = fcm_sigma(a)
    dd = sg * sg - Sigma * Sigma
    x, r, nn, eye = _geometry(x)
    ediff = erfc(r / (2.0 * Sigma)) - erfc(r / (2.0 * sg))
    out = (oseen(x, eta) + sg * sg * laplacian_oseen(x, eta)) * _b(ediff)
    out = out + S3(x, sg * math.sqrt(2.0), eta) - S3(x, Sigma * math.sqrt(2.0), eta)
    out = out - dd * Q2(x, Sigma * math.sqrt(2.0), eta)
    out = out - 0.25 * dd * dd * T_tensor(x, Sigma * math.sqrt(2.0), eta)
    return out


def correction_WF(x, Sigma, Sigma_D=None, a=1.0, eta=1.0):
    """M_WF - M~_WF, the correction_WF equation (Section 3.4).

    R(x; sqrt(sigma^2+sigma_D^2)) - R(x; sqrt(Sigma^2+Sigma_D^2)) - dd/2 K(x; sqrt(Sigma^2+Sigma_D^2)).
    The matching M_VT - M~_VT block is its transpose at -x, which equals it.
    """
    Sigma_D = Sigma if Sigma_D is None else Sigma_D
    sg, sd = fcm_sigma(a), fcm_sigma_D(a)
    dd = sg * sg - Sigma * Sigma
    st_small = math.sqrt(sg * sg + sd * sd)
    st_big = math.sqrt(Sigma * Sigma + Sigma_D * Sigma_D)
    return R_tensor(x, st_small, eta) - R_tensor(x, st_big, eta) - 0.5 * dd * K_tensor(x, st_big, eta)


def correction_WT(x, Sigma, Sigma_D=None, a=1.0, eta=1.0):
    """M_WT - M~_WT = (P(x; sigma_D sqrt2) - P(x; Sigma_D sqrt2)) / 2 (correction_WT, with the 1/2 of M_WT)."""
    Sigma_D = Sigma if Sigma_D is None else Sigma_D
    sd = fcm_sigma_D(a)
    return 0.5 * (P_tensor(x, sd * math.sqrt(2.0), eta) - P_tensor(x, Sigma_D * math.sqrt(2.0), eta))


def self_correction_VF(Sigma, a=1.0, eta=1.0):
    """Limit r -> 0 of M_VF - M~_VF (Appendix B, first equation), a scalar times I."""
    sg = fcm_sigma(a)
    dd = sg * sg - Sigma * Sigma
    sp = Sigma * math.sqrt(PI)
    return (1.0 / (6.0 * PI * eta * a) - 1.0 / (6.0 * PI * eta * sp)
            + dd / (12.0 * eta * sp ** 3) - dd * dd / (32.0 * eta * Sigma ** 5 * PI ** 1.5))


def self_correction_WT(Sigma_D, a=1.0, eta=1.0):
    """Limit r -> 0 of M_WT - M~_WT (Appendix B, second equation), a scalar times I."""
    return 1.0 / (8.0 * PI * eta * a ** 3) - 1.0 / (48.0 * eta * (Sigma_D * math.sqrt(PI)) ** 3)


def splitting_function(k, Sigma, a=1.0):
    """H_FCM(k) = p(k) exp(-(Sigma^2 - sigma^2) k^2), p = 1 - dd k^2 + dd^2 k^4 / 4 (Section 3.3)."""
    sg = fcm_sigma(a)
    dd = sg * sg - Sigma * Sigma
    k = np.asarray(k, dtype=np.float64)
    p = 1.0 - dd * k * k + 0.25 * dd * dd * k ** 4
    return p * np.exp(-(Sigma * Sigma - sg * sg) * k * k)
