"""Pins of the Brownian-increment oracle (positive splitting, Section 3.3; fluctuating FCM for
the grid part and a square root of the pairwise correction, as Section 7 proposes).

The grid part is a linear map B from grid noise to particle velocities; B B^T must equal
2 kT M~ exactly (M~ built column by column from the deterministic grid product). The pair
matrix must reproduce the oracle's pair correction and be positive definite.
"""
import numpy as np
import pytest

from oracle import brownian as ob
from oracle import closed_forms as cf
from oracle import grid_fcm as og
from oracle import params as op
from paper_2310_12651_gb300 import inputs


def _grid_mobility(Y, L, M, MG, Sigma, Sigma_D, eta=1.0):
    n = Y.shape[0]
    cols = []
    for k in range(6 * n):
        v = np.zeros(6 * n)
        v[k] = 1.0
        F = v[:3 * n].reshape(n, 3)
        T = v[3 * n:].reshape(n, 3)
        U, W = og.grid_apply(Y, F, T, L, M, MG, Sigma, Sigma_D, eta=eta)
        cols.append(np.concatenate([U.ravel(), W.ravel()]))
    return np.array(cols).T


@pytest.mark.parametrize("M, eta", [((10, 10, 10), 1.0), ((10, 8, 12), 1.7)])
def test_grid_noise_map_squares_to_the_grid_mobility(M, eta):
    """B B^T = 2 kT M~ for the map B: grid noise -> (U, W), built one unit noise vector at a time."""
    L = (9.0, 7.5, 11.0)
    Sigma, kT = 1.2, 0.7
    rng = np.random.default_rng(3)
    Y = rng.random((3, 3)) * np.array(L)
    MG = 8
    Mt = og._as3(M, np.int64)
    cols = []
    for k in range(3 * int(np.prod(Mt))):
        xi = np.zeros(3 * int(np.prod(Mt)))
        xi[k] = 1.0
        U, W = ob.brownian_grid(Y, xi.reshape(3, *Mt), L, MG, Sigma, Sigma, kT, eta=eta)
        cols.append(np.concatenate([U.ravel(), W.ravel()]))
    B = np.array(cols).T
    Mgrid = _grid_mobility(Y, L, Mt, MG, Sigma, Sigma, eta)
    err = np.linalg.norm(B @ B.T - 2.0 * kT * Mgrid) / np.linalg.norm(Mgrid)
    assert err < 1e-10, err


def test_pair_matrix_reproduces_the_pair_correction():
    L, n, Sigma = 30.0, 80, 2.0
    Y = inputs.random_suspension(n, L, inputs.BASE_SEED + 80, min_sep=1.0)
    rc = op.cutoff_radius(Sigma, 1e-6)
    A = ob.pair_correction_matrix(Y, L, rc, Sigma)
    F, _ = inputs.random_loads(n, inputs.BASE_SEED + 81, torques=False)
    U, _ = og.pair_correction(Y, F, None, L, rc, Sigma, Sigma)
    assert np.allclose(A @ F.ravel(), U.ravel(), rtol=0, atol=1e-12 * np.abs(U).max())
    assert np.allclose(A, A.T, rtol=0, atol=1e-14 * np.abs(A).max())


@pytest.mark.parametrize("min_sep, Sigma", [(2.2, 2.0), (0.3, 1.5), (0.0, 3.0)])
def test_pair_correction_is_positive_definite(min_sep, Sigma):
    """Positive splitting (Section 3.3): M - M~ is SPD, also with overlapping particles."""
    L, n = 25.0, 120
    Y = inputs.random_suspension(n, L, inputs.BASE_SEED + 82, min_sep=min_sep)
    rc = min(op.cutoff_radius(Sigma, 1e-8), 0.5 * L)
    w = np.linalg.eigvalsh(ob.pair_correction_matrix(Y, L, rc, Sigma))
    assert w.min() > 0.0, w.min()
    # a single particle: the Appendix B self correction, positive because Sigma > sigma
    assert cf.self_correction_VF(Sigma) > 0.0


def test_square_root_and_pair_increment():
    L, n, Sigma, kT = 20.0, 40, 2.0, 1.3
    Y = inputs.random_suspension(n, L, inputs.BASE_SEED + 83)
    rc = op.cutoff_radius(Sigma, 1e-6)
    A = ob.pair_correction_matrix(Y, L, rc, Sigma)
    S = ob.matrix_sqrt_spd(A)
    assert np.linalg.norm(S @ S - A) < 1e-12 * np.linalg.norm(A)
    z = np.random.default_rng(5).standard_normal((n, 3))
    Ub = ob.brownian_pair(Y, z, L, rc, Sigma, kT)
    assert np.allclose(Ub.ravel(), np.sqrt(2 * kT) * (S @ z.ravel()), rtol=1e-13, atol=0)
    with pytest.raises(ValueError):
        ob.matrix_sqrt_spd(-A)
