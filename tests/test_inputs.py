"""The seeded workload generators: reproducible, non-overlapping, the stated shapes."""
import math
import os

import numpy as np

from paper_2310_12651_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _min_periodic_distance(Y, L):
    d = Y[:, None, :] - Y[None, :, :]
    d -= L * np.round(d / L)
    r = np.sqrt(np.einsum("ijk,ijk->ij", d, d))
    np.fill_diagonal(r, np.inf)
    return r.min()


def test_box_edge_matches_volume_fraction():
    L = inputs.box_edge(65536, 0.05)
    assert abs(L - 176.41391792668995) < 1e-9
    assert abs(65536 * 4 * math.pi / 3 / L ** 3 - 0.05) < 1e-15


def test_random_suspension_is_reproducible_and_non_overlapping():
    L = inputs.box_edge(800, 0.1)
    a = inputs.random_suspension(800, L, 5)
    b = inputs.random_suspension(800, L, 5)
    assert np.array_equal(a, b)
    assert a.shape == (800, 3) and np.all(a >= 0) and np.all(a < L)
    assert _min_periodic_distance(a, L) >= 2.2


def test_random_loads_are_mean_free():
    F, T = inputs.random_loads(1000, 9)
    assert np.max(np.abs(F.mean(axis=0))) < 1e-15 and np.max(np.abs(T.mean(axis=0))) < 1e-15
    F2, T2 = inputs.random_loads(1000, 9, torques=False, bias=(0, 0, -1))
    assert T2 is None and abs(F2[:, 2].mean() + 1) < 1e-14


def test_random_rods_geometry():
    L = 60.0
    Y, phi = inputs.random_rods(6, 8, L, 3)
    assert Y.shape == (48, 3)
    assert _min_periodic_distance(Y, L) >= 2.2 - 1e-9
    # consecutive spheres of a rod sit one bond apart
    d = Y[1:8] - Y[0:7]
    d -= L * np.round(d / L)
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 2.2, atol=1e-9)


def test_rods_without_rejection_keep_their_bonds():
    L = 50.0
    pos, phi = inputs.random_rods(100, 64, L, 3, min_sep=0.0)
    assert pos.shape == (6400, 3) and np.all(pos >= 0) and np.all(pos < L)
    d = np.diff(pos.reshape(100, 64, 3), axis=1)
    d -= L * np.round(d / L)
    assert np.allclose(np.linalg.norm(d, axis=2), 2.2)
    assert abs(phi - 6400 * 4 * np.pi / 3 / L ** 3) < 1e-12


def test_serving_pool_shares_parameters_within_a_class():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    pool, classes = bench.serve_pool(pool=8)
    assert len(pool) == 8 and sum(s["rods"] for s in pool) == 4
    for s in pool:
        L, ch = classes[s["cls"]]
        assert s["L"] == L and 2000 <= s["n"] <= 200000 + 64
        assert s["params"].M[0] == ch["M"] and 32 <= ch["M"] <= 256
        assert s["n"] * 4 * np.pi / 3 / L ** 3 <= 0.2 + 1e-9
        assert all(a.dtype == np.float32 and a.shape == (s["n"], 3) for a in s["arrays"])


def test_doublet_rods_geometry():
    """Rods of 11 alternating doublets: neighbours 2a apart, length 10 sqrt(2) a = 14.14a,
    centroid at the rod centre in the plane z = L_z/2, lattice spacing L/ceil(sqrt(N_R))."""
    from scipy.spatial.distance import pdist
    pos, off, X = inputs.doublet_rods(9, 60.0, 24.0, inputs.BASE_SEED + 300)
    assert pos.shape == (9 * 22, 3) and off.tolist() == list(range(0, 9 * 22 + 1, 22))
    assert np.allclose(X[:, 2], 12.0) and np.allclose(sorted(set(np.round(X[:, 0], 9))), [10.0, 30.0, 50.0])
    for b in range(9):
        r = pos[off[b]:off[b + 1]] - X[b]
        r -= np.array([60.0, 60.0, 24.0]) * np.round(r / np.array([60.0, 60.0, 24.0]))
        assert np.allclose(r.mean(axis=0), 0.0, atol=1e-12)
        assert abs(pdist(r).min() - 2.0) < 1e-12
        ends = 0.5 * (r[20] + r[21]) - 0.5 * (r[0] + r[1])
        assert abs(np.linalg.norm(ends) - 10 * np.sqrt(2.0)) < 1e-12 and abs(ends[2]) < 1e-12
        assert np.allclose(np.sort(r[:, 2]), np.sort(-r[:, 2]))   # symmetric about the plane
    ft = inputs.rod_loads(5, 1, gravity=(1.0, 0.0, 0.0))
    assert np.allclose(ft, [[22.0, 0, 0, 0, 0, 0]] * 5)
