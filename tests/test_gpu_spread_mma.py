"""The tensor-core spread (spread_kernel = 3): the spread grid point by point against the oracle and
against the row-stationary kernel, the whole product against the oracle, batched passes, and the
cases its pipeline treats separately: more than one staged pass of particles per CTA, regions that
wrap around the periodic x edge, x extents that are not a multiple of 4 (scalar flush), forces only,
Sigma_D != Sigma, and every supported support width M_G."""
import numpy as np
import pytest

from gpu_util import FP32_TOL, System, assert_parity, ensure_built, rel_l2, rounded, suspension, torch_cuda
from oracle import grid_fcm as og

pytestmark = pytest.mark.gpu

TENSOR, ROWS = 3, 1


@pytest.fixture(scope="module")
def fcm():
    return ensure_built()


def _spread_grid(fcm, s, kernel, tile=(8, 8, 8)):
    torch = torch_cuda()
    M = np.broadcast_to(np.asarray(s.M), (3,))
    p = fcm.make_params(s.L, s.M, s.Sigma, s.r_c, s.M_G, s.n, fcm.FCM_FP32, Sigma_D=s.Sigma_D, tile=tile,
                        spread_kernel=kernel)
    st = torch.cuda.current_stream().cuda_stream
    with fcm.Handle(p) as h:
        pos = torch.as_tensor(s.Y, dtype=torch.float32, device="cuda")
        F = torch.as_tensor(s.F, dtype=torch.float32, device="cuda")
        T = torch.as_tensor(s.T, dtype=torch.float32, device="cuda") if s.T is not None else None
        h.spread(s.n, pos, F, T, st)
        grid = torch.empty(3 * int(np.prod(M)), dtype=torch.float32, device="cuda")
        h.copy_grid(grid, st)
        torch.cuda.synchronize()
        assert h.check() == 0
    # [c][z][y][x] -> [c][x][y][z]
    return grid.double().cpu().numpy().reshape(3, M[2], M[1], M[0]).transpose(0, 3, 2, 1)


def _oracle_grid(fcm, s):
    """The oracle's spread on the FP32-rounded inputs, window starts decided in FP32 as the kernels
    decide them (this matters only for particles on grid points)."""
    SD = s.Sigma_D if s.Sigma_D else s.Sigma
    r = lambda x: rounded(x, fcm.FCM_FP32)
    return og.spread(r(s.Y), r(s.F), r(s.T), s.L, s.M, s.M_G, s.Sigma, SD, fp32_windows=True)


def _check_grid(fcm, s, what):
    got = _spread_grid(fcm, s, TENSOR)
    rows = _spread_grid(fcm, s, ROWS)
    assert np.all(np.isfinite(got))
    assert_parity(got, _oracle_grid(fcm, s), FP32_TOL, f"tensor spread grid vs oracle, {what}")
    # both FP32 kernels evaluate the same terms (the split TF32 products carry FP32-level rounding);
    # they differ by rounding only: 1e-6 on random suspensions, 3e-6 where ~190 particles overlap
    r = rel_l2(got, rows)
    print(f"tensor vs row-stationary spread grid, {what}: rel L2 {r:.3e}")
    assert r < 1e-5, f"{what}: tensor and row-stationary spreads differ by {r:.3e}"


@pytest.mark.parametrize("M_G", [10, 12, 14])
@pytest.mark.parametrize("torques", [True, False])
def test_tensor_spread_grid(fcm, M_G, torques):
    s = System(3000, 60.0, 48, 2.0, M_G, 10.0, 301 + M_G, torques=torques)
    _check_grid(fcm, s, f"M_G={M_G} torques={torques}")


def test_tensor_spread_grid_torque_width_differs(fcm):
    s = System(3000, 60.0, 48, 2.0, 14, 10.0, 311, Sigma_D=1.6)
    _check_grid(fcm, s, "Sigma_D != Sigma")


def test_tensor_spread_grid_dense_several_passes(fcm):
    """About 190 particles per two-tile region: three staged passes of 64 per CTA."""
    rng = np.random.default_rng(312)
    n, L = 6000, 40.0
    s = System(n, L, 32, 1.6, 12, 8.0, 312, Y=rng.random((n, 3)) * L)
    _check_grid(fcm, s, "dense")


def test_tensor_spread_grid_scalar_flush_and_anisotropic(fcm):
    """M_x = 42 (not a multiple of 4: the scalar flush everywhere), a non-cubic box and grid."""
    rng = np.random.default_rng(313)
    L = np.array([52.5, 50.0, 45.0])
    n = 2500
    s = System(n, L, (42, 40, 36), 2.0, 12, 9.0, 313, Y=rng.random((n, 3)) * L)
    _check_grid(fcm, s, "M = (42, 40, 36)")


def test_tensor_spread_grid_edges_and_few_particles(fcm):
    """Particles on the box faces and corners and on grid points (h = 1.2: 12.0 and 24.0), one per
    region, regions wrapping at every face."""
    L = 48.0
    pts = [[0.0, 0.0, 0.0], [47.999, 0.01, 23.9], [12.0, 47.99, 47.99], [24.0, 24.0, 0.0], [0.5, 31.0, 47.5],
           [36.0, 1.2, 46.8]]
    Y = np.array(pts)
    s = System(len(pts), L, 40, 2.0, 14, 10.0, 314, Y=Y)
    _check_grid(fcm, s, "edges")


def test_tensor_spread_full_product_matches_oracle(fcm):
    torch = torch_cuda()
    s = suspension(5000, 0.05, 48, 2.0, 1e-6, 66)
    assert s.M_G in (10, 12, 14), s.M_G
    p = fcm.make_params(s.L, s.M, s.Sigma, s.r_c, s.M_G, s.n, fcm.FCM_FP32, tile=(8, 8, 8), spread_kernel=TENSOR)
    from gpu_util import run_gpu
    with fcm.Handle(p) as h:
        U, W = run_gpu(s, fcm.FCM_FP32, handle=h)
    Uo, Wo = s.oracle(fcm.FCM_FP32)
    assert_parity(U, Uo, FP32_TOL, "U tensor spread")
    assert_parity(W, Wo, FP32_TOL, "W tensor spread")
    del torch


def test_tensor_spread_batched_equals_alone(fcm):
    """Three systems in one batched pass (a ragged one among them) equal each system alone."""
    torch = torch_cuda()
    dev = torch.device("cuda:0")
    st = torch.cuda.current_stream().cuda_stream
    L, M, MG, Sg, rc = 50.0, 40, 12, 1.8, 9.0
    sizes = [1500, 37, 1200]
    systems = [System(n, L, M, Sg, MG, rc, 320 + k) for k, n in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)]).tolist()
    cat = lambda a: torch.as_tensor(np.concatenate(a), dtype=torch.float32, device=dev)
    pos, F, T = cat([s.Y for s in systems]), cat([s.F for s in systems]), cat([s.T for s in systems])
    U, W = torch.empty_like(F), torch.empty_like(F)
    p = fcm.make_params(L, M, Sg, rc, MG, sum(sizes), fcm.FCM_FP32, tile=(8, 8, 8), spread_kernel=TENSOR)
    with fcm.Handle(p, 0, max_systems=len(sizes)) as h:
        h.batch_apply(off, pos, F, T, U, W, st)
        torch.cuda.synchronize()
        assert h.check() == 0
    Ub, Wb = U.double().cpu().numpy(), W.double().cpu().numpy()
    for k, s in enumerate(systems):
        Uo, Wo = s.oracle(fcm.FCM_FP32)
        assert_parity(Ub[off[k]:off[k + 1]], Uo, FP32_TOL, f"U batched system {k}")
        assert_parity(Wb[off[k]:off[k + 1]], Wo, FP32_TOL, f"W batched system {k}")
