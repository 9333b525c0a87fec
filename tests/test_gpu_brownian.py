"""Brownian increments on the GPU (fcm_brownian) against the oracle of oracle/brownian.py.

Both sides take the same random inputs: grid noise xi (layout [c][z][y][x] on the device,
[c][x][y][z] for the oracle) and the normal vector z of the pair part, so the comparison is
element by element: the grid part exactly (FFT, square-root projection, interpolation), the
pair part against the oracle's exact matrix square root to the Lanczos tolerance.
"""
import numpy as np
import pytest

from gpu_util import FP32_TOL, FP64_TOL, assert_parity, ensure_built, rounded, torch_cuda
from oracle import brownian as ob
from oracle import params as op
from paper_2310_12651_gb300 import inputs

pytestmark = pytest.mark.gpu

KT = 0.8


@pytest.fixture(scope="module")
def fcm():
    torch_cuda()
    return ensure_built()


def _setup(n=400, L=30.0, M=32, Sigma=1.5, seed=90):
    Y = inputs.random_suspension(n, L, inputs.BASE_SEED + seed)
    assert op.cutoff_radius(Sigma, 1e-6) <= 0.5 * L
    rng = np.random.default_rng(seed)
    xi = rng.standard_normal((3, M, M, M))            # device layout [c][z][y][x]
    z = rng.standard_normal((n, 3))
    MG = op.support_points(Sigma, L / M, 4.8)
    rc = op.cutoff_radius(Sigma, 1e-6)
    return Y, xi, z, L, M, MG, Sigma, rc


def _run(fcm, prec, Y, xi, z, L, M, MG, Sigma, rc, max_iter=60, tol=1e-10, want_W=True):
    import torch
    dt = torch.float32 if prec == fcm.FCM_FP32 else torch.float64
    dev = torch.device("cuda:0")
    n = Y.shape[0]
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev) if a is not None else None
    pos, xid, zd = t(Y), t(None if xi is None else xi.ravel()), t(z)
    U = torch.empty((n, 3), dtype=dt, device=dev)
    W = torch.empty((n, 3), dtype=dt, device=dev) if want_W else None
    with fcm.Handle(fcm.make_params(L, M, Sigma, rc, MG, n, prec)) as h:
        it = h.brownian(n, pos, KT, xid, zd, U, W, max_iter=max_iter, tol=tol,
                        stream=torch.cuda.current_stream().cuda_stream)
    return U.double().cpu().numpy(), (W.double().cpu().numpy() if W is not None else None), it


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_grid_part_matches_the_oracle(fcm, precision):
    prec = fcm.FCM_FP32 if precision == "fp32" else fcm.FCM_FP64
    Y, xi, z, L, M, MG, Sigma, rc = _setup()
    U, W, it = _run(fcm, prec, Y, xi, None, L, M, MG, Sigma, rc)
    assert it == 0
    Yr, xir = rounded(Y, prec), rounded(xi, prec)
    Uo, Wo = ob.brownian_grid(Yr, xir.transpose(0, 3, 2, 1), L, MG, Sigma, Sigma, KT)
    tol = FP32_TOL if precision == "fp32" else FP64_TOL
    assert_parity(U, Uo, tol, f"U Brownian grid part {precision}")
    assert_parity(W, Wo, tol, f"W Brownian grid part {precision}")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_pair_part_matches_the_exact_square_root(fcm, precision):
    prec = fcm.FCM_FP32 if precision == "fp32" else fcm.FCM_FP64
    Y, xi, z, L, M, MG, Sigma, rc = _setup(n=300, L=30.0, M=24, Sigma=2.0, seed=91)
    tol = 1e-6 if precision == "fp32" else 1e-11
    U, _, it = _run(fcm, prec, Y, None, z, L, M, MG, Sigma, rc, tol=tol, want_W=False)
    assert 2 <= it <= 60, it
    Uo = ob.brownian_pair(rounded(Y, prec), rounded(z, prec), L, rc, Sigma, KT)
    bar = FP32_TOL if precision == "fp32" else 1e-9
    assert_parity(U, Uo, bar, f"U Brownian pair part {precision} ({it} Lanczos iterations)")


def test_both_parts_add(fcm):
    prec = fcm.FCM_FP64
    Y, xi, z, L, M, MG, Sigma, rc = _setup(n=200, L=30.0, M=24, Sigma=2.0, seed=92)
    U, W, _ = _run(fcm, prec, Y, xi, z, L, M, MG, Sigma, rc)
    Ug, Wg = ob.brownian_grid(Y, xi.transpose(0, 3, 2, 1), L, MG, Sigma, Sigma, KT)
    Up = ob.brownian_pair(Y, z, L, rc, Sigma, KT)
    assert_parity(U, Ug + Up, 1e-9, "U Brownian both parts")
    assert_parity(W, Wg, FP64_TOL, "W Brownian (grid part only)")


def test_bad_arguments_are_rejected(fcm):
    import torch
    Y, xi, z, L, M, MG, Sigma, rc = _setup(n=50, L=24.0, M=16, Sigma=1.5, seed=93)
    with fcm.Handle(fcm.make_params(L, M, Sigma, rc, MG, 50, fcm.FCM_FP32)) as h:
        pos = torch.as_tensor(Y, dtype=torch.float32, device="cuda")
        U = torch.empty_like(pos)
        for kw, msg in ((dict(kT=0.0), "kT"), (dict(max_iter=0), "max_iter"), (dict(max_iter=65), "max_iter"),
                        (dict(tol=0.0), "tol")):
            args = dict(kT=1.0, max_iter=10, tol=1e-6)
            args.update(kw)
            with pytest.raises(fcm.FcmError) as e:
                h.brownian(50, pos, args["kT"], None, None, U, None, max_iter=args["max_iter"], tol=args["tol"])
            assert e.value.code == fcm.FCM_ERR_ARG and msg in str(e.value)
