"""The autotuner on the GPU: timed candidates, and the tuned parameters' accuracy through the C-ABI."""
import numpy as np
import pytest

from gpu_util import ensure_built, torch_cuda
from oracle import spectral_sum as ss
from paper_2310_12651_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fcm():
    torch_cuda()
    return ensure_built()


def _tensors(torch, Y, F, T):
    dev = torch.device("cuda:0")
    return tuple(torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float32, device=dev) for x in (Y, F, T))


def test_choose_times_the_cheapest_candidates(fcm):
    import torch
    from paper_2310_12651_gb300 import tune
    n, phi = 65536, 0.05
    L = inputs.box_edge(n, phi)
    Y = inputs.random_suspension(n, L, inputs.BASE_SEED + 50)
    F, T = inputs.random_loads(n, inputs.BASE_SEED + 51)
    pos, Fd, Td = _tensors(torch, Y, F, T)
    best = tune.choose(n, L, 1e-5, measure=tune.gpu_timer(pos, Fd, Td, L), top=3)
    top = tune.candidates(n, L, 1e-5)[:3]
    assert any(best["Sigma"] == c["Sigma"] for c in top)
    assert 0 < best["measured_s"] < 0.05, best


@pytest.mark.parametrize("tol", [1e-3, 1e-4])
def test_tuned_parameters_reach_the_tolerance_on_the_gpu(fcm, tol):
    """FP32 CUDA path with the tuner's first choice against the direct Fourier sum."""
    import torch
    from paper_2310_12651_gb300 import tune
    n, phi = 250, 0.2
    L = inputs.box_edge(n, phi)
    Y = inputs.random_suspension(n, L, inputs.BASE_SEED + 40)
    F, T = inputs.random_loads(n, inputs.BASE_SEED + 41)
    Ub, Wb = ss.apply(Y, F, T, L)
    pos, Fd, Td = _tensors(torch, Y, F, T)
    for c in tune.candidates(n, L, tol, max_grid=96)[:2]:
        with fcm.Handle(tune.make_params(c, L, n)) as h:
            U, W = fcm.apply_tensors(h, pos, Fd, Td)
            assert h.check() == 0
        U, W = U.double().cpu().numpy(), W.double().cpu().numpy()
        eu = np.mean(np.linalg.norm(U - Ub, axis=1) / np.linalg.norm(Ub, axis=1))
        ew = np.mean(np.linalg.norm(W - Wb, axis=1) / np.linalg.norm(Wb, axis=1))
        assert eu < tol and ew < tol, (c, eu, ew)
