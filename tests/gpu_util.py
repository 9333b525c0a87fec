"""Helpers of the GPU tests: run the CUDA path through the C-ABI on seeded
inputs and compare with the oracle element by element."""
import math

import numpy as np

from oracle import closed_forms as cf
from oracle import grid_fcm as og
from oracle import params as op
from paper_2310_12651_gb300 import inputs

FP32_TOL = 1e-4    # relative L2 bar of the FP32 path against the FP64 oracle
FP64_TOL = 1e-10   # relative L2 bar of the FP64 path against the FP64 oracle


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    return torch


def ensure_built():
    from paper_2310_12651_gb300 import build
    build.build()
    from paper_2310_12651_gb300 import fcm
    return fcm


def rounded(x, precision):
    """Inputs as the device sees them: FP32 runs get float32-rounded values."""
    if x is None:
        return None
    fcm = ensure_built()
    return np.asarray(x, dtype=np.float32 if precision == fcm.FCM_FP32 else np.float64).astype(np.float64)


class System:
    """A seeded periodic system plus the parameters both sides use."""

    def __init__(self, n, L, M, Sigma, M_G, r_c, seed, torques=True, Sigma_D=0.0, min_sep=2.2, Y=None):
        self.n, self.L, self.M, self.Sigma, self.M_G, self.r_c = n, L, M, Sigma, M_G, r_c
        self.Sigma_D = Sigma_D
        Lv = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,))
        if Y is None:
            if np.all(Lv == Lv[0]):
                Y = inputs.random_suspension(n, float(Lv[0]), seed, min_sep=min_sep)
            else:
                rng = np.random.default_rng(seed)
                Y = rng.random((n, 3)) * Lv
        self.Y = np.asarray(Y, dtype=np.float64)
        self.F, self.T = inputs.random_loads(n, seed + 1000, torques=torques)

    def oracle(self, precision, stages=3):
        Y, F, T = rounded(self.Y, precision), rounded(self.F, precision), rounded(self.T, precision)
        SD = self.Sigma_D if self.Sigma_D else self.Sigma
        U = np.zeros((self.n, 3))
        W = np.zeros((self.n, 3))
        if stages & 1:
            Ug, Wg = og.grid_apply(Y, F, T, self.L, self.M, self.M_G, self.Sigma, SD)
            U, W = U + Ug, W + Wg
        if stages & 2:
            Up, Wp = og.pair_correction(Y, F, T, self.L, self.r_c, self.Sigma, SD)
            U, W = U + Up, W + Wp
        return U, W


def params_for(fcm, s: System, precision, max_n=None, tile=(0, 0, 0)):
    return fcm.make_params(s.L, s.M, s.Sigma, s.r_c, s.M_G, max_n or max(s.n, 1), precision,
                           Sigma_D=s.Sigma_D, tile=tile)


def run_gpu(s: System, precision, stages=3, want_W=True, tile=(0, 0, 0), handle=None, Y=None):
    torch = torch_cuda()
    fcm = ensure_built()
    dt = torch.float32 if precision == fcm.FCM_FP32 else torch.float64
    dev = torch.device("cuda:0")
    Yd = s.Y if Y is None else Y
    pos = torch.as_tensor(np.ascontiguousarray(Yd), dtype=dt, device=dev)
    F = torch.as_tensor(s.F, dtype=dt, device=dev)
    T = torch.as_tensor(s.T, dtype=dt, device=dev) if s.T is not None else None
    own = handle is None
    h = handle or fcm.Handle(params_for(fcm, s, precision, tile=tile))
    try:
        U, W = fcm.apply_tensors(h, pos, F, T, want_W=want_W, stages=stages)
        flags = h.check()
    finally:
        if own:
            h.close()
    assert flags == 0, f"device status flags {flags}"
    Un = U.double().cpu().numpy()
    Wn = W.double().cpu().numpy() if W is not None else None
    return Un, Wn


def rel_l2(got, ref):
    return float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))


def assert_parity(got, ref, tol, what=""):
    """Relative L2 below tol and every element within 10 tol of the rms of the reference."""
    rl = rel_l2(got, ref)
    rms = math.sqrt(float(np.mean(ref * ref))) if ref.size else 0.0
    worst = float(np.max(np.abs(got - ref))) / max(rms, 1e-300) if ref.size else 0.0
    print(f"{what}: rel L2 {rl:.3e}, max element error / rms {worst:.3e}")
    assert rl <= tol, f"{what}: relative L2 error {rl:.3e} > {tol:.1e}"
    assert worst <= 10 * tol, f"{what}: element error {worst:.3e} rms > {10 * tol:.1e}"


def suspension(n, phi, M, Sigma, tol, seed, torques=True, c_trunc=4.8):
    """A random suspension shaped like the paper's (min separation 2.2a), parameters from the rules."""
    L = inputs.box_edge(n, phi)
    h = L / M
    MG = min(op.support_points(Sigma, h, c_trunc), 24, M)
    rc = min(op.cutoff_radius(Sigma, tol, torques=torques), 0.5 * L)
    return System(n, L, M, Sigma, MG, rc, seed, torques=torques)


SIGMA = cf.fcm_sigma()
SIGMA_D = cf.fcm_sigma_D()
