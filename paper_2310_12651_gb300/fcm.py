"""ctypes binding of libfcm (include/fcm.h): argument marshalling only.

Every computation runs inside the compiled library. Pointers are plain
integers (device addresses); ``*_tensors`` helpers accept torch tensors and
pass their ``data_ptr()`` and the current CUDA stream. The library must have
been built (``paper_2310_12651_gb300.build.build()``); importing this module
raises if ``libfcm.so`` is missing, there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfcm.so")

FCM_OK, FCM_ERR_ARG, FCM_ERR_OOM, FCM_ERR_CUDA, FCM_ERR_CUFFT, FCM_ERR_TIMEOUT, FCM_ERR_INPUT = range(7)
FCM_FP32, FCM_FP64 = 0, 1
STAGE_GRID, STAGE_PAIR, STAGE_ALL = 1, 2, 3
NUM_STAGES = 6
STAGE_NAMES = ("binning", "spread", "fft_solve", "gather", "pair", "apply")


class FcmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libfcm error {code}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_double * 3),
        ("M", ctypes.c_int * 3),
        ("a", ctypes.c_double),
        ("eta", ctypes.c_double),
        ("Sigma", ctypes.c_double),
        ("Sigma_D", ctypes.c_double),
        ("r_c", ctypes.c_double),
        ("M_G", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("max_n", ctypes.c_int),
        ("tile", ctypes.c_int * 3),
        ("spread_kernel", ctypes.c_int),
    ]


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2310_12651_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, d, ll, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong, ctypes.c_size_t
    sig = {
        "fcm_version": (i, []),
        "fcm_params_default": (i, [ctypes.POINTER(Params)]),
        "fcm_create": (i, [ctypes.POINTER(Params), i, ctypes.POINTER(vp)]),
        "fcm_destroy": (i, [vp]),
        "fcm_apply": (i, [vp, i, vp, vp, vp, vp, vp, vp]),
        "fcm_apply_stages": (i, [vp, i, vp, vp, vp, vp, vp, i, vp]),
        "fcm_spread": (i, [vp, i, vp, vp, vp, vp]),
        "fcm_copy_grid": (i, [vp, vp, vp]),
        "fcm_check": (i, [vp, vp, i, ctypes.POINTER(i)]),
        "fcm_set_timing": (i, [vp, i]),
        "fcm_read_timing": (i, [vp, ctypes.POINTER(d), ctypes.POINTER(ll)]),
        "fcm_launch_count": (ll, [vp]),
        "fcm_workspace_bytes": (sz, [vp]),
        "fcm_cutoff_radius": (i, [d, d, d, d, d, i, ctypes.POINTER(d)]),
        "fcm_pair_correction_noalloc": (i, [ctypes.POINTER(Params), i, vp, vp, vp, vp, vp, vp]),
        "fcm_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()

#: symbols declared in include/fcm.h, for the export check
EXPORTED = ("fcm_version", "fcm_params_default", "fcm_create", "fcm_destroy", "fcm_apply", "fcm_apply_stages",
            "fcm_spread", "fcm_copy_grid", "fcm_check", "fcm_set_timing", "fcm_read_timing", "fcm_launch_count",
            "fcm_workspace_bytes", "fcm_cutoff_radius", "fcm_pair_correction_noalloc", "fcm_last_error")

#: capacity of fcm_pair_correction_noalloc's fixed scratch (include/fcm.h)
NOALLOC_MAX_N = 65536
NOALLOC_MAX_CELLS = 65536


def library():
    return _lib


def _check(code: int):
    if code != FCM_OK:
        raise FcmError(code, _lib.fcm_last_error().decode())


def version() -> int:
    return _lib.fcm_version()


def make_params(L, M, Sigma, r_c, M_G, max_n, precision=FCM_FP32, a=1.0, eta=1.0, Sigma_D=0.0, tile=(0, 0, 0),
                spread_kernel=0):
    p = Params()
    _check(_lib.fcm_params_default(ctypes.byref(p)))
    Ls = [float(L)] * 3 if not hasattr(L, "__len__") else [float(v) for v in L]
    Ms = [int(M)] * 3 if not hasattr(M, "__len__") else [int(v) for v in M]
    for k in range(3):
        p.L[k] = Ls[k]
        p.M[k] = Ms[k]
        p.tile[k] = int(tile[k])
    p.a, p.eta, p.Sigma, p.Sigma_D, p.r_c = float(a), float(eta), float(Sigma), float(Sigma_D), float(r_c)
    p.M_G, p.precision, p.max_n = int(M_G), int(precision), int(max_n)
    p.spread_kernel = int(spread_kernel)
    return p


def cutoff_radius(Sigma, tol, Sigma_D=0.0, a=1.0, eta=1.0, torques=False) -> float:
    out = ctypes.c_double()
    _check(_lib.fcm_cutoff_radius(float(Sigma), float(Sigma_D), float(a), float(eta), float(tol),
                                  1 if torques else 0, ctypes.byref(out)))
    return out.value


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


class Handle:
    """One periodic system's workspace on one GPU (fcm_create / fcm_destroy)."""

    def __init__(self, params: Params, device: int = 0):
        self._h = ctypes.c_void_p()
        _check(_lib.fcm_create(ctypes.byref(params), int(device), ctypes.byref(self._h)))
        self.params = params
        self.device = device

    def close(self):
        if self._h:
            _check(_lib.fcm_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def ptr(self) -> int:
        return self._h.value

    def apply(self, n, pos, F, T, U, W, stream=0):
        _check(_lib.fcm_apply(self._h, int(n), _ptr(pos), _ptr(F), _ptr(T), _ptr(U), _ptr(W), stream or None))

    def apply_stages(self, n, pos, F, T, U, W, stages, stream=0):
        _check(_lib.fcm_apply_stages(self._h, int(n), _ptr(pos), _ptr(F), _ptr(T), _ptr(U), _ptr(W), int(stages),
                                     stream or None))

    def spread(self, n, pos, F, T, stream=0):
        _check(_lib.fcm_spread(self._h, int(n), _ptr(pos), _ptr(F), _ptr(T), stream or None))

    def copy_grid(self, dst, stream=0):
        _check(_lib.fcm_copy_grid(self._h, _ptr(dst), stream or None))

    def check(self, stream=0, timeout_ms=10000) -> int:
        flags = ctypes.c_int()
        code = _lib.fcm_check(self._h, stream or None, int(timeout_ms), ctypes.byref(flags))
        if code not in (FCM_OK, FCM_ERR_INPUT):
            _check(code)
        return flags.value

    def set_timing(self, enable: bool):
        _check(_lib.fcm_set_timing(self._h, 1 if enable else 0))

    def read_timing(self):
        ms = (ctypes.c_double * NUM_STAGES)()
        cnt = (ctypes.c_longlong * NUM_STAGES)()
        _check(_lib.fcm_read_timing(self._h, ms, cnt))
        return {STAGE_NAMES[k]: (ms[k], cnt[k]) for k in range(NUM_STAGES)}

    def launch_count(self) -> int:
        return int(_lib.fcm_launch_count(self._h))

    def workspace_bytes(self) -> int:
        return int(_lib.fcm_workspace_bytes(self._h))


def pair_correction_noalloc(params: Params, n, pos, F, T, U, W, stream=0):
    """(M - M~)(F, T) through the entry point that allocates no device memory."""
    _check(_lib.fcm_pair_correction_noalloc(ctypes.byref(params), int(n), _ptr(pos), _ptr(F), _ptr(T), _ptr(U),
                                            _ptr(W), stream or None))


# ---- torch helpers (memory and streams only) ------------------------------------

def _stream_of(stream):
    if stream is not None:
        return stream
    import torch
    return torch.cuda.current_stream().cuda_stream


def apply_tensors(handle: Handle, pos, F, T=None, U=None, W=None, want_W=True, stages=STAGE_ALL, stream=None):
    """(U, W) = M (F, T) for torch CUDA tensors of shape (n, 3); allocates U, W if not given."""
    import torch
    n = pos.shape[0]
    for t in (pos, F, T):
        if t is not None and not (t.is_cuda and t.is_contiguous() and t.shape == (n, 3)):
            raise ValueError("pos, F, T must be contiguous CUDA tensors of shape (n, 3)")
    if U is None:
        U = torch.empty_like(F)
    if W is None and (want_W or T is not None):
        W = torch.empty_like(F)
    handle.apply_stages(n, pos, F, T, U, W, stages, _stream_of(stream))
    return U, W
