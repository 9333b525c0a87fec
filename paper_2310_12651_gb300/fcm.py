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

(FCM_OK, FCM_ERR_ARG, FCM_ERR_OOM, FCM_ERR_CUDA, FCM_ERR_CUFFT, FCM_ERR_TIMEOUT, FCM_ERR_INPUT, FCM_ERR_BUSY,
 FCM_ERR_CANCELED, FCM_ERR_NOT_CONVERGED) = range(10)
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


class Request(ctypes.Structure):
    _fields_ = [
        ("params", Params),
        ("n", ctypes.c_int),
        ("pos", ctypes.c_void_p),
        ("F", ctypes.c_void_p),
        ("T", ctypes.c_void_p),
        ("U", ctypes.c_void_p),
        ("W", ctypes.c_void_p),
    ]


class ServerStats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_longlong) for name in
                ("submitted", "completed", "rejected", "canceled", "failed", "pending", "batches", "batched_requests",
                 "handles_created", "handles_evicted", "graph_passes")] + [
        ("hbm_bytes", ctypes.c_size_t),
        ("hbm_budget", ctypes.c_size_t),
        ("latency_p50_us", ctypes.c_double),
        ("latency_p99_us", ctypes.c_double),
        ("latency_max_us", ctypes.c_double),
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
        "fcm_create_batch": (i, [ctypes.POINTER(Params), i, i, ctypes.POINTER(vp)]),
        "fcm_batch_apply": (i, [vp, i, ctypes.POINTER(i), vp, vp, vp, vp, vp, vp]),
        "fcm_batch_apply_stages": (i, [vp, i, ctypes.POINTER(i), vp, vp, vp, vp, vp, i, vp]),
        "fcm_max_systems": (i, [vp]),
        "fcm_brownian": (i, [vp, i, vp, d, vp, vp, vp, vp, i, d, ctypes.POINTER(i), vp]),
        "fcm_rigid_solve": (i, [vp, i, vp, i, vp, vp, vp, vp, vp, i, d, i, i, ctypes.POINTER(i), ctypes.POINTER(d), vp]),
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
        "fcm_server_create": (i, [i, sz, i, ctypes.POINTER(vp)]),
        "fcm_server_submit": (i, [vp, ctypes.POINTER(Request), ctypes.POINTER(ll)]),
        "fcm_server_poll": (i, [vp, ll, ll, ctypes.POINTER(i)]),
        "fcm_server_cancel": (i, [vp, ll]),
        "fcm_server_get_stats": (i, [vp, ctypes.POINTER(ServerStats)]),
        "fcm_server_reset_latency": (i, [vp]),
        "fcm_server_destroy": (i, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()

#: symbols declared in include/fcm.h, for the export check
EXPORTED = ("fcm_version", "fcm_params_default", "fcm_create", "fcm_destroy", "fcm_apply", "fcm_apply_stages",
            "fcm_create_batch", "fcm_batch_apply", "fcm_batch_apply_stages", "fcm_max_systems", "fcm_brownian",
            "fcm_rigid_solve", "fcm_spread", "fcm_copy_grid", "fcm_check", "fcm_set_timing", "fcm_read_timing",
            "fcm_launch_count",
            "fcm_workspace_bytes", "fcm_cutoff_radius", "fcm_pair_correction_noalloc", "fcm_last_error",
            "fcm_server_create", "fcm_server_submit", "fcm_server_poll", "fcm_server_cancel", "fcm_server_get_stats",
            "fcm_server_reset_latency", "fcm_server_destroy")

#: most systems of one batched pass (include/fcm.h)
MAX_BATCH = 1024
#: most Lanczos iterations of fcm_brownian (include/fcm.h)
LANCZOS_MAX_ITER = 64
#: most Broyden iterations of fcm_rigid_solve (include/fcm.h)
BROYDEN_MAX_ITER = 256
#: Broyden's starting Jacobian in fcm_rigid_solve, and the body preconditioner's size limit (include/fcm.h)
RIGID_PRECOND_DIAGONAL, RIGID_PRECOND_BODY = 0, 1
RIGID_BODY_MAX = 32

#: bits of the device status word returned by Handle.check (include/fcm.h)
STATUS_NONFINITE, STATUS_WAIT_TIMEOUT = 1, 2

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
    """fcm_params for fcm_create (include/fcm.h). spread_kernel: 0 = the library's choice (pencil kernel),
    1 = row-stationary per pair of tiles, 2 = shared-memory atomics, 3 = tensor cores per pair of tiles,
    4 = tensor cores along pencils (3, 4: 8^3 tiles and M_G in {10, 12, 14}, 4 also Sigma_D = Sigma;
    otherwise as 0)."""
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

    def __init__(self, params: Params, device: int = 0, max_systems: int = 1):
        self._h = ctypes.c_void_p()
        _check(_lib.fcm_create_batch(ctypes.byref(params), int(max_systems), int(device), ctypes.byref(self._h)))
        self.params = params
        self.device = device
        self.max_systems = int(max_systems)

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

    def batch_apply(self, offsets, pos, F, T, U, W, stream=0, stages=STAGE_ALL):
        """Stacked systems: system s owns rows offsets[s] .. offsets[s+1]-1 (host sequence of ints)."""
        n_sys = len(offsets) - 1
        arr = (ctypes.c_int * max(len(offsets), 1))(*[int(v) for v in offsets])
        _check(_lib.fcm_batch_apply_stages(self._h, int(n_sys), arr, _ptr(pos), _ptr(F), _ptr(T), _ptr(U), _ptr(W),
                                           int(stages), stream or None))

    def brownian(self, n, pos, kT, xi, z, U, W=None, max_iter=40, tol=1e-6, stream=0) -> int:
        """Brownian increment velocity (positive splitting); returns the Lanczos iterations used."""
        it = ctypes.c_int()
        _check(_lib.fcm_brownian(self._h, int(n), _ptr(pos), float(kT), _ptr(xi), _ptr(z), _ptr(U), _ptr(W),
                                 int(max_iter), float(tol), ctypes.byref(it), stream or None))
        return it.value

    def rigid_solve(self, n, pos, n_bodies, body_off, X, ft, F, UG, max_iter=100, tol=1e-4, warm=False,
                    stream=0, check=True, precond=RIGID_PRECOND_DIAGONAL):
        """Rigid-body mobility solve (Broyden); returns (status, iterations, relative residual).

        Raises FcmError on any status but FCM_OK, except FCM_ERR_NOT_CONVERGED when ``check`` is False.
        """
        it, res = ctypes.c_int(), ctypes.c_double()
        code = _lib.fcm_rigid_solve(self._h, int(n), _ptr(pos), int(n_bodies), _ptr(body_off), _ptr(X), _ptr(ft),
                                    _ptr(F), _ptr(UG), int(max_iter), float(tol), int(precond), 1 if warm else 0,
                                    ctypes.byref(it), ctypes.byref(res), stream or None)
        if code != FCM_OK and (check or code != FCM_ERR_NOT_CONVERGED):
            _check(code)
        return code, it.value, res.value

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


# ---- serving engine ------------------------------------------------------------------

class Ticket:
    """A submitted request: its id and the host arrays the server reads and writes."""

    def __init__(self, rid, arrays, U, W):
        self.id = rid
        self._arrays = arrays   # keeps inputs alive until the request is done
        self.U = U
        self.W = W
        self.status = None


class Server:
    """fcm_server_*: requests of any size and box from any thread, batched per grid class on one GPU.

    ``submit`` takes C-contiguous numpy arrays of shape (n, 3) (float32 for FCM_FP32 parameters,
    float64 for FCM_FP64) and returns a Ticket whose U (and W) arrays hold the result once ``wait``
    reports it done."""

    def __init__(self, device=0, hbm_budget=8 << 30, max_batch=64):
        self._s = ctypes.c_void_p()
        _check(_lib.fcm_server_create(int(device), int(hbm_budget), int(max_batch), ctypes.byref(self._s)))

    def close(self):
        if self._s:
            _check(_lib.fcm_server_destroy(self._s))
            self._s = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, params: Params, pos, F, T=None, want_W=True) -> Ticket:
        import numpy as np
        dt = np.float64 if params.precision == FCM_FP64 else np.float32
        arrs = []
        for a in (pos, F, T):
            if a is None:
                arrs.append(None)
                continue
            a = np.ascontiguousarray(a, dtype=dt)
            if a.ndim != 2 or a.shape[1] != 3:
                raise ValueError("pos, F, T must have shape (n, 3)")
            arrs.append(a)
        n = arrs[0].shape[0]
        U = np.empty((n, 3), dtype=dt)
        W = np.empty((n, 3), dtype=dt) if (want_W or T is not None) else None
        r = Request()
        r.params = params
        r.n = n
        r.pos, r.F = arrs[0].ctypes.data, arrs[1].ctypes.data
        r.T = arrs[2].ctypes.data if arrs[2] is not None else None
        r.U = U.ctypes.data
        r.W = W.ctypes.data if W is not None else None
        rid = ctypes.c_longlong()
        _check(_lib.fcm_server_submit(self._s, ctypes.byref(r), ctypes.byref(rid)))
        return Ticket(rid.value, arrs, U, W)

    def wait(self, t: Ticket, timeout_s: float = 60.0) -> bool:
        """True once done (t.status holds its result code), False if still running after timeout_s."""
        if t.status is not None:
            return True
        st = ctypes.c_int()
        code = _lib.fcm_server_poll(self._s, t.id, int(timeout_s * 1e6), ctypes.byref(st))
        if code == FCM_ERR_TIMEOUT:
            return False
        _check(code)
        t.status = st.value
        return True

    def cancel(self, t: Ticket) -> bool:
        """True if removed before launch, False if it already launched."""
        code = _lib.fcm_server_cancel(self._s, t.id)
        if code == FCM_ERR_BUSY:
            return False
        _check(code)
        return True

    def stats(self) -> dict:
        st = ServerStats()
        _check(_lib.fcm_server_get_stats(self._s, ctypes.byref(st)))
        return {name: getattr(st, name) for name, _ in ServerStats._fields_}

    def reset_latency(self):
        _check(_lib.fcm_server_reset_latency(self._s))
