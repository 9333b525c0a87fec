"""The C-ABI library without a GPU: it loads, exports every declared symbol,
rejects bad parameters on the host, and its host-side cutoff rule agrees with
the oracle's (no kernel runs here)."""
import ctypes
import os
import re

import pytest

from oracle import params as oracle_params

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fcm():
    from paper_2310_12651_gb300 import build
    build.build()
    from paper_2310_12651_gb300 import fcm as mod
    return mod


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "fcm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fcm_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(fcm):
    lib = ctypes.CDLL(fcm.LIB_PATH)
    names = _declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(fcm.EXPORTED)


def test_params_struct_matches_header(fcm):
    text = open(os.path.join(ROOT, "include", "fcm.h")).read()
    body = re.search(r"typedef struct fcm_params \{(.*?)\} fcm_params;", text, re.S).group(1)
    fields = re.findall(r"^\s*(?:double|int)\s+(\w+)", body, re.M)
    assert fields == [f[0] for f in fcm.Params._fields_]
    assert ctypes.sizeof(fcm.Params) == 3 * 8 + 3 * 4 + 4 + 5 * 8 + 3 * 4 + 3 * 4 + 4 + 4


@pytest.mark.parametrize("change, message", [
    (dict(Sigma=0.3), "Sigma must be >= sigma"),
    (dict(M_G=80), "M_G"),
    (dict(M_G=0), "M_G"),
    (dict(r_c=60.0), "r_c"),
    (dict(r_c=0.0), "r_c"),
    (dict(eta=-1.0), "eta"),
    (dict(L=float("nan")), "L must"),
    (dict(precision=7), "precision"),
    (dict(Sigma_D=0.1), "Sigma_D"),
    (dict(r_c=1e-9), "pair cells"),
])
def test_invalid_parameters_are_rejected_on_the_host(fcm, change, message):
    kw = dict(L=100.0, M=64, Sigma=2.0, r_c=16.9, M_G=12, max_n=10)
    kw.update(change)
    p = fcm.make_params(**kw)
    with pytest.raises(fcm.FcmError) as e:
        fcm.Handle(p)
    assert e.value.code in (fcm.FCM_ERR_ARG, fcm.FCM_ERR_CUDA)
    if e.value.code == fcm.FCM_ERR_ARG:
        assert message in str(e.value)


@pytest.mark.parametrize("Sigma, tol, torques", [(2.0, 1e-8, False), (2.0, 1e-6, True), (1.5, 1e-4, True),
                                                 (3.0, 1e-6, False), (0.9, 1e-10, True)])
def test_cutoff_rule_matches_oracle(fcm, Sigma, tol, torques):
    ours = fcm.cutoff_radius(Sigma, tol, torques=torques)
    ref = oracle_params.cutoff_radius(Sigma, tol, torques=torques)
    assert abs(ours - ref) < 1e-6 * ref


def test_last_error_is_a_message(fcm):
    assert isinstance(fcm.library().fcm_last_error(), bytes)


@pytest.mark.parametrize("max_systems", [0, -3, 1025])
def test_batch_handle_rejects_bad_system_counts(fcm, max_systems):
    p = fcm.make_params(L=100.0, M=64, Sigma=2.0, r_c=16.9, M_G=12, max_n=10)
    with pytest.raises(fcm.FcmError) as e:
        fcm.Handle(p, max_systems=max_systems)
    assert e.value.code == fcm.FCM_ERR_ARG and "max_systems" in str(e.value)


def _struct_fields(name):
    text = open(os.path.join(ROOT, "include", "fcm.h")).read()
    body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (name, name), text, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        parts = [p.strip().lstrip("*") for p in decl.split(",")]
        first = parts[0].split()[-1].lstrip("*")
        names.append(first)
        names.extend(parts[1:])
    return names


def test_server_structs_match_header(fcm):
    assert _struct_fields("fcm_request") == [f[0] for f in fcm.Request._fields_]
    assert _struct_fields("fcm_server_stats") == [f[0] for f in fcm.ServerStats._fields_]
    assert ctypes.sizeof(fcm.Request) == 112 + 8 + 5 * 8
    assert ctypes.sizeof(fcm.ServerStats) == 11 * 8 + 2 * 8 + 3 * 8


@pytest.mark.parametrize("budget, max_batch, message", [(0, 4, "hbm_budget"), (1 << 30, 0, "max_batch"),
                                                        (1 << 30, 5000, "max_batch")])
def test_server_rejects_bad_arguments_on_the_host(fcm, budget, max_batch, message):
    with pytest.raises(fcm.FcmError) as e:
        fcm.Server(hbm_budget=budget, max_batch=max_batch)
    assert e.value.code == fcm.FCM_ERR_ARG and message in str(e.value)


def test_status_codes_match_header(fcm):
    text = open(os.path.join(ROOT, "include", "fcm.h")).read()
    codes = dict((k, int(v)) for k, v in re.findall(r"\b(FCM_(?:OK|ERR_[A-Z_]+))\s*=\s*(\d+)", text))
    assert codes == {k: getattr(fcm, k) for k in codes} and codes["FCM_ERR_NOT_CONVERGED"] == 9
    assert len(codes) == 10


def test_rigid_solve_rejects_a_null_handle_on_the_host(fcm):
    """Argument checks run before any CUDA call, so they work without a device."""
    it, res = ctypes.c_int(7), ctypes.c_double(3.0)
    lib = fcm.library()
    code = lib.fcm_rigid_solve(None, 10, None, 1, None, None, None, None, None, 10, 1e-4, 0, 0, ctypes.byref(it),
                               ctypes.byref(res), None)
    assert code == fcm.FCM_ERR_ARG and b"handle is NULL" in lib.fcm_last_error()
    assert it.value == 0 and res.value == 0.0
    header = open(os.path.join(ROOT, "include", "fcm.h")).read()
    for name, value in (("FCM_BROYDEN_MAX_ITER", fcm.BROYDEN_MAX_ITER), ("FCM_RIGID_BODY_MAX", fcm.RIGID_BODY_MAX),
                        ("FCM_RIGID_PRECOND_DIAGONAL", fcm.RIGID_PRECOND_DIAGONAL),
                        ("FCM_RIGID_PRECOND_BODY", fcm.RIGID_PRECOND_BODY),
                        ("FCM_STATUS_NONFINITE", fcm.STATUS_NONFINITE),
                        ("FCM_STATUS_WAIT_TIMEOUT", fcm.STATUS_WAIT_TIMEOUT)):
        assert value == int(re.search(r"#define " + name + r" (\d+)", header).group(1)), name
