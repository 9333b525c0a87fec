"""Host logic of bench.py for N > 1 ranks (replicas, max over ranks), on CPU with gloo."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slowest = bench.max_over_ranks(10.0 + rank, world, None)
        bench.barrier(world)
        out[rank] = slowest
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world_2():
    import torch.multiprocessing as mp
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert dict(out) == {0: 11.0, 1: 11.0}


def test_workload_parameters_match_the_documented_rules():
    sys.path.insert(0, ROOT)
    import bench
    w = bench.workload("c2")
    assert w["n"] == 65536 and w["M"] == 128 and w["M_G"] == 14
    assert abs(w["L"] - 176.41391792668995) < 1e-9
    from oracle import params
    assert abs(w["r_c"] - params.cutoff_radius(2.0, 1e-6, torques=True)) < 1e-6
    small = bench.workload("c2", n=16384, h_ref=w["h"])
    assert abs(small["h"] - w["h"]) / w["h"] < 0.02 and small["M_G"] == 14


@pytest.mark.parametrize("n_rods, tol", [(7744, 1e-4), (2304, 1e-4), (16, 1e-4), (2304, 1e-6)])
def test_rod_suspension_parameters_follow_the_rules(n_rods, tol):
    """The rod-suspension parameters: Sigma resolved at the tolerance's Table 1 ratio on the coarser
    spacing, the window rule for M_G, FFT-friendly even grids, and a cutoff inside half the 60a height."""
    import math
    sys.path.insert(0, ROOT)
    import bench
    from paper_2310_12651_gb300 import tune
    L_xy, L_z = 960.0 * math.sqrt(n_rods / 2304.0), 60.0
    pr = bench.rod_suspension_params(L_xy, L_z, 22 * n_rods, tol)
    Mx, My, Mz = pr["M"]
    h = max(L_xy / Mx, L_z / Mz)
    assert Mx == My and all(m % 2 == 0 and tune._smooth(m) for m in pr["M"])
    assert pr["Sigma"] / h >= tune.resolution_for(tune.GRID_SHARE * tol) - 1e-12
    assert pr["M_G"] == tune.support_points(pr["Sigma"], min(L_xy / Mx, L_z / Mz), tune.truncation_for(tune.GRID_SHARE * tol))
    assert 0 < pr["r_c"] <= 0.5 * L_z and pr["M_G"] <= min(24, Mz)
    assert pr["r_c"] >= tune.cutoff(pr["Sigma"], 0.5 * tol, torques=False) - 1e-9


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the FP64 oracle on a bounded sample, host cores only) prints one JSON line
    with the contract's keys, its own cpu_baseline and an e2e object with zero copy bytes."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["dtype"] == "f64" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_oracle_legs_load_nothing_of_the_product():
    """The reference arm and the CPU baseline take their parameters from oracle/params.py: after a
    reference-arm run the process has neither mapped libfcm.so nor imported the binding or the tuner."""
    import subprocess
    code = (
        "import sys, argparse, io, contextlib; sys.path.insert(0, %r)\n"
        "import bench\n"
        "a = argparse.Namespace(steps=1, warmup=0, gpus=1, workload='c2')\n"
        "with contextlib.redirect_stdout(io.StringIO()):\n"
        "    bench.reference_arm(a, 1, 0)\n"
        "w = bench.oracle_workload('c2')\n"
        "maps = open('/proc/self/maps').read()\n"
        "assert 'libfcm' not in maps, 'libfcm.so mapped'\n"
        "bad = [m for m in sys.modules if m.startswith('paper_2310_12651_gb300.') and m != 'paper_2310_12651_gb300.inputs']\n"
        "assert not bad, bad\n"
        "print('ok', w['M_G'], w['r_c'])\n" % ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    ok, mg, rc = r.stdout.split()
    assert ok == "ok" and int(mg) == 14
    import bench
    assert abs(float(rc) - bench.workload("c2")["r_c"]) < 1e-6
