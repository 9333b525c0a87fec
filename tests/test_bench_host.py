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
