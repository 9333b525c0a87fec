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
