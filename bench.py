#!/usr/bin/env python
"""Throughput of the fast-FCM mobility product (U, W) = M (F, T) on GB300.

One step = one pass of the whole hot path (binning, spread, FFT Stokes solve,
gather, pair correction) over one batch of ``--batch`` independent periodic
systems, each a seeded uniform suspension of N = 65,536 spheres at 5% volume
fraction (L = 176.41a) on a 128^3 grid with Sigma = 2a, forces and torques,
FP32. The systems are stacked along the particle axis and the step is one
fcm_batch_apply call (every stage one launch over all systems; ``--mode
single`` runs one fcm_apply per system instead). Every system's inputs stay
resident in HBM; L2 is flushed (256 MB write) before every step and each step
is timed with CUDA events on the stream it runs on. ``value`` = particles
processed / summed step time.

``e2e`` repeats the measurement through the same C-ABI call with host
buffers: pinned host -> device copies of pos, F, T and device -> host copies of
U, W inside each timed step.

``--impl reference`` times the FP64 CPU oracle on the host cores instead, on a
bounded sample of the same workload (same density, Sigma, M_G, r_c; fewer
particles in a proportionally smaller box).

For N > 1 GPUs (torchrun) every rank runs the same batch on its own GPU
(replicas; no collective on the data path): value = all ranks' particles / the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-applies/s, FP32 batched vs FP64 plain at rel err≤1e-4; serve p50/p99"
UNIT = "particle-applies/s"
FLUSH_BYTES = 256 << 20
TRUNC = 4.8          # window half-width in Sigma (grid part error ~2e-5)
TOL = 1e-6           # pair cutoff tolerance
# Workloads: N per system, volume fraction, grid points per side, Sigma, default systems per step.
WORKLOADS = {
    "c2": dict(n=65536, phi=0.05, grid=128, Sigma=2.0, batch=32),
    "large": dict(n=1048576, phi=0.10, grid=256, Sigma=1.5, batch=2),
}
# dram__bytes_read.sum + dram__bytes_write.sum per system of a launch (cold caches), from one ncu capture of
# the current kernels; a launch over B systems moves B times this. None once a kernel changes after the capture.
TRAFFIC_BYTES = {"c2": {"spread": 29.16e6, "gather": 26.49e6, "pair": 4.75e6}}
# Algorithmic work per unit for the roofline (the hot-path scope table's figures): flops per (particle,
# window point) of the spread and of the gather, and per ordered pair within r_c of the pair correction;
# forces + torques and forces only.
FLOPS_POINT = {True: 22.0, False: 8.0}
FLOPS_PAIR = {True: 250.0, False: 100.0}


def workload(name="c2", n=None, h_ref=None):
    from paper_2310_12651_gb300 import inputs, tune
    spec = WORKLOADS[name]
    n = spec["n"] if n is None else n
    L = inputs.box_edge(n, spec["phi"])
    M = spec["grid"] if h_ref is None else max(8, int(round(L / h_ref)))
    h = L / M
    Sigma = spec["Sigma"]
    MG = tune.support_points(Sigma, h, TRUNC)
    rc = tune.cutoff(Sigma, TOL, torques=True)
    return dict(name=name, n=n, phi=spec["phi"], L=L, M=M, h=h, Sigma=Sigma, M_G=MG, r_c=rc)


def oracle_workload(name="c2", n=None, h_ref=None):
    """The same workload with its parameters taken from the oracle's own rules (oracle/params.py), so
    that the oracle's timed legs load nothing of the product (the two rules agree: tests/test_tune.py)."""
    from oracle import params as op
    from paper_2310_12651_gb300 import inputs
    spec = WORKLOADS[name]
    n = spec["n"] if n is None else n
    L = inputs.box_edge(n, spec["phi"])
    M = spec["grid"] if h_ref is None else max(8, int(round(L / h_ref)))
    h = L / M
    Sigma = spec["Sigma"]
    MG = op.support_points(Sigma, h, TRUNC)
    rc = op.cutoff_radius(Sigma, TOL, torques=True)
    return dict(name=name, n=n, phi=spec["phi"], L=L, M=M, h=h, Sigma=Sigma, M_G=MG, r_c=rc)


def describe(w, batch, precision="FP32"):
    return (f"uniform suspension, N={w['n']} spheres/system, phi={w['phi']:.0%} (L={w['L']:.2f}a), "
            f"{w['M']}^3 grid, Sigma={w['Sigma']}a, M_G={w['M_G']}, r_c={w['r_c']:.2f}a (1e-6 rule), "
            f"forces+torques, {precision}, batch of {batch} systems")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled in the background."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "50"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        self.t0 = time.time()

    def stop(self):
        self.t1 = time.time()
        if self.proc is None:
            return None
        time.sleep(0.06)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        rows = [r.split(",") for r in out.strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip() == "Active"})
        power = [float(r[3]) for r in rows if r[3].strip().replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(power) if power else None}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_cpu_oracle(w, seed, torques=True):
    """One oracle apply on workload w; returns seconds."""
    from oracle import grid_fcm
    from paper_2310_12651_gb300 import inputs
    Y = inputs.random_suspension(w["n"], w["L"], seed)
    F, T = inputs.random_loads(w["n"], seed + 1)
    t = time.perf_counter()
    grid_fcm.fast_fcm_apply(Y, F, T if torques else None, w["L"], w["M"], w["M_G"], w["Sigma"], w["r_c"])
    return time.perf_counter() - t


def _oracle_worker(args):
    w, seed = args
    return run_cpu_oracle(w, seed)


def cpu_baseline(name, target_s=15.0):
    """The oracle timed on a bounded sample of the workload (same density, spacing, Sigma, M_G, r_c):
    on one core, then on every host core at once (one independent sample system per core, as the
    batched workload is independent systems; worker processes started with spawn, one BLAS thread
    each)."""
    import multiprocessing as mp
    h_full = oracle_workload(name)["h"]
    n = 16384
    w = oracle_workload(name, n=n, h_ref=h_full)
    secs = run_cpu_oracle(w, 2310126590)
    reps = 1
    while secs * (reps + 1) / reps < target_s and reps < 4:
        secs += run_cpu_oracle(w, 2310126590 + reps)
        reps += 1
    one = n * reps / secs
    cores = len(os.sched_getaffinity(0))
    value, used, wall = one, 1, secs
    if cores > 1:
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"
        try:
            with mp.get_context("spawn").Pool(cores) as pool:
                pool.map(_oracle_worker, [(oracle_workload(name, n=512, h_ref=h_full), 1)] * cores)  # start-up
                t0 = time.perf_counter()
                pool.map(_oracle_worker, [(w, 2310126600 + k) for k in range(cores)])
                wall = time.perf_counter() - t0
            value, used = n * cores / wall, cores
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
    return {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"oracle applies of {n} spheres at phi={w['phi']:.0%} (L={w['L']:.1f}a, {w['M']}^3, "
                      f"h={w['h']:.3f}a, Sigma={w['Sigma']}a, M_G={w['M_G']}, r_c={w['r_c']:.2f}a), forces+torques, "
                      f"FP64 numpy: {used} at once on {used} cores ({wall:.1f} s wall); one core alone "
                      f"{reps} apply(s) in {secs:.1f} s",
            "one_core": {"value": one, "cores": 1},
            "host_cores": cores}


# ---- error against the FP64 oracle, per configuration (outside every timed region)
#
# The oracle runs in worker processes started with spawn (they never touch the GPU) while the GPU
# measurements run; the GPU results are compared afterwards. Full C2 systems are checked on a seeded
# sample of particles: the oracle's grid part needs the whole spread and FFT, so the spread is split
# over the workers and summed, then the velocity field is interpolated at the sample and the pair
# correction is summed for the sample alone.
ERR_SIGMAS = (1.5, 2.0, 3.0)
ERR_SAMPLE = 4096
ERR_SPREAD_CHUNKS = {1.5: 2, 2.0: 4, 3.0: 8}


def _c2_inputs(n, L, seed):
    """C2 inputs as the FP32 path sees them (rounded to float32, held in float64)."""
    import numpy as np
    from paper_2310_12651_gb300 import inputs
    Y = inputs.random_suspension(n, L, seed)
    F, T = inputs.random_loads(n, seed + 1)
    return tuple(np.asarray(a, dtype=np.float32).astype(np.float64) for a in (Y, F, T))


def _sigma_workload(Sigma):
    from oracle import params as op
    w = dict(oracle_workload("c2"))
    w["Sigma"] = Sigma
    w["M_G"] = op.support_points(Sigma, w["h"], TRUNC)
    w["r_c"] = op.cutoff_radius(Sigma, TOL, torques=True)
    return w


def _c1_params():
    """C1: N = 1,000 in a 100a box on 64^3, Sigma = 2a, window +-4 Sigma, r_c from the 1e-8 rule, forces only."""
    from oracle import params as op
    L, M, Sigma = 100.0, 64, 2.0
    return dict(n=1000, L=L, M=M, Sigma=Sigma, M_G=op.support_points(Sigma, L / M, 4.0),
                r_c=op.cutoff_radius(Sigma, 1e-8), seed=2310126510)


def _standard_grid(L, c=6.3, ratio=1.39):
    """Standard FCM (oracle-A) grid resolving sigma: sigma/h >= 1.39 (Table 1's 1e-8 row) on an
    FFT-friendly M, window +-6.3 sigma."""
    from oracle import closed_forms as cf
    from oracle import params as op
    sg = cf.fcm_sigma(1.0)
    M = max(8, int(math.ceil(L * ratio / sg)))
    while True:
        m = M
        for f in (2, 3, 5):
            while m % f == 0:
                m //= f
        if m == 1 and M % 2 == 0:
            break
        M += 1
    return M, op.support_points(sg, L / M, c)


def _oracle_error_job(job):
    import numpy as np
    from oracle import grid_fcm as og
    from paper_2310_12651_gb300 import inputs
    kind = job[0]
    if kind == "spread":                        # partial C2 grid of particles [a, b) at Sigma
        _, Sigma, a, b = job
        w = _sigma_workload(Sigma)
        Y, F, T = _c2_inputs(w["n"], w["L"], inputs.BASE_SEED + 1)
        return og.spread(Y[a:b], F[a:b], T[a:b], w["L"], w["M"], w["M_G"], Sigma, Sigma, fp32_windows=True)
    if kind == "finish":                         # solve, interpolate at the sample, pair sums for the sample
        _, Sigma, grid, idx = job
        w = _sigma_workload(Sigma)
        Y, F, T = _c2_inputs(w["n"], w["L"], inputs.BASE_SEED + 1)
        u = og.stokes_solve(grid, w["L"])
        Ug, Wg = og.interpolate(u, Y[idx], w["L"], w["M_G"], Sigma, Sigma)
        Up, Wp = og.pair_correction_subset(Y, F, T, w["L"], w["r_c"], Sigma, Sigma, idx)
        return Ug + Up, Wg + Wp
    if kind == "c1_fast":                        # oracle-C on C1 (FP64 inputs)
        c = _c1_params()
        Y = inputs.random_suspension(c["n"], c["L"], c["seed"])
        F, _ = inputs.random_loads(c["n"], c["seed"] + 1, torques=False)
        return og.fast_fcm_apply(Y, F, None, c["L"], c["M"], c["M_G"], c["Sigma"], c["r_c"])
    if kind == "c1_standard":                    # oracle-A on C1
        c = _c1_params()
        Y = inputs.random_suspension(c["n"], c["L"], c["seed"])
        F, _ = inputs.random_loads(c["n"], c["seed"] + 1, torques=False)
        M, MG = _standard_grid(c["L"])
        return og.standard_fcm_apply(Y, F, None, c["L"], M, MG)
    if kind == "c2s_standard":                   # oracle-A on a C2-density sample system (FP32-rounded inputs)
        _, n = job
        w = oracle_workload("c2", n=n, h_ref=oracle_workload("c2")["h"])
        Y, F, T = _c2_inputs(n, w["L"], inputs.BASE_SEED + 77)
        M, MG = _standard_grid(w["L"])
        return og.standard_fcm_apply(Y, F, T, w["L"], M, MG)
    raise ValueError(kind)


class OracleErrors:
    """Starts the oracle jobs at once (spawned workers), finishes them on demand."""

    def __init__(self, workers=None):
        import multiprocessing as mp
        import numpy as np
        self.n = WORKLOADS["c2"]["n"]
        self.idx = np.sort(np.random.default_rng(2310126531).choice(self.n, ERR_SAMPLE, replace=False))
        self.n_c2s = 4096
        cores = len(os.sched_getaffinity(0))
        self.pool = mp.get_context("spawn").Pool(workers or max(1, min(cores - 1, 16)))
        self.spread = {}
        for Sigma in ERR_SIGMAS:
            k = ERR_SPREAD_CHUNKS[Sigma]
            cuts = [self.n * i // k for i in range(k + 1)]
            self.spread[Sigma] = self.pool.map_async(_oracle_error_job,
                                                     [("spread", Sigma, cuts[i], cuts[i + 1]) for i in range(k)])
        self.c1_fast = self.pool.apply_async(_oracle_error_job, (("c1_fast",),))
        self.c1_std = self.pool.apply_async(_oracle_error_job, (("c1_standard",),))
        self.c2s_std = self.pool.apply_async(_oracle_error_job, (("c2s_standard", self.n_c2s),))

    def results(self, timeout=1800):
        finish = {}
        for Sigma in ERR_SIGMAS:
            grid = sum(self.spread[Sigma].get(timeout))
            finish[Sigma] = self.pool.apply_async(_oracle_error_job, (("finish", Sigma, grid, self.idx),))
        out = {"c2": {S: f.get(timeout) for S, f in finish.items()}, "c1_fast": self.c1_fast.get(timeout),
               "c1_standard": self.c1_std.get(timeout), "c2s_standard": self.c2s_std.get(timeout)}
        self.pool.close()
        self.pool.join()
        return out


def _errs(got, ref):
    """Relative L2 over all components and the paper's mean relative error (Section 5.1)."""
    import numpy as np
    got, ref = np.asarray(got, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    rn = np.linalg.norm(ref, axis=1)
    return {"rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
            "mean_rel": float(np.mean(np.linalg.norm(got - ref, axis=1) / np.where(rn > 0, rn, 1.0)))}


def error_vs_oracle(device, oracle_jobs):
    """FP32 (and FP64 plain) GPU results against the oracle, per configuration:
    * C2 at Sigma = 1.5, 2, 3a (system 0 of the bench, 128^3, forces + torques): FP32 against
      oracle-C (fast FCM, FP64) on a seeded sample of 4,096 particles;
    * C1 (N = 1,000, 64^3, forces only): the FP64 plain path against oracle-C;
    * the method's total error: the FP64 plain path on C1, and the FP32 path on a 4,096-sphere
      system at C2's density and parameters, against standard FCM (oracle-A on a sigma-resolving grid)."""
    import numpy as np
    import torch
    from paper_2310_12651_gb300 import fcm, inputs
    dev = torch.device("cuda", device)
    st = torch.cuda.current_stream(dev).cuda_stream
    ref = oracle_jobs.results()
    out = {"sample_particles": ERR_SAMPLE, "metrics": "rel_l2 over all components; mean_rel = (1/N) sum |V - U| / |U| "
                                                      "(Section 5.1)"}
    # both sides take the same parameter values (those of the oracle's rules)
    c2 = {}
    for Sigma in ERR_SIGMAS:
        sw = _sigma_workload(Sigma)
        n, L, MG, rc = sw["n"], sw["L"], sw["M_G"], sw["r_c"]
        Y, F, T = _c2_inputs(n, L, inputs.BASE_SEED + 1)
        pos, Fd, Td = (torch.as_tensor(a, dtype=torch.float32, device=dev) for a in (Y, F, T))
        with fcm.Handle(fcm.make_params(L, WORKLOADS["c2"]["grid"], Sigma, rc, MG, n, fcm.FCM_FP32), device) as hh:
            U, W = fcm.apply_tensors(hh, pos, Fd, Td, stream=st)
            assert hh.check() == 0
        Ug, Wg = U.double().cpu().numpy()[oracle_jobs.idx], W.double().cpu().numpy()[oracle_jobs.idx]
        Uo, Wo = ref["c2"][Sigma]
        c2[f"Sigma={Sigma}a"] = {"M_G": MG, "r_c": rc, "U": _errs(Ug, Uo), "W": _errs(Wg, Wo)}
    out["c2_fp32_vs_oracle"] = c2
    c = _c1_params()
    Y = inputs.random_suspension(c["n"], c["L"], c["seed"])
    F, _ = inputs.random_loads(c["n"], c["seed"] + 1, torques=False)
    pos, Fd = (torch.as_tensor(a, dtype=torch.float64, device=dev) for a in (Y, F))
    with fcm.Handle(fcm.make_params(c["L"], c["M"], c["Sigma"], c["r_c"], c["M_G"], c["n"], fcm.FCM_FP64), device) as hh:
        U, _ = fcm.apply_tensors(hh, pos, Fd, None, want_W=False, stream=st)
        assert hh.check() == 0
    U = U.cpu().numpy()
    Uf, _ = ref["c1_fast"]
    Us, _ = ref["c1_standard"]
    out["c1_fp64_vs_oracle"] = {"U": _errs(U, Uf)}
    out["c1_method_fp64_vs_standard_fcm"] = {"U": _errs(U, Us), "standard_grid": _standard_grid(c["L"])}
    w = oracle_workload("c2", n=4096, h_ref=oracle_workload("c2")["h"])
    MG, rc = w["M_G"], w["r_c"]
    Y, F, T = _c2_inputs(4096, w["L"], inputs.BASE_SEED + 77)
    pos, Fd, Td = (torch.as_tensor(a, dtype=torch.float32, device=dev) for a in (Y, F, T))
    with fcm.Handle(fcm.make_params(w["L"], w["M"], w["Sigma"], rc, MG, 4096, fcm.FCM_FP32), device) as hh:
        U, W = fcm.apply_tensors(hh, pos, Fd, Td, stream=st)
        assert hh.check() == 0
    Us, Ws = ref["c2s_standard"]
    out["c2_density_method_fp32_vs_standard_fcm"] = {
        "U": _errs(U.double().cpu().numpy(), Us), "W": _errs(W.double().cpu().numpy(), Ws),
        "system": f"N=4096 at phi=5% (L={w['L']:.1f}a, {w['M']}^3, Sigma={w['Sigma']}a, M_G={MG}, r_c={rc:.2f}a)",
        "standard_grid": _standard_grid(w["L"])}
    return out


def large_sweep(device, grids=(192, 256, 320), tol=1e-5, steps=3, warmup=2, seed=2310126800):
    """The large precision/roofline configuration: one system of N = 1,048,576 spheres at 10% (L =
    352.83a; uniform RSA, F and T i.i.d. N(0,1)), on 192^3, 256^3 and 320^3 grids, each with the
    (Sigma, M_G, r_c) the autotuner picks at tolerance tol for that grid (the three cheapest
    candidates of its cost model timed on the GPU). Per grid: particle-applies/s of fcm_apply (FP32,
    inputs resident, L2 flushed between applies, CUDA events), per-stage times, the FP32 ALU roofline
    of the dominant kernel, and the FP32 error against the FP64 plain path on the same GPU. This is
    the trade-off of the paper's Section 5.2 (grid against pairs, set by Sigma) at GB300 scale."""
    import numpy as np
    import torch
    from paper_2310_12651_gb300 import fcm, inputs, tune
    n, phi = 1048576, 0.10
    L = inputs.box_edge(n, phi)
    dev = torch.device("cuda", device)
    st = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    Y = inputs.random_suspension(n, L, seed)
    F, T = inputs.random_loads(n, seed + 1)
    gen_s = time.perf_counter() - t0
    pos, Fd, Td = (torch.as_tensor(a, dtype=torch.float32, device=dev) for a in (Y, F, T))
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sm_count * 128 * 2 * (peaks().get("sm_max_mhz") or 2070.0) * 1e6 / 1e12
    hbm = peaks().get("hbm_gbs", 6800.0)
    rows = []
    for M in grids:
        ch = tune.choose(n, L, tol, torques=True, measure=tune.gpu_timer(pos, Fd, Td, L, device, reps=2, warmup=1),
                         top=3, grid=M, max_grid=M)
        p = tune.make_params(ch, L, n)
        U = torch.empty_like(Fd)
        W = torch.empty_like(Fd)
        with fcm.Handle(p, device) as h:
            for _ in range(warmup):
                h.apply(n, pos, Fd, Td, U, W, st.cuda_stream)
            h.set_timing(True)
            h.read_timing()
            ms = 0.0
            for _ in range(steps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                h.apply(n, pos, Fd, Td, U, W, st.cuda_stream)
                e1.record(st)
                e1.synchronize()
                ms += e0.elapsed_time(e1)
            stage = h.read_timing()
            h.set_timing(False)
            assert h.check() == 0
        avg = {k: (v[0] / v[1] if v[1] else None) for k, v in stage.items()}
        MG = ch["M_G"]
        flops = {"spread": FLOPS_POINT[True] * n * MG ** 3, "gather": FLOPS_POINT[True] * n * MG ** 3,
                 "pair": FLOPS_PAIR[True] * n * (n / L ** 3 * 4.0 / 3.0 * math.pi * ch["r_c"] ** 3)}
        dom = max(flops, key=lambda k: avg[k] or 0.0)
        achieved = flops[dom] / (avg[dom] * 1e-3) / 1e12
        p64 = fcm.make_params(L, M, ch["Sigma"], ch["r_c"], MG, n, fcm.FCM_FP64)
        pos64, F64, T64 = (t.double() for t in (pos, Fd, Td))
        with fcm.Handle(p64, device) as h64:
            U64, W64 = fcm.apply_tensors(h64, pos64, F64, T64, stream=st.cuda_stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.zero_()
            e0.record(st)
            h64.apply(n, pos64, F64, T64, U64, W64, st.cuda_stream)
            e1.record(st)
            e1.synchronize()
            ms64 = e0.elapsed_time(e1)
            assert h64.check() == 0
        eu = float(torch.linalg.norm(U.double() - U64) / torch.linalg.norm(U64))
        ew = float(torch.linalg.norm(W.double() - W64) / torch.linalg.norm(W64))
        del U64, W64, pos64, F64, T64
        rows.append({"M": M, "Sigma": ch["Sigma"], "Sigma_over_sigma": ch["Sigma_over_sigma"], "M_G": MG,
                     "r_c": ch["r_c"], "tuned_candidate_ms": ch["measured_s"] * 1e3,
                     "ms_per_apply": ms / steps, "particle_applies_per_s": n * steps / (ms * 1e-3),
                     "stage_ms": {k: round(v, 4) for k, v in avg.items() if v},
                     "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak,
                                  "unit": "TFLOP/s", "frac": achieved / peak},
                     "fft_solve_frac_hbm": (72.0 * M ** 3 / (avg["fft_solve"] * 1e-3) / 1e9 / hbm)
                     if avg.get("fft_solve") else None,
                     "fp32_rel_l2_vs_fp64": {"U": eu, "W": ew},
                     "fp64_plain_particle_applies_per_s": n / (ms64 * 1e-3)})
    return {"workload": f"N={n} uniform spheres (RSA, min separation 2.2a) at phi=10% (L={L:.2f}a), forces+torques, "
                        f"FP32, one fcm_apply per step, inputs resident, L2 flushed between applies; parameters from "
                        f"the autotuner at tolerance {tol:g} per grid",
            "positions_generation_s": gen_s, "rows": rows}


# The paper's performance study (Section 5.2, Table 3): forces only, a/L = 1/400, eps = 1e-4, Sigma/dx = 1.00,
# M_G = 10, and per volume fraction the optimal Sigma/sigma and R_c/sigma it reports; its peak was about 7e6
# particle-applies/s (PTPS) on an RTX 2080 Ti in FP32.
PAPER_SWEEP = [(0.0005, 5.9, 32.6), (0.002, 5.1, 27.9), (0.008, 3.4, 18.6), (0.032, 1.8, 9.8), (0.128, 1.4, 8.1)]
PAPER_PEAK_PTPS = 7.0e6


def paper_sweep(device, reps=5, warmup=3, full=False):
    """PTPS of single-system applies on the paper's performance workloads (FP32, forces only). The
    12.8% row (N = 1.96M; about a minute of host-side RSA placement) runs only with full=True."""
    import numpy as np
    import torch
    from paper_2310_12651_gb300 import fcm, inputs, tune
    L = 400.0
    sg = 1.0 / math.sqrt(math.pi)
    dev = torch.device("cuda", device)
    stream = torch.cuda.current_stream(dev)
    rows = []
    for phi, s_sigma, rc_sigma in PAPER_SWEEP if full else PAPER_SWEEP[:-1]:
        n = int(round(phi * L ** 3 / (4.0 * math.pi / 3.0)))
        Sigma = s_sigma * sg
        M = tune.grid_for(L, Sigma, 1.0)
        Y = inputs.random_suspension(n, L, 2310127000 + n, min_sep=2.2)
        F, _ = inputs.random_loads(n, 2310127001 + n, torques=False)
        pos, Fd = (torch.as_tensor(a, dtype=torch.float32, device=dev) for a in (Y, F))
        U = torch.empty_like(Fd)
        p = fcm.make_params(L, M, Sigma, rc_sigma * sg, 10, n, fcm.FCM_FP32)
        with fcm.Handle(p, device) as h:
            for _ in range(warmup):
                h.apply(n, pos, Fd, None, U, None, stream.cuda_stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                h.apply(n, pos, Fd, None, U, None, stream.cuda_stream)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / reps
            # one more apply with per-stage events (not part of the timed loop above)
            h.set_timing(True)
            h.read_timing()
            h.apply(n, pos, Fd, None, U, None, stream.cuda_stream)
            stages = {k: round(v[0], 4) for k, v in h.read_timing().items() if v[1]}
            h.set_timing(False)
            assert h.check() == 0
        rows.append({"phi": phi, "N": n, "M": M, "Sigma_over_sigma": s_sigma, "R_c_over_sigma": rc_sigma, "M_G": 10,
                     "ms_per_apply": ms, "ptps": n / (ms * 1e-3), "ratio_to_paper_peak": n / (ms * 1e-3) / PAPER_PEAK_PTPS,
                     "stage_ms": stages})
    return {"workload": "paper's Table 3 settings: L = 400a, forces only, eps = 1e-4, Sigma/dx = 1, M_G = 10, "
                        "optimal Sigma and R_c per phi; one fcm_apply per step, inputs resident, no L2 flush",
            "paper_peak_ptps": PAPER_PEAK_PTPS, "paper_hardware": "RTX 2080 Ti, FP32", "rows": rows}


def rods_bench(device, systems=8, steps=5, warmup=3, tol=1e-4):
    """The filament layout (clustered, uneven pair load): 1,024 rods x 64 spheres per system at 5%
    (bond 2.2a, centres uniform, axes isotropic, rods may cross), F = (0,0,-1) + 0.1 N(0,1) per sphere,
    T = 0.1 N(0,1); 128^3 grid with Sigma, M_G and R_c from the autotuner at tol; one batched pass over
    `systems` systems per step; FP32 error against the FP64 plain path on system 0."""
    import numpy as np
    import torch
    from paper_2310_12651_gb300 import fcm, inputs, tune
    n = 65536
    L = inputs.box_edge(n, 0.05)
    ch = tune.choose(n, L, tol, torques=True, grid=128)
    dev = torch.device("cuda", device)
    stream = torch.cuda.current_stream(dev)
    Ys, Fs, Ts = [], [], []
    for b in range(systems):
        Y, _ = inputs.random_rods(1024, 64, L, 2310127100 + b, min_sep=0.0)
        F, T = inputs.random_loads(n, 2310127200 + b, scale=0.1, mean_free=False, bias=(0.0, 0.0, -1.0))
        Ys.append(Y)
        Fs.append(F)
        Ts.append(T)
    pos, F, T = (torch.as_tensor(np.concatenate(a), dtype=torch.float32, device=dev) for a in (Ys, Fs, Ts))
    U = torch.empty_like(F)
    W = torch.empty_like(F)
    offsets = [b * n for b in range(systems + 1)]
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    p = tune.make_params(ch, L, n * systems)
    with fcm.Handle(p, device, max_systems=systems) as h:
        for _ in range(warmup):
            h.batch_apply(offsets, pos, F, T, U, W, stream.cuda_stream)
        ms = 0.0
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.batch_apply(offsets, pos, F, T, U, W, stream.cuda_stream)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
        h.set_timing(True)
        h.read_timing()
        h.batch_apply(offsets, pos, F, T, U, W, stream.cuda_stream)
        stages = {k: round(v[0], 4) for k, v in h.read_timing().items() if v[1]}
        h.set_timing(False)
        assert h.check() == 0
    p64 = tune.make_params(ch, L, n, precision=fcm.FCM_FP64)
    with fcm.Handle(p64, device) as h64:
        U64 = torch.empty((n, 3), dtype=torch.float64, device=dev)
        W64 = torch.empty_like(U64)
        h64.apply(n, pos[:n].double(), F[:n].double(), T[:n].double(), U64, W64, stream.cuda_stream)
        torch.cuda.synchronize()
    eu = float(torch.linalg.norm(U[:n].double() - U64) / torch.linalg.norm(U64))
    ew = float(torch.linalg.norm(W[:n].double() - W64) / torch.linalg.norm(W64))
    return {"workload": f"{systems} systems x 1,024 rods x 64 spheres, phi = 5% (L = {L:.2f}a), rods may cross, "
                        f"F = (0,0,-1) + 0.1 N(0,1), T = 0.1 N(0,1), 128^3, autotuned at tol {tol:g}",
            "Sigma_over_sigma": ch["Sigma_over_sigma"], "M_G": ch["M_G"], "r_c": ch["r_c"],
            "ms_per_step": ms / steps, "particle_applies_per_s": n * systems * steps / (ms * 1e-3),
            "stage_ms_one_pass": stages, "fp32_rel_l2_vs_fp64": {"U": eu, "W": ew}}


def crossover_study(device, a_over_L=(0.012, 0.008, 0.004), tols=(1e-4, 1e-6),
                    phis=(0.005, 0.01, 0.02, 0.04, 0.08, 0.12, 0.16, 0.2), reps=5, warmup=3):
    """Fast FCM against standard FCM (Sigma = sigma, Sigma_D = sigma_D, no pair correction) on the
    paper's crossover study shape (Section 5.3, Fig. 3): forces only, one system per apply, each
    method with the autotuner's parameters for the tolerance (fast FCM: the three cheapest Sigma
    candidates timed on the GPU, the fastest kept). Returns per point the two times and their ratio,
    and per (a/L, tol) the volume fraction where the ratio crosses 1 (linear in log phi)."""
    import numpy as np
    import torch
    from paper_2310_12651_gb300 import fcm, inputs, tune
    dev = torch.device("cuda", device)
    stream = torch.cuda.current_stream(dev)
    rows, crossings = [], []
    systems = {}
    for aL in a_over_L:
        L = 1.0 / aL
        for tol in tols:
            ratios = []
            for phi in phis:
                n = int(round(phi * L ** 3 / (4.0 * math.pi / 3.0)))
                if (aL, phi) not in systems:
                    Y = inputs.random_suspension(n, L, 2310127300 + n, min_sep=2.0, max_rounds=400)
                    F, _ = inputs.random_loads(n, 2310127301 + n, torques=False)
                    systems[(aL, phi)] = tuple(torch.as_tensor(a, dtype=torch.float32, device=dev) for a in (Y, F))
                pos, Fd = systems[(aL, phi)]
                U = torch.empty_like(Fd)

                def timed(choice):
                    with fcm.Handle(tune.make_params(choice, L, n), device) as h:
                        for _ in range(warmup):
                            h.apply(n, pos, Fd, None, U, None, stream.cuda_stream)
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        for _ in range(reps):
                            h.apply(n, pos, Fd, None, U, None, stream.cuda_stream)
                        e1.record(stream)
                        e1.synchronize()
                        return e0.elapsed_time(e1) * 1e-3 / reps

                cands = tune.candidates(n, L, tol, torques=False, max_grid=768)
                std = [c for c in cands if c["Sigma_over_sigma"] == 1.0]
                fast = [c for c in cands if c["Sigma_over_sigma"] != 1.0][:3]
                if not std or not fast:
                    continue
                t_std = timed(std[0])
                best = min(((timed(c), c) for c in fast), key=lambda x: x[0])
                ratio = t_std / best[0]
                ratios.append((phi, ratio))
                rows.append({"a_over_L": aL, "tol": tol, "phi": phi, "N": n,
                             "fast": {"Sigma_over_sigma": best[1]["Sigma_over_sigma"], "M": best[1]["M"],
                                      "M_G": best[1]["M_G"], "r_c": round(best[1]["r_c"], 2), "ms": best[0] * 1e3},
                             "standard": {"M": std[0]["M"], "M_G": std[0]["M_G"], "ms": t_std * 1e3},
                             "speedup_fast_over_standard": ratio})
                print(json.dumps(rows[-1]), flush=True)
            phi_c = None
            for (p0, r0), (p1, r1) in zip(ratios, ratios[1:]):
                if r0 >= 1.0 > r1:
                    f = (1.0 - r0) / (r1 - r0)
                    phi_c = math.exp(math.log(p0) + f * (math.log(p1) - math.log(p0)))
                    break
            crossings.append({"a_over_L": aL, "tol": tol, "phi_c": phi_c,
                              "paper_fit_phi_c": -9.24 * aL + 0.22})
    return {"rows": rows, "crossings": crossings}


def brownian_bench(device, reps=5, tol=1e-6, with_oracle=False):
    """fcm_brownian on one system of the 128^3 workload (N = 65,536, phi = 5%, Sigma = 2a, FP32): the
    grid part (noise -> square-root Stokes projection -> interpolation) and the Lanczos pair part,
    each timed on its own (the call is synchronous; host wall clock around the call). with_oracle: the
    oracle timed beside it on a bounded sample."""
    import numpy as np
    import torch
    from paper_2310_12651_gb300 import fcm, inputs
    w = workload("c2")
    n, M = w["n"], w["M"]
    dev = torch.device("cuda", device)
    Y = inputs.random_suspension(n, w["L"], inputs.BASE_SEED + 1)
    rng = np.random.default_rng(2310127400)
    pos = torch.as_tensor(Y, dtype=torch.float32, device=dev)
    xi = torch.as_tensor(rng.standard_normal(3 * M ** 3), dtype=torch.float32, device=dev)
    z = torch.as_tensor(rng.standard_normal((n, 3)), dtype=torch.float32, device=dev)
    U = torch.empty_like(pos)
    W = torch.empty_like(pos)
    st = torch.cuda.current_stream(dev).cuda_stream
    out = {}
    with fcm.Handle(fcm.make_params(w["L"], M, w["Sigma"], w["r_c"], w["M_G"], n, fcm.FCM_FP32), device) as h:
        for name, (a, b, ww) in {"grid_part": (xi, None, W), "pair_part": (None, z, None)}.items():
            h.brownian(n, pos, 1.0, a, b, U, ww, max_iter=40, tol=tol, stream=st)
            t0 = time.perf_counter()
            for _ in range(reps):
                it = h.brownian(n, pos, 1.0, a, b, U, ww, max_iter=40, tol=tol, stream=st)
            ms = (time.perf_counter() - t0) * 1e3 / reps
            out[name] = {"ms": ms, "lanczos_iterations": it}
    out["workload"] = (f"one system of N={n}, phi=5%, {M}^3, Sigma=2a, M_G={w['M_G']}, r_c={w['r_c']:.2f}a, FP32, "
                       f"Lanczos tol {tol:g}; synchronous call timed on the host")
    out["particle_increments_per_s"] = n / ((out["grid_part"]["ms"] + out["pair_part"]["ms"]) * 1e-3)
    if with_oracle:   # the oracle as it stands (exact matrix square root of the pair part) on a bounded sample
        from oracle import brownian as ob
        ns = 600
        ws = workload("c2", n=ns, h_ref=w["h"])
        Ys = inputs.random_suspension(ns, ws["L"], inputs.BASE_SEED + 5)
        xis = rng.standard_normal((3, ws["M"], ws["M"], ws["M"]))
        zs = rng.standard_normal((ns, 3))
        t0 = time.perf_counter()
        ob.brownian_grid(Ys, xis, ws["L"], ws["M_G"], ws["Sigma"], ws["Sigma"], 1.0)
        t1 = time.perf_counter()
        ob.brownian_pair(Ys, zs, ws["L"], ws["r_c"], ws["Sigma"], 1.0)
        t2 = time.perf_counter()
        out["oracle"] = {"kind": "oracle", "cores": 1, "grid_part_ms": (t1 - t0) * 1e3, "pair_part_ms": (t2 - t1) * 1e3,
                         "particle_increments_per_s": ns / (t2 - t0),
                         "sample": f"N={ns} at phi=5% (L={ws['L']:.1f}a, {ws['M']}^3, h={ws['h']:.3f}a, Sigma=2a, "
                                   f"M_G={ws['M_G']}, r_c={ws['r_c']:.2f}a), FP64 "
                                   f"numpy single thread; pair part by dense eigendecomposition"}
    return out


def rod_suspension_params(L_xy, L_z, n, tol, precision=None):
    """Fast-FCM parameters for the planar rod suspensions of Section 6.1 (box L_xy x L_xy x L_z, rods
    in the plane z = L_z/2, forces only): for grid spacings h on a ladder, Sigma = (Table 1 ratio) h,
    M_G from the window rule and r_c from the neighbour-aware cutoff with the in-plane density
    (n / L_xy^2 particles per area: about 0.75 n / (L_xy^2 r_c) per volume within r_c of a particle);
    r_c must stay below L_z / 2. Keeps the admissible spacing of least modelled cost."""
    from paper_2310_12651_gb300 import fcm, tune
    ratio = tune.resolution_for(tune.GRID_SHARE * tol)
    c = tune.truncation_for(tune.GRID_SHARE * tol)
    best = None
    for h in (3.0, 3.5, 4.0, 4.5, 5.0, 5.5, 6.0):
        Mxy = tune.grid_for(L_xy, h, 1.0)
        Mz = tune.grid_for(L_z, h, 1.0)
        hmax = max(L_xy / Mxy, L_z / Mz)
        Sigma = ratio * hmax
        MG = tune.support_points(Sigma, min(L_xy / Mxy, L_z / Mz), c)
        if MG > 24 or MG > Mz:
            continue
        rc = tune.cutoff(Sigma, 0.5 * tol, torques=False)
        for _ in range(3):
            rc = tune.pair_cutoff(Sigma, tol, 0.75 * n / (L_xy ** 2 * rc), torques=False)
        if rc > 0.5 * L_z:
            continue
        cand = n / L_xy ** 2 * math.pi * (1.5 * rc) ** 2
        cost = (tune.COST["point"] * n * MG ** 3 + tune.COST["candidate"] * n * cand
                + tune.COST["grid"] * Mxy * Mxy * Mz)
        if best is None or cost < best["cost_model_s"]:
            best = dict(M=(Mxy, Mxy, Mz), Sigma=Sigma, M_G=MG, r_c=rc, h=hmax, cost_model_s=cost)
    if best is None:
        raise ValueError("no admissible parameters for the rod suspension")
    return best


def rigid_oracle_sample(tol, n_rods=16):
    """The oracle's rigid-body Broyden (fast-FCM oracle product, FP64 numpy) on n_rods rods at the
    10.5% area fraction of the rod suspension (box 960a sqrt(n_rods / 2304) x same x 60a)."""
    from oracle import rigid as orr
    from paper_2310_12651_gb300 import inputs
    L_xy, L_z = 960.0 * math.sqrt(n_rods / 2304.0), 60.0
    Y, off, X = inputs.doublet_rods(n_rods, L_xy, L_z, 2310127510)
    ft = inputs.rod_loads(n_rods, 2310127511, gravity=(1.0, 0.0, 0.0))
    pr = rod_suspension_params(L_xy, L_z, Y.shape[0], tol)
    t0 = time.perf_counter()
    _, _, it, _ = orr.fast_fcm_rigid_broyden(Y, off, X, ft, (L_xy, L_xy, L_z), pr["M"], pr["M_G"], pr["Sigma"],
                                             pr["r_c"], tol, 256)
    secs = time.perf_counter() - t0
    return {"kind": "oracle", "cores": 1, "iterations": it, "solve_s": secs,
            "particle_iterations_per_s": Y.shape[0] * max(it, 1) / secs,
            "sample": f"{n_rods} rods x 22 particles, box {L_xy:.0f}a x {L_xy:.0f}a x {L_z:.0f}a, grid "
                      f"{pr['M'][0]}x{pr['M'][1]}x{pr['M'][2]}, Broyden tol {tol:g}, FP64 numpy single thread"}


def rigid_roofline(stages, n, M_G, device):
    """FP32 ALU roofline of the spread inside the rigid solve: forces only, 8 algorithmic flops per
    window point, against 152 SMs x 128 lanes x 2 x the maximum SM clock."""
    import torch
    ms, cnt = stages.get("spread", (0.0, 0))
    if not cnt:
        return None
    sm_count = torch.cuda.get_device_properties(device).multi_processor_count
    sm_max = peaks().get("sm_max_mhz") or 2070.0
    peak = sm_count * 128 * 2 * sm_max * 1e6 / 1e12
    achieved = FLOPS_POINT[False] * n * M_G ** 3 / (ms / cnt * 1e-3) / 1e12
    return {"bound": "alu", "kernel": "spread", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "spread_ms_per_launch": ms / cnt,
            "stage_share": {k: v[0] / sum(x[0] for kk, x in stages.items() if kk != "apply")
                            for k, v in stages.items() if k != "apply"}}


def rigid_bench(device, n_rods=7744, tol=1e-4, reps=3, with_oracle=False):
    """fcm_rigid_solve on the rod suspension of Section 6.1: n_rods rods of 22 particles (alternating
    doublets, length 14.14a) on a square lattice, randomly oriented in the plane z = 30a of an
    L x L x 60a box at the paper's 10.5% area fraction (L = 960a for 2,304 rods), each particle
    under gravity F_0 x (no barrier forces at the lattice start), Broyden tolerance 1e-4 and fast
    FCM at 1e-4 as in the paper, FP32. Times whole solves (synchronous; CUDA events on the stream)
    and the fast-FCM product alone, checks the equations on the host (rigid particle velocities
    under fcm_apply, rod force sums), and compares the rod velocities with an FP64 solve; the same
    solve started from each rod's own FCM mobility (the body preconditioner) beside it. with_oracle:
    the oracle's Broyden (fast-FCM oracle product) timed beside it on 16 rods at the same area
    fraction."""
    import numpy as np
    import torch
    from paper_2310_12651_gb300 import fcm, inputs
    L_xy, L_z = 960.0 * math.sqrt(n_rods / 2304.0), 60.0
    Y, off, X = inputs.doublet_rods(n_rods, L_xy, L_z, 2310127500)
    ft = inputs.rod_loads(n_rods, 2310127501, gravity=(1.0, 0.0, 0.0))
    n = Y.shape[0]
    pr = rod_suspension_params(L_xy, L_z, n, tol)
    dev = torch.device("cuda", device)
    st = torch.cuda.current_stream(dev)

    def solve(prec, t, precond=0):
        dt = torch.float32 if prec == fcm.FCM_FP32 else torch.float64
        tens = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
        pos, Xd, ftd = tens(Y), tens(X), tens(ft)
        offd = torch.as_tensor(off, device=dev)
        F = torch.zeros((n, 3), dtype=dt, device=dev)
        UG = torch.zeros((n_rods, 6), dtype=dt, device=dev)
        p = fcm.make_params((L_xy, L_xy, L_z), pr["M"], pr["Sigma"], pr["r_c"], pr["M_G"], n, prec)
        out = {}
        with fcm.Handle(p, device) as h:
            _, it, res = h.rigid_solve(n, pos, n_rods, offd, Xd, ftd, F, UG, max_iter=256, tol=t,
                                       stream=st.cuda_stream, precond=precond)
            if prec == fcm.FCM_FP32:
                times = []
                for _ in range(reps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(st)
                    _, it, res = h.rigid_solve(n, pos, n_rods, offd, Xd, ftd, F, UG, max_iter=256, tol=t,
                                               stream=st.cuda_stream, precond=precond)
                    e1.record(st)
                    e1.synchronize()
                    times.append(e0.elapsed_time(e1))
                V = torch.empty_like(F)
                for _ in range(3):
                    h.apply(n, pos, F, None, V, None, st.cuda_stream)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                for _ in range(reps * 4):
                    h.apply(n, pos, F, None, V, None, st.cuda_stream)
                e1.record(st)
                e1.synchronize()
                out["solve_ms"] = statistics.median(times)
                # per-stage CUDA-event times over one more solve: the spread's roofline inside the solve
                h.set_timing(True)
                h.read_timing()
                h.rigid_solve(n, pos, n_rods, offd, Xd, ftd, F, UG, max_iter=256, tol=t, stream=st.cuda_stream,
                              precond=precond)
                out["stages"] = {k: v for k, v in h.read_timing().items() if v[1]}
                h.set_timing(False)
                out["apply_ms"] = e0.elapsed_time(e1) / (reps * 4)
                out["V"] = V.double().cpu().numpy()
            out.update(iterations=it, residual=res, F=F.double().cpu().numpy(), UG=UG.double().cpu().numpy())
        return out

    r32 = solve(fcm.FCM_FP32, tol)
    rb = solve(fcm.FCM_FP32, tol, precond=fcm.RIGID_PRECOND_BODY)
    r64 = solve(fcm.FCM_FP64, 1e-8)
    # the equations on the host, body by body (22 particles each)
    Lv = np.array([L_xy, L_xy, L_z])
    Yr = Y.astype(np.float32).astype(np.float64).reshape(n_rods, 22, 3)
    r = Yr - X.astype(np.float32).astype(np.float64)[:, None, :]
    r -= Lv * np.round(r / Lv)
    UG, F, V = r32["UG"], r32["F"].reshape(n_rods, 22, 3), r32["V"].reshape(n_rods, 22, 3)
    rigid = UG[:, None, :3] + np.cross(UG[:, None, 3:], r)
    sums = np.concatenate([F.sum(axis=1), np.cross(r, F).sum(axis=1)], axis=1)
    it = r32["iterations"]
    return {"workload": (f"{n_rods} rods x 22 particles (alternating doublets), square lattice, random in-plane "
                         f"orientation, box {L_xy:.0f}a x {L_xy:.0f}a x {L_z:.0f}a (10.5% area fraction), "
                         f"gravity F_0 x per particle, grid {pr['M'][0]}x{pr['M'][1]}x{pr['M'][2]}, "
                         f"Sigma={pr['Sigma']:.3f}a, M_G={pr['M_G']}, r_c={pr['r_c']:.2f}a, FP32, "
                         f"Broyden tol {tol:g}"),
            "particles": n, "iterations": it, "relative_residual": r32["residual"],
            "solve_ms": r32["solve_ms"], "ms_per_iteration": r32["solve_ms"] / max(it, 1),
            "apply_ms": r32["apply_ms"],
            "fcm_share_of_iteration": r32["apply_ms"] * it / r32["solve_ms"] if it else None,
            "rod_solves_per_s": 1e3 / r32["solve_ms"],
            "particle_iterations_per_s": n * max(it, 1) / (r32["solve_ms"] * 1e-3),
            "roofline": rigid_roofline(r32["stages"], n, pr["M_G"], device),
            "rigid_motion_rel": float(np.linalg.norm(V - rigid) / np.linalg.norm(V)),
            "force_torque_sum_rel": float(np.linalg.norm(sums - ft) / np.linalg.norm(ft)),
            "fp64_iterations_at_1e-8": r64["iterations"],
            "oracle": rigid_oracle_sample(tol) if with_oracle else None,
            "rod_velocity_rel_l2_vs_fp64": float(np.linalg.norm(UG - r64["UG"]) / np.linalg.norm(r64["UG"])),
            "body_preconditioner": {
                "iterations": rb["iterations"], "solve_ms": rb["solve_ms"], "relative_residual": rb["residual"],
                "speedup_vs_diagonal": r32["solve_ms"] / rb["solve_ms"],
                "rod_velocity_rel_l2_vs_fp64": float(np.linalg.norm(rb["UG"] - r64["UG"]) / np.linalg.norm(r64["UG"])),
                "note": "Broyden from each rod's own free-space FCM mobility (not the paper's diagonal start)"}}


SERVE_CLASSES = 8          # box-size ladder of the serving mix (log-spaced L, one grid class each)
SERVE_POOL = 32            # distinct systems drawn for the mix (half spheres, half 64-sphere rods)


def serve_pool(seed=2310126900, pool=SERVE_POOL, tol=1e-4):
    """Systems shaped like the serving mix: N log-uniform in [2e3, 2e5], phi uniform in [0.01, 0.2],
    half random suspensions (min separation 2a) and half rods of 64 spheres (bond 2.2a, rods may
    cross). Each box is rounded up to the next of SERVE_CLASSES log-spaced edges between the mix's
    extremes (34.7a and 437.6a), so requests of one edge share a grid class, whose parameters the
    autotuner picks for the class's median N at tolerance tol (grids 32^3 to 256^3)."""
    import numpy as np
    from paper_2310_12651_gb300 import fcm, inputs, tune
    rng = np.random.default_rng(seed)
    lo, hi = inputs.box_edge(2000, 0.2), inputs.box_edge(200000, 0.01)
    edges = np.exp(np.linspace(np.log(lo), np.log(hi), SERVE_CLASSES))
    draws = []
    for k in range(pool):
        n = int(np.exp(rng.uniform(np.log(2000), np.log(200000))))
        phi = rng.uniform(0.01, 0.2)
        rods = k % 2 == 1
        if rods:
            n = max(64, 64 * round(n / 64))
        L = inputs.box_edge(n, phi)
        c = int(np.searchsorted(edges, L * (1 - 1e-12)))
        draws.append((n, rods, min(c, SERVE_CLASSES - 1)))
    classes = {}
    for c in sorted({d[2] for d in draws}):
        ns = sorted(d[0] for d in draws if d[2] == c)
        ch = tune.choose(ns[len(ns) // 2], float(edges[c]), tol, torques=True, max_grid=256, min_grid=32)
        classes[c] = (float(edges[c]), ch)
    systems = []
    for k, (n, rods, c) in enumerate(draws):
        L, ch = classes[c]
        if rods:
            Y, _ = inputs.random_rods(n // 64, 64, L, seed + 10 * k, min_sep=0.0)
        else:
            Y = inputs.random_suspension(n, L, seed + 10 * k, min_sep=2.0, max_rounds=400)
        F, T = inputs.random_loads(n, seed + 10 * k + 1)
        arrays = tuple(np.ascontiguousarray(a, dtype=np.float32) for a in (Y, F, T))
        systems.append(dict(n=n, L=L, cls=c, rods=rods, params=tune.make_params(ch, L, n), arrays=arrays))
    return systems, classes


def serve_bench(device, requests=1024, loads=(0.5, 0.9, 1.0, 2.0), seed=2310126950):
    """The serving engine on the mix: capacity with every request queued at once, then Poisson
    arrivals at fractions of that capacity; latency = submit to completion (host clocks)."""
    import threading
    import numpy as np
    from paper_2310_12651_gb300 import fcm
    t_gen = time.time()
    pool, classes = serve_pool()
    t_gen = time.time() - t_gen
    rng = np.random.default_rng(seed)
    order = rng.integers(0, len(pool), size=requests)
    out = {"pool_systems": len(pool), "grid_classes": len(classes), "requests_per_phase": requests,
           "classes": [{"L": round(L, 2), "M": ch["M"], "Sigma_over_sigma": ch["Sigma_over_sigma"], "M_G": ch["M_G"],
                        "r_c": round(ch["r_c"], 2)} for L, ch in classes.values()],
           "pool_generation_s": round(t_gen, 1), "tolerance": 1e-4}
    with fcm.Server(device=device, hbm_budget=48 << 30, max_batch=64) as srv:
        warm = [srv.submit(s["params"], *s["arrays"]) for s in pool]
        for t in warm:
            assert srv.wait(t, 120.0) and t.status == fcm.FCM_OK, t.status
        # capacity: all requests queued at once
        srv.reset_latency()
        b0 = srv.stats()
        t0 = time.perf_counter()
        tickets = [srv.submit(pool[i]["params"], *pool[i]["arrays"]) for i in order]
        for t in tickets:
            assert srv.wait(t, 300.0) and t.status == fcm.FCM_OK
        wall = time.perf_counter() - t0
        st = srv.stats()
        particles = int(sum(pool[i]["n"] for i in order))
        cap_rps = requests / wall
        out["capacity"] = {"requests_per_s": cap_rps, "particle_applies_per_s": particles / wall,
                           "p50_ms": st["latency_p50_us"] / 1e3, "p99_ms": st["latency_p99_us"] / 1e3,
                           "mean_batch": (st["batched_requests"] - b0["batched_requests"]) /
                                         max(1, st["batches"] - b0["batches"])}
        out["open_loop"] = []
        for load in loads:
            rate = load * cap_rps
            gaps = rng.exponential(1.0 / rate, size=requests)
            srv.reset_latency()
            b0 = srv.stats()
            tickets = []
            t0 = time.perf_counter()
            due = t0
            for k, i in enumerate(order):
                due += gaps[k]
                delay = due - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                tickets.append(srv.submit(pool[i]["params"], *pool[i]["arrays"]))
            for t in tickets:
                assert srv.wait(t, 300.0) and t.status == fcm.FCM_OK
            wall = time.perf_counter() - t0
            st = srv.stats()
            out["open_loop"].append({"load": load, "offered_requests_per_s": rate,
                                     "particle_applies_per_s": particles / wall,
                                     "p50_ms": st["latency_p50_us"] / 1e3, "p99_ms": st["latency_p99_us"] / 1e3,
                                     "max_ms": st["latency_max_us"] / 1e3,
                                     "mean_batch": (st["batched_requests"] - b0["batched_requests"]) /
                                                   max(1, st["batches"] - b0["batches"])})
        st = srv.stats()
        out["graph_passes"] = st["graph_passes"]
        out["passes"] = st["batches"]
        out["handles_created"] = st["handles_created"]
        out["handles_evicted"] = st["handles_evicted"]
        out["hbm_bytes"] = st["hbm_bytes"]
        out["hbm_budget"] = st["hbm_budget"]
    return out


def reference_arm(args, world, rank):
    if rank != 0:
        return 0
    n = 4096
    w = oracle_workload(args.workload, n=n, h_ref=oracle_workload(args.workload)["h"])
    for k in range(args.warmup):
        run_cpu_oracle(w, 2310126700 + k)
    t = 0.0
    for k in range(args.steps):
        t += run_cpu_oracle(w, 2310126800 + k)
    value = n * args.steps / t
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"oracle (FP64 numpy) on a bounded sample: {n} spheres at phi={w['phi']:.0%}, "
                                   f"{w['M']}^3 (h={w['h']:.3f}a), Sigma={w['Sigma']}a, M_G={w['M_G']}, "
                                   f"r_c={w['r_c']:.2f}a, forces+torques",
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} oracle applies of {n} spheres"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--batch", type=int, default=0, help="systems per step (0: the workload's default)")
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-oracle-errors", action="store_true",
                    help="skip the per-configuration error against the FP64 oracle (also skipped with --no-cpu-baseline)")
    ap.add_argument("--spread-kernel", type=int, default=0, help="0 choose, 1 row-stationary, 2 shared atomics, 3 tensor cores (tcgen05)")
    ap.add_argument("--tile", default="0,0,0", help="spread/gather tile x,y,z in grid points (0,0,0: the library's choice)")
    ap.add_argument("--study", default=None, choices=["crossover", "rigid", "brownian", "large"],
                    help="run one measurement instead of the bench line: crossover = fast vs standard FCM against "
                         "phi; rigid = the rigid-rod solve on the 7,744-rod suspension; brownian = fcm_brownian")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving-mix measurement")
    ap.add_argument("--no-sweep", action="store_true", help="skip the paper-settings PTPS sweep")
    ap.add_argument("--no-rods", action="store_true", help="skip the filament-layout measurement")
    ap.add_argument("--no-brownian", action="store_true", help="skip the Brownian-increment measurement")
    ap.add_argument("--no-rigid", action="store_true", help="skip the rigid-rod mobility solve measurement")
    ap.add_argument("--no-large", action="store_true", help="skip the N = 1,048,576 sweep over 192^3-320^3 grids")
    ap.add_argument("--sweep-full", action="store_true", help="include the 12.8%% (N = 1.96M) sweep row")
    ap.add_argument("--large-grids", default="192,256,320", help="grids of the N = 1,048,576 sweep (comma list)")
    ap.add_argument("--serve-requests", type=int, default=1024)
    ap.add_argument("--mode", default="batched", choices=["batched", "single"],
                    help="batched: one fcm_batch_apply over the stacked systems; single: one fcm_apply per system")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return reference_arm(args, world, rank)

    import numpy as np
    import torch

    from paper_2310_12651_gb300 import build as libbuild
    if rank == 0:
        libbuild.build()
    barrier(world)
    from paper_2310_12651_gb300 import fcm, inputs

    torch.cuda.set_device(local)
    if args.study is not None:
        if rank == 0:
            if args.study == "crossover":
                res = crossover_study(local)
            elif args.study == "large":
                res = large_sweep(local, grids=tuple(int(x) for x in args.large_grids.split(",")))
            else:
                run = {"rigid": rigid_bench, "brownian": brownian_bench}[args.study]
                res = run(local, with_oracle=not args.no_cpu_baseline)
            print(json.dumps({"study": args.study, **res}), flush=True)
        return 0
    oracle_jobs = None
    if rank == 0 and world == 1 and args.workload == "c2" and not (args.no_oracle_errors or args.no_cpu_baseline):
        oracle_jobs = OracleErrors()   # spawned workers; they run while the GPU is measured
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    w = workload(args.workload)
    B = args.batch or WORKLOADS[args.workload]["batch"]
    n = w["n"]
    batched = args.mode == "batched"
    tile = tuple(int(v) for v in args.tile.split(","))
    params = fcm.make_params(w["L"], w["M"], w["Sigma"], w["r_c"], w["M_G"], n * B if batched else n, fcm.FCM_FP32,
                             spread_kernel=args.spread_kernel, tile=tile)
    h = fcm.Handle(params, local, max_systems=B if batched else 1)
    Ys, Fs, Ts = [], [], []
    for b in range(B):
        seed = inputs.BASE_SEED + 1 + 100 * b + 10000 * rank
        Ys.append(inputs.random_suspension(n, w["L"], seed))
        F, T = inputs.random_loads(n, seed + 1)
        Fs.append(F)
        Ts.append(T)
    # the B systems stacked along the particle axis: system b owns rows b n .. (b + 1) n - 1
    pos_all, F_all, T_all = (torch.as_tensor(np.concatenate(a), dtype=torch.float32, device=dev) for a in (Ys, Fs, Ts))
    offsets = [b * n for b in range(B + 1)]
    U = torch.empty((n * B, 3), dtype=torch.float32, device=dev)
    W = torch.empty_like(U)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step(pos, F, T):
        if batched:
            h.batch_apply(offsets, pos, F, T, U, W, sptr)
        else:
            for b in range(B):
                r = slice(b * n, (b + 1) * n)
                h.apply(n, pos[r], F[r], T[r], U[r], W[r], sptr)

    for k in range(args.warmup):
        step(pos_all, F_all, T_all)
    torch.cuda.synchronize()
    assert h.check() == 0

    # ---- timed region (device time, inputs resident)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    barrier(world)
    torch.cuda.synchronize()
    h.set_timing(True)
    h.read_timing()
    launches0 = h.launch_count()
    for k in range(args.steps):
        flush.zero_()
        starts[k].record(stream)
        step(pos_all, F_all, T_all)
        ends[k].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    launches = h.launch_count() - launches0
    stage = h.read_timing()
    h.set_timing(False)
    step_ms = [starts[i].elapsed_time(ends[i]) for i in range(args.steps)]
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    value = world * n * B * args.steps / (total_ms * 1e-3)
    ms_per_step = total_ms / args.steps

    # ---- the FFT chain alone: grid-part passes (no pair kernel beside it on the side stream)
    fft_alone = gather_alone = pair_alone = None
    if batched:
        h.set_timing(True)
        h.read_timing()
        for k in range(3):
            flush.zero_()
            h.batch_apply(offsets, pos_all, F_all, T_all, U, W, sptr, stages=fcm.STAGE_GRID)
        st_alone = h.read_timing()
        ms_fft, cnt_fft = st_alone["fft_solve"]
        if cnt_fft:
            fft_alone = ms_fft / cnt_fft
        ms_g, cnt_g = st_alone["gather"]
        gather_alone = ms_g / cnt_g if cnt_g else None
        # the pair kernel alone: pair-only passes (inside the full pass it shares the SMs with the FFT chain
        # and the gather)
        for k in range(3):
            flush.zero_()
            h.batch_apply(offsets, pos_all, F_all, T_all, U, W, sptr, stages=fcm.STAGE_PAIR)
        ms_p, cnt_p = h.read_timing()["pair"]
        h.set_timing(False)
        pair_alone = ms_p / cnt_p if cnt_p else None

    # ---- end to end through host buffers: pinned host -> device inputs, the pass, device -> host outputs
    hpos, hF, hT = (t.cpu().pin_memory() for t in (pos_all, F_all, T_all))
    Uh = torch.empty((n * B, 3), dtype=torch.float32).pin_memory()
    Wh = torch.empty_like(Uh).pin_memory()
    dpos, dF, dT = (torch.empty((n * B, 3), dtype=torch.float32, device=dev) for _ in range(3))
    e2e_steps = max(1, min(args.steps, 10))
    e2e_ms = 0.0
    for rep in range(args.warmup + e2e_steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dpos.copy_(hpos, non_blocking=True)
        dF.copy_(hF, non_blocking=True)
        dT.copy_(hT, non_blocking=True)
        step(dpos, dF, dT)
        Uh.copy_(U, non_blocking=True)
        Wh.copy_(W, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        if rep >= args.warmup:
            e2e_ms += e0.elapsed_time(e1)
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    e2e_value = world * n * B * e2e_steps / (e2e_ms * 1e-3)

    # ---- FP64 plain path on the same workload, and the FP32 error against it
    fp64 = None
    if not args.no_fp64:
        h64 = fcm.Handle(fcm.make_params(w["L"], w["M"], w["Sigma"], w["r_c"], w["M_G"], n, fcm.FCM_FP64), local)
        pos, F, T = (t[:n].double() for t in (pos_all, F_all, T_all))
        U64 = torch.empty((n, 3), dtype=torch.float64, device=dev)
        W64 = torch.empty_like(U64)
        h64.apply(n, pos, F, T, U64, W64, sptr)
        torch.cuda.synchronize()
        reps = 3
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        t64 = 0.0
        for _ in range(reps):
            flush.zero_()
            e0.record(stream)
            h64.apply(n, pos, F, T, U64, W64, sptr)
            e1.record(stream)
            e1.synchronize()
            t64 += e0.elapsed_time(e1)
        step(pos_all, F_all, T_all)
        torch.cuda.synchronize()
        eu = float(torch.linalg.norm(U[:n].double() - U64) / torch.linalg.norm(U64))
        ew = float(torch.linalg.norm(W[:n].double() - W64) / torch.linalg.norm(W64))
        fp64 = {"value": n * reps / (t64 * 1e-3), "unit": UNIT, "ms_per_apply": t64 / reps,
                "fp32_rel_l2_vs_fp64": {"U": eu, "W": ew}}
        h64.close()

    # ---- roofline of the dominant kernel
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    pk = peaks()
    sm_max = (clocks or {}).get("sm_max_mhz") or pk.get("sm_max_mhz") or 2070.0
    alu_peak = sm_count * 128 * 2 * sm_max * 1e6 / 1e12          # FP32 TFLOP/s, FMA = 2 flops
    avg = {name: (ms / cnt if cnt else None) for name, (ms, cnt) in stage.items()}
    per_launch = B if batched else 1        # systems one kernel launch processes
    pts = per_launch * n * w["M_G"] ** 3
    flops = {"spread": FLOPS_POINT[True] * pts, "gather": FLOPS_POINT[True] * pts}
    n_nb = n / w["L"] ** 3 * 4.0 / 3.0 * math.pi * w["r_c"] ** 3
    flops["pair"] = FLOPS_PAIR[True] * per_launch * n * n_nb
    dominant = max(("spread", "gather", "pair"), key=lambda s: avg[s] or 0.0)
    achieved = flops[dominant] / (avg[dominant] * 1e-3) / 1e12
    traffic = TRAFFIC_BYTES.get(args.workload, {}).get(dominant)
    roofline = {"bound": "alu", "kernel": dominant, "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved / alu_peak, "traffic": traffic * per_launch if traffic else None,
                "peak_source": f"{sm_count} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz",
                "flops_per_launch": flops[dominant]}
    M3 = per_launch * w["M"] ** 3
    fft_bytes = 72.0 * M3
    hbm = pk.get("hbm_gbs", 6800.0)
    stages_out = {name: {"ms_avg": avg[name], "launches": int(stage[name][1])} for name in stage}
    if avg["fft_solve"]:
        # inside the full pass the chain shares the GPU with the pair kernel on the side stream
        stages_out["fft_solve"]["GBps_beside_pair"] = fft_bytes / (avg["fft_solve"] * 1e-3) / 1e9
    if fft_alone:
        stages_out["fft_solve"]["ms_alone"] = fft_alone
        stages_out["fft_solve"]["GBps"] = fft_bytes / (fft_alone * 1e-3) / 1e9
        stages_out["fft_solve"]["frac_hbm"] = stages_out["fft_solve"]["GBps"] / hbm
        stages_out["fft_solve"]["bytes"] = "72 B per grid point: 6 transforms x 8 B + 24 B for the projection kernel"
    if gather_alone:
        stages_out["gather"]["ms_alone"] = gather_alone
    if pair_alone:
        stages_out["pair"]["ms_alone"] = pair_alone
        stages_out["pair"]["TFLOPs_alone"] = flops["pair"] / (pair_alone * 1e-3) / 1e12
        stages_out["pair"]["frac_alu_alone"] = stages_out["pair"]["TFLOPs_alone"] / alu_peak
    if avg["pair"]:
        stages_out["pair"]["TFLOPs"] = flops["pair"] / (avg["pair"] * 1e-3) / 1e12
        stages_out["pair"]["frac_alu"] = stages_out["pair"]["TFLOPs"] / alu_peak
    for s_ in ("spread", "gather"):
        if avg[s_]:
            stages_out[s_]["TFLOPs"] = flops[s_] / (avg[s_] * 1e-3) / 1e12
            stages_out[s_]["frac_alu"] = stages_out[s_]["TFLOPs"] / alu_peak
            byts = 12.0 * M3 + 48.0 * n * per_launch
            stages_out[s_]["GBps"] = byts / (avg[s_] * 1e-3) / 1e9
            stages_out[s_]["frac_hbm"] = stages_out[s_]["GBps"] / hbm

    serve = None
    if not args.no_serve:
        serve = serve_bench(local, requests=args.serve_requests)
    sweep = None if args.no_sweep else paper_sweep(local, full=args.sweep_full)
    rods = None if args.no_rods else rods_bench(local)
    oracle_here = rank == 0 and world == 1 and not args.no_cpu_baseline
    brown = None if args.no_brownian else brownian_bench(local, with_oracle=oracle_here)
    rigid = None if args.no_rigid else rigid_bench(local, with_oracle=oracle_here)
    large_grids = tuple(int(x) for x in args.large_grids.split(","))
    large = None if (args.no_large or args.workload != "c2") else large_sweep(local, grids=large_grids)

    err = error_vs_oracle(local, oracle_jobs) if oracle_jobs is not None else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload)

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": describe(w, B), "particles_per_step_per_gpu": n * B,
                      "mode": ("one batched pass (fcm_batch_apply) over the stacked systems" if batched
                               else "one fcm_apply per system"),
                      "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                      "l2": "flushed (256 MB write) before every step"},
           "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": B * 3 * n * 3 * 4,
                   "d2h_bytes_per_step": B * 2 * n * 3 * 4},
           "gpu_launches": int(launches), "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks,
           "fp64_plain": fp64, "error_vs_oracle": err, "serve": serve, "paper_sweep": sweep, "rods": rods, "brownian": brown,
           "rigid_rods": rigid, "large_sweep": large,
           "speedup_vs_fp64_plain": (value / world / fp64["value"]) if fp64 else None,
           "stages": stages_out, "step_ms_median": statistics.median(step_ms),
           "workspace_bytes": h.workspace_bytes()}
    if rank == 0:
        print(json.dumps(out), flush=True)
    h.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
