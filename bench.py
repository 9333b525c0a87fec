#!/usr/bin/env python
"""Throughput of the fast-FCM mobility product (U, W) = M (F, T) on GB300.

One step = one pass of the whole hot path (binning, spread, FFT Stokes solve,
gather, pair correction) over one batch of ``--batch`` independent periodic
systems, each a seeded uniform suspension of N = 65,536 spheres at 5% volume
fraction (L = 176.41a) on a 128^3 grid with Sigma = 2a, forces and torques,
FP32. Every system's inputs stay resident in HBM; L2 is flushed (256 MB
write) before every apply and each apply is timed with CUDA events on the
stream it runs on. ``value`` = particles processed / summed apply time.

``e2e`` repeats the measurement through the same C-ABI call with host
buffers: pinned host -> device copies of pos, F, T and device -> host copies of
U, W inside each timed apply.

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
# dram__bytes_read.sum + dram__bytes_write.sum per launch, one ncu --set full capture of the c2 workload with the
# current kernels (cold caches); None once a kernel changes after the capture.
TRAFFIC_BYTES = {"c2": {"gather": 27.826176e6, "spread": 28.370944e6, "pair": 3.251968e6}}


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


def cpu_baseline(name, target_s=15.0):
    """The oracle timed on a bounded sample of the workload (same density, spacing, Sigma, M_G, r_c)."""
    full = workload(name)
    n = 16384
    w = workload(name, n=n, h_ref=full["h"])
    secs = run_cpu_oracle(w, 2310126590)
    reps = 1
    while secs * (reps + 1) / reps < target_s and reps < 4:
        secs += run_cpu_oracle(w, 2310126590 + reps)
        reps += 1
    return {"value": n * reps / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{reps} oracle apply(s) of {n} spheres at phi={w['phi']:.0%} (L={w['L']:.1f}a, {w['M']}^3, "
                      f"h={w['h']:.3f}a, Sigma={w['Sigma']}a, M_G={w['M_G']}, r_c={w['r_c']:.2f}a), forces+torques, "
                      f"FP64 numpy single thread, {secs:.1f} s",
            "host_cores": len(os.sched_getaffinity(0))}


def reference_arm(args, world, rank):
    if rank != 0:
        return 0
    full = workload(args.workload)
    n = 4096
    w = workload(args.workload, n=n, h_ref=full["h"])
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
    ap.add_argument("--spread-kernel", type=int, default=0, help="0 choose, 1 row-stationary, 2 shared atomics")
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
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    w = workload(args.workload)
    B = args.batch or WORKLOADS[args.workload]["batch"]
    n = w["n"]
    params = fcm.make_params(w["L"], w["M"], w["Sigma"], w["r_c"], w["M_G"], n, fcm.FCM_FP32,
                             spread_kernel=args.spread_kernel)
    h = fcm.Handle(params, local)
    systems = []
    for b in range(B):
        seed = inputs.BASE_SEED + 1 + 100 * b + 10000 * rank
        Y = inputs.random_suspension(n, w["L"], seed)
        F, T = inputs.random_loads(n, seed + 1)
        systems.append(tuple(torch.as_tensor(a, dtype=torch.float32, device=dev) for a in (Y, F, T)))
    U = torch.empty((n, 3), dtype=torch.float32, device=dev)
    W = torch.empty_like(U)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def apply(b):
        pos, F, T = systems[b]
        h.apply(n, pos, F, T, U, W, sptr)

    for k in range(args.warmup):
        for b in range(B):
            apply(b)
    torch.cuda.synchronize()
    assert h.check() == 0

    # ---- timed region (device time, inputs resident)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(B * args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(B * args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    barrier(world)
    torch.cuda.synchronize()
    h.set_timing(True)
    h.read_timing()
    launches0 = h.launch_count()
    k = 0
    for s in range(args.steps):
        for b in range(B):
            flush.zero_()
            starts[k].record(stream)
            apply(b)
            ends[k].record(stream)
            k += 1
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    launches = h.launch_count() - launches0
    stage = h.read_timing()
    h.set_timing(False)
    apply_ms = [starts[i].elapsed_time(ends[i]) for i in range(k)]
    total_ms = max_over_ranks(sum(apply_ms), world, dev)
    value = world * n * B * args.steps / (total_ms * 1e-3)
    ms_per_step = total_ms / args.steps

    # ---- end to end through host buffers
    host = []
    for b in range(min(B, 4)):
        host.append(tuple(t.cpu().pin_memory() for t in systems[b]))
    Uh = torch.empty((n, 3), dtype=torch.float32).pin_memory()
    Wh = torch.empty_like(Uh).pin_memory()
    dpos, dF, dT = (torch.empty((n, 3), dtype=torch.float32, device=dev) for _ in range(3))
    e2e_steps = max(1, min(args.steps, 10))
    e2e_ms = 0.0
    for rep in range(args.warmup + e2e_steps):
        for b in range(B):
            hp, hF, hT = host[b % len(host)]
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            dpos.copy_(hp, non_blocking=True)
            dF.copy_(hF, non_blocking=True)
            dT.copy_(hT, non_blocking=True)
            h.apply(n, dpos, dF, dT, U, W, sptr)
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
        pos, F, T = (t.double() for t in systems[0])
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
        apply(0)
        torch.cuda.synchronize()
        eu = float(torch.linalg.norm(U.double() - U64) / torch.linalg.norm(U64))
        ew = float(torch.linalg.norm(W.double() - W64) / torch.linalg.norm(W64))
        fp64 = {"value": n * reps / (t64 * 1e-3), "unit": UNIT, "ms_per_apply": t64 / reps,
                "fp32_rel_l2_vs_fp64": {"U": eu, "W": ew}}
        h64.close()

    # ---- roofline of the dominant kernel
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    pk = peaks()
    sm_max = (clocks or {}).get("sm_max_mhz") or pk.get("sm_max_mhz") or 2070.0
    alu_peak = sm_count * 128 * 2 * sm_max * 1e6 / 1e12          # FP32 TFLOP/s, FMA = 2 flops
    napply = B * args.steps
    avg = {name: (ms / cnt if cnt else None) for name, (ms, cnt) in stage.items()}
    pts = n * w["M_G"] ** 3
    flops = {"spread": 16.0 * pts, "gather": 16.0 * pts}
    n_nb = n / w["L"] ** 3 * 4.0 / 3.0 * math.pi * w["r_c"] ** 3
    flops["pair"] = 150.0 * n * n_nb
    dominant = max(("spread", "gather", "pair"), key=lambda s: avg[s] or 0.0)
    achieved = flops[dominant] / (avg[dominant] * 1e-3) / 1e12
    roofline = {"bound": "alu", "kernel": dominant, "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved / alu_peak, "traffic": TRAFFIC_BYTES.get(args.workload, {}).get(dominant),
                "peak_source": f"{sm_count} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz",
                "flops_per_launch": flops[dominant]}
    M3 = w["M"] ** 3
    fft_bytes = 72.0 * M3
    hbm = pk.get("hbm_gbs", 6800.0)
    stages_out = {name: {"ms_avg": avg[name], "launches": int(stage[name][1])} for name in stage}
    if avg["fft_solve"]:
        stages_out["fft_solve"]["GBps"] = fft_bytes / (avg["fft_solve"] * 1e-3) / 1e9
        stages_out["fft_solve"]["frac_hbm"] = stages_out["fft_solve"]["GBps"] / hbm
    for s_ in ("spread", "gather"):
        if avg[s_]:
            stages_out[s_]["TFLOPs"] = flops[s_] / (avg[s_] * 1e-3) / 1e12
            stages_out[s_]["frac_alu"] = stages_out[s_]["TFLOPs"] / alu_peak
            byts = 12.0 * M3 + 48.0 * n
            stages_out[s_]["GBps"] = byts / (avg[s_] * 1e-3) / 1e9
            stages_out[s_]["frac_hbm"] = stages_out[s_]["GBps"] / hbm

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload)

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": describe(w, B), "particles_per_step_per_gpu": n * B,
                      "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                      "l2": "flushed (256 MB write) before every apply"},
           "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": B * 3 * n * 3 * 4,
                   "d2h_bytes_per_step": B * 2 * n * 3 * 4},
           "gpu_launches": int(launches), "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks,
           "fp64_plain": fp64,
           "speedup_vs_fp64_plain": (value / world / fp64["value"]) if fp64 else None,
           "stages": stages_out, "apply_ms_median": statistics.median(apply_ms),
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
