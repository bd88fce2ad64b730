#!/usr/bin/env python
"""Benchmark of the HISQ even/odd hot path on GB300.

Workload (one step = one pass of the hot path): a mixed-precision CG solve of
A = 4m^2 - D_eo D_oe on a 48^3x12 lattice (eps = 0.3 synthetic links, m = 0.01, Gaussian
source) from x = 0 to true relative residual 1e-10: FP32 link/spinor inner iterations
(D_oe, D_eo with fused axpy + FP64 dot, FP64-reduced BLAS-1), FP64 reliable updates every
50 iterations (FP64 Dslash), FP64 solution accumulator.

Metric: Dslash GB/s (algorithmic bytes of every Dslash application in the solve / solve
time) -- the whole-job throughput of the step -- with the roofline of the dominant kernel
(the FP32 Dslash, timed live with CUDA events on its stream) against the measured HBM peak,
and CG time-to-1e-10 of the mixed-precision and plain FP64 solves at m = 0.01 and 0.002.

--impl reference runs the CPU FP64 oracle (the reference arm of this build) on a bounded
sample of the same workload. N > 1 GPUs run independent replicas (the path is not sharded).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Dslash GB/s & % HBM peak; CG time-to-1e-10 (mixed/learned vs FP64, 1 GB300)"
DIMS = (48, 48, 48, 12)
MASS = 0.01
TOL = 1e-10
GAUGE_SEED, SOURCE_SEED = 1001, 2001
FALLBACK_HBM = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-extras", action="store_true",
                    help="time the steps only: no e2e, comparison solves or CPU baseline (for profiler launch lists)")
    ap.add_argument("--sweep", action="store_true", help="Dslash sweep over lattices/precisions (table, not the contract line)")
    return ap.parse_args()


# ----------------------------------------------------------------------------- helpers
def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "of measured"
    except Exception:
        return FALLBACK_HBM, "of fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for name in ("dslash_impl.cuh", "internal.cuh", "dslash_launch.cuh"):
        with open(os.path.join(ROOT, "paper_2111_10354_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(profile_name: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", profile_name)
    try:
        kv = {}
        with open(path) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_source_hash") != kernel_source_hash():
            return None
        return float(kv["dram_bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, device_index: int):
        self.dev = device_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + ",".join(self.FIELDS), "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == len(self.FIELDS):
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def gen_workload(rank: int):
    import hisq_inputs as hin
    fat, lng = hin.gen_links(DIMS, GAUGE_SEED + rank, 0.3, 0.1)
    half = int(np.prod(DIMS)) // 2
    b = hin.gen_source(SOURCE_SEED + rank, half, 1)
    return fat, lng, b


# ----------------------------------------------------------------------------- CPU oracle
def oracle_sample(fat, lng, b, target_s: float = 12.0):
    """The oracle's FP64 CG on the same lattice, bounded: enough iterations for ~target_s seconds.
    Returns (GB/s of Dslash algorithmic bytes at FP64, seconds, iterations, threads)."""
    import oracle
    L = DIMS
    ff, lf = oracle.fold_links(L, fat.reshape(-1, 4, 3, 3), lng.reshape(-1, 4, 3, 3))
    half = int(np.prod(L)) // 2
    t0 = time.perf_counter()
    oracle.apply_A(L, ff, lf, MASS, b[0])
    t_apply = time.perf_counter() - t0
    iters = max(1, int(target_s / max(t_apply, 1e-3)) - 1)
    t0 = time.perf_counter()
    oracle.cg(L, ff, lf, MASS, b[0], tol=1e-30, maxiter=iters)
    dt = time.perf_counter() - t0
    n_dslash = 2 * (iters + 1)  # initial residual + one A per iteration
    bytes_ = n_dslash * half * (16 * 18 + 12) * 8.0
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return bytes_ / dt / 1e9, dt, iters, threads


def run_reference(args, rank, world):
    """Reference arm: the CPU FP64 oracle, as it stands, on the host cores (rank 0 only)."""
    if rank != 0:
        return
    fat, lng, b = gen_workload(0)
    vals = []
    per_step_target = 6.0
    for i in range(args.warmup + args.steps):
        gbs, dt, iters, threads = oracle_sample(fat, lng, b, target_s=per_step_target if i >= args.warmup else 2.0)
        if i >= args.warmup:
            vals.append((gbs, dt, iters))
    value = statistics.mean(v[0] for v in vals)
    ms = 1000 * statistics.mean(v[1] for v in vals)
    sample = "oracle FP64 CG on %s m=%g, %d iterations per step (%d Dslash), OpenMP" % (
        "x".join(map(str, DIMS)), MASS, vals[0][2], 2 * (vals[0][2] + 1))
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(), "lattice": list(DIMS), "mass": MASS},
            "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_name():
    return "HISQ mixed-precision CG to 1e-10 on 48^3x12 (FP32 inner D_eo/D_oe, FP64 reliable updates every 50), m=0.01"


# ----------------------------------------------------------------------------- GPU arm
def vec_like(torch, half, prec, nrhs=1, seed=5):
    import hisq_inputs as hin
    v = torch.from_numpy(hin.gen_source(seed, half, nrhs))
    if prec == 0:
        return v.cuda()
    if prec == 1:
        return v.to(torch.complex64).cuda()
    r = torch.view_as_real(v.to(torch.complex64))
    return r.to(torch.float16 if prec == 2 else torch.bfloat16).contiguous().cuda()


def time_dslash(torch, lat, prec, nrhs, reps, stream):
    """Average device time of one Dslash launch (alternating D_oe, D_eo) with CUDA events on its stream."""
    x = vec_like(torch, lat.half, prec, nrhs)
    y, z = torch.empty_like(x), torch.empty_like(x)
    with torch.cuda.stream(stream):
        for _ in range(3):
            lat.dslash(1, y, x, prec, nrhs)
            lat.dslash(0, z, y, prec, nrhs)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            lat.dslash(1, y, x, prec, nrhs)
            lat.dslash(0, z, y, prec, nrhs)
        e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / (2 * reps)


def run_ours(args, rank, world, local):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2111_10354_gb300 as h

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    fat, lng, b_np = gen_workload(rank)
    stream = torch.cuda.Stream()
    lat = h.Lattice(DIMS, precs=(h.HISQ_F64, h.HISQ_F32, h.HISQ_F16), stream=stream).load(fat, lng)
    half = lat.half
    b = torch.from_numpy(b_np).cuda()
    x = torch.zeros_like(b)
    opts = dict(inner_prec=h.HISQ_F32, reliable_period=50)

    def solve(xv, bv, **o):
        with torch.cuda.stream(stream):
            xv.zero_()
        return lat.cg(xv, bv, MASS, TOL, 20000, **(o or opts))

    for _ in range(args.warmup):
        solve(x, b)
    barrier()
    launches = 0
    dbytes = 0.0
    iters = []
    dev_index = torch.cuda.current_device()
    with ClockSampler(dev_index) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            rc, st = solve(x, b)
            launches += st["kernel_launches"]
            dbytes += st["dslash_bytes"]
            iters.append((st["iters"], st["reliable_updates"], st["true_rel_residual"]))
        e1.record(stream)
        e1.synchronize()
        barrier()
    t_ms = e0.elapsed_time(e1)
    t_max = t_ms
    tot_bytes = dbytes
    if dist:
        tt = torch.tensor([t_ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
        bb = torch.tensor([dbytes], device="cuda", dtype=torch.float64)
        dist.all_reduce(bb)
        tot_bytes = float(bb.item())
    value = tot_bytes / (t_max * 1e-3) / 1e9
    worst_res = max(r for _, _, r in iters)

    if args.skip_extras:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup,
                              "ms_per_step": round(t_max / args.steps, 3), "gpu_launches": int(launches),
                              "note": "--skip-extras: timed steps only"}), flush=True)
        if dist:
            dist.destroy_process_group()
        return

    # end to end through the C ABI with host buffers (copies inside the timed region)
    b_host = np.ascontiguousarray(b_np)
    x_host = np.zeros_like(b_host)
    barrier()
    t0 = time.perf_counter()
    e2e_bytes = 0.0
    for _ in range(args.steps):
        x_host[:] = 0
        rc, st = lat.cg(x_host, b_host, MASS, TOL, 20000, **opts)
        e2e_bytes += st["dslash_bytes"]
    barrier()
    t_e2e = time.perf_counter() - t0
    if dist:
        tt = torch.tensor([t_e2e], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_e2e = float(tt.item())
        bb = torch.tensor([e2e_bytes], device="cuda", dtype=torch.float64)
        dist.all_reduce(bb)
        e2e_bytes = float(bb.item())
    vec_bytes = b_host.nbytes

    # roofline of the dominant kernel: the FP32 Dslash, timed live on its stream
    reps = 50
    ms_launch = time_dslash(torch, lat, h.HISQ_F32, 1, reps, stream)
    bytes_launch = lat.dslash_bytes(h.HISQ_F32, 1)
    peak, peak_src = peaks()
    achieved = bytes_launch / (ms_launch * 1e-3) / 1e9
    launches += 2 * (reps + 3)

    # time-to-1e-10 comparisons (mixed FP32, mixed FP16, plain FP64) at both masses
    cmp = {}
    for m in (0.01, 0.002):
        row = {}
        for name, o in (("mixed_f32", dict(inner_prec=h.HISQ_F32)), ("mixed_f16", dict(inner_prec=h.HISQ_F16)),
                        ("fp64", dict(inner_prec=h.HISQ_F64))):
            xs = torch.zeros_like(b)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, st = lat.cg(xs, b, m, TOL, 20000, **o)
            dt = time.perf_counter() - t0
            row[name] = {"s": round(dt, 4), "iters": st["iters"], "true_res": st["true_rel_residual"]}
        cmp["m=%g" % m] = row

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        gbs, dt, it, threads = oracle_sample(fat, lng, b_np, 12.0)
        cpu = {"value": round(gbs, 4), "unit": "GB/s", "cores": threads, "kind": "oracle",
               "sample": "oracle FP64 CG on 48x48x48x12 m=0.01: %d iterations (%d Dslash) in %.1f s" % (
                   it, 2 * (it + 1), dt)}
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t_max / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 inner / f64 reliable", "data": "synthetic",
        "config": {"workload": workload_name(), "lattice": list(DIMS), "mass": MASS, "tol": TOL,
                   "inner_prec": "f32", "reliable_period": 50, "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2: FP64+FP32+FP16 links %.2f GB resident" % (
                       half * 16 * 18 * (8 + 4 + 2) / 1e9),
                   "iters_per_solve": iters[0][0], "reliable_updates": iters[0][1],
                   "worst_true_rel_residual": worst_res},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "peak_source": peak_src,
                     "kernel": "dslash_kernel<float,float,1,EPI_PLAIN> 48^3x12",
                     "us_per_launch": round(ms_launch * 1e3, 2), "bytes_per_launch": bytes_launch,
                     "traffic": ncu_traffic("ncu_dslash_f32_48c12.txt")},
        "cpu_baseline": cpu,
        "e2e": {"value": round(e2e_bytes / t_e2e / 1e9, 2), "unit": "GB/s", "h2d_bytes_per_step": 2 * vec_bytes,
                "d2h_bytes_per_step": vec_bytes},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "time_to_1e-10": cmp,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_sweep():
    """Dslash throughput over the lattice sizes and precisions of the precision workload (table)."""
    import torch

    import __graft_entry__
    import hisq_inputs as hin
    __graft_entry__.build()
    import paper_2111_10354_gb300 as h
    peak, src = peaks()
    stream = torch.cuda.Stream()
    sizes = [(32, 32, 32, 8), (48, 48, 48, 12), (64, 64, 64, 16), (96, 96, 96, 24), (144, 144, 144, 36)]
    for L in sizes:
        V = int(np.prod(L))
        precs = (h.HISQ_F64, h.HISQ_F32, h.HISQ_F16)
        lat = h.Lattice(L, precs=precs, stream=stream)
        # slab by slab keeps the host link arrays small even at 144^3x36
        nt = max(1, min(L[3], int(2e8 // (L[0] * L[1] * L[2] * 4 * 9 * 16))))
        for t0 in range(0, L[3], nt):
            n = min(nt, L[3] - t0)
            fat, lng = hin.gen_links(L, GAUGE_SEED, 0.3, 0.1, t0=t0, nt=n)
            h.hisq_load_links_slab(lat.ctx, t0, n, fat, lng)
        for p in precs:
            for nrhs in ((1, 4, 8, 16) if p == h.HISQ_F32 and L == (48, 48, 48, 12) else (1,)):
                ms = time_dslash(torch, lat, p, nrhs, 20, stream)
                by = lat.dslash_bytes(p, nrhs)
                print(json.dumps({"lattice": "x".join(map(str, L)), "prec": h.PREC_NAMES[p], "nrhs": nrhs,
                                  "us": round(ms * 1e3, 2), "GB/s": round(by / ms / 1e6, 1),
                                  "frac_hbm": round(by / ms / 1e6 / peak, 3),
                                  "sites_per_s": round(nrhs * V / 2 / (ms * 1e-3), 1),
                                  "GFLOP/s": round(1146 * nrhs * V / 2 / (ms * 1e-3) / 1e9, 1)}), flush=True)
        lat.close()
        del lat
        torch.cuda.empty_cache()


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.sweep:
        run_sweep()
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
