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

--impl reference runs the CPU FP64 oracle (the reference arm: there is no reference code) on a bounded
sample of the same workload. N > 1 GPUs run independent replicas (the path is not sharded).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import re
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
FP64_PIPE_TFLOPS = 1.20  # GB300 DFMA throughput, measured on this GPU type with an independent-FMA loop


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
    ap.add_argument("--kernel-case", choices=["dslash-f64", "dslash-df64", "dslash-f16", "dslash-f32-comp", "dslash-f32-nr8",
                                                   "cg-f32-nr8", "ptc", "fcg", "batch", "smear-f64", "smear-df64",
                                                   "dslash-f16-il64-tc", "cg-f32", "multishift", "dslash-f32-il8",
                                                   "dslash-f32-il16", "dslash-f32-48", "dslash-f32-96",
                                                   "dslash-f32-144"],
                    help="run a few launches of one kernel on a small case (for profiler captures)")
    ap.add_argument("--row", choices=["multirhs", "multishift", "batch", "learned", "smear"],
                    help="measure one of the batching / learned-preconditioner workloads (JSON lines)")
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


def _code_only(text: str) -> str:
    """Source text without comments and blank lines (an edit to a comment compiles to the same kernel)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = (re.sub(r"//.*", "", l).rstrip() for l in text.splitlines())
    return "\n".join(l for l in lines if l.strip())


def kernel_source_hash():
    """Hash of the code the single-vector Dslash kernel is compiled from (kernel body, its helpers and
    types), comments left out."""
    h = hashlib.sha256()
    for name in ("dslash_impl.cuh", "internal.cuh", "df64.cuh", "pdl.cuh"):
        with open(os.path.join(ROOT, "paper_2111_10354_gb300", "csrc", name)) as f:
            h.update(_code_only(f.read()).encode())
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
def omp_threads(n=None):
    """Set (n given) and return the OpenMP thread count of the oracle's runtime (libgomp)."""
    import ctypes
    try:
        gomp = ctypes.CDLL("libgomp.so.1")
    except OSError:
        return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    if n is not None:
        gomp.omp_set_num_threads(int(n))
    return int(gomp.omp_get_max_threads())


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the CPU-baseline record."""
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_sample(fat, lng, b, target_s: float = 12.0):
    """The oracle's FP64 CG on the same lattice, bounded: enough iterations for ~target_s seconds.
    Returns (GB/s of Dslash algorithmic bytes at FP64, seconds, iterations, threads)."""
    import oracle
    oracle.build()
    threads = omp_threads()
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
    return bytes_ / dt / 1e9, dt, iters, threads


def oracle_solve(fat, lng, b, tol: float = 1e-12, maxiter: int = 600):
    """The oracle's FP64 CG on the same lattice and source, run to convergence (relative residual tol):
    the timed CPU baseline, and the solution every GPU solve's final error is stated against.
    Returns (GB/s of Dslash algorithmic bytes at FP64, seconds, iterations, threads, x)."""
    import oracle
    oracle.build()
    threads = omp_threads()
    L = DIMS
    ff, lf = oracle.fold_links(L, fat.reshape(-1, 4, 3, 3), lng.reshape(-1, 4, 3, 3))
    half = int(np.prod(L)) // 2
    t0 = time.perf_counter()
    x, its = oracle.cg(L, ff, lf, MASS, b[0], tol=tol, maxiter=maxiter)
    dt = time.perf_counter() - t0
    iters = its if its >= 0 else maxiter
    bytes_ = 2 * (iters + 1) * half * (16 * 18 + 12) * 8.0
    return bytes_ / dt / 1e9, dt, iters, threads, (x if its >= 0 else None)


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
                             "cpu_model": cpu_model(),
                             "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_name():
    return "HISQ mixed-precision CG to 1e-10 on 48^3x12 (FP32 inner D_eo/D_oe, FP64 reliable updates every 50), m=0.01"


def aggregate(t_local, bytes_local, dist, device):
    """Whole-job figures of N replicas: the slowest rank's time and the bytes of all ranks."""
    if dist is None:
        return float(t_local), float(bytes_local)
    import torch
    tt = torch.tensor([float(t_local)], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    bb = torch.tensor([float(bytes_local)], device=device, dtype=torch.float64)
    dist.all_reduce(bb)
    return float(tt.item()), float(bb.item())


# ----------------------------------------------------------------------------- GPU arm
def vec_like(torch, half, prec, nrhs=1, seed=5):
    import hisq_inputs as hin
    v = torch.from_numpy(hin.gen_source(seed, half, nrhs))
    if prec in (0, 4):  # FP64 and double-float take complex128 vectors
        return v.cuda()
    if prec == 1:
        return v.to(torch.complex64).cuda()
    r = torch.view_as_real(v.to(torch.complex64))
    return r.to(torch.float16 if prec == 2 else torch.bfloat16).contiguous().cuda()


def antiherm_rel(torch, lat, prec):
    """|<u, D_eo v> + <D_oe u, v>| / |<u, D_eo v>| for random u, v: zero up to rounding for any correct
    operator at any lattice size (the check the sweep records where the oracle cannot be run)."""
    u, v = vec_like(torch, lat.half, prec, 1, seed=11), vec_like(torch, lat.half, prec, 1, seed=12)
    Dv, Du = torch.empty_like(v), torch.empty_like(u)
    torch.cuda.synchronize()  # inputs were written on torch's stream, the library runs on its own
    lat.dslash(0, Dv, v, prec, 1)
    lat.dslash(1, Du, u, prec, 1)
    torch.cuda.synchronize()

    def c128(t):
        if t.dtype in (torch.float16, torch.bfloat16):
            t = torch.view_as_complex(t.float().contiguous())
        return t.to(torch.complex128).flatten()
    lhs = complex(torch.vdot(c128(u), c128(Dv)))
    rhs = -complex(torch.vdot(c128(Du), c128(v)))
    return abs(lhs - rhs) / abs(lhs)


def lanczos_record(st):
    """A's extreme eigenvalues and condition number as a CG solve's Lanczos coefficients estimate them."""
    if not st.get("lanczos_steps") or st["lambda_min"] <= 0:
        return None
    return {"lambda_min": float("%.5g" % st["lambda_min"]), "lambda_max": float("%.5g" % st["lambda_max"]),
            "kappa": float("%.5g" % (st["lambda_max"] / st["lambda_min"])), "lanczos_steps": st["lanczos_steps"]}


def time_dslash(torch, lat, prec, nrhs, reps, stream, interleaved=False):
    """Average device time of one Dslash launch (alternating D_oe, D_eo) with CUDA events on its stream.
    interleaved: the rhs-interleaved layout [cb][color][rhs] (the same Gaussian entries, placed per site)."""
    x = vec_like(torch, lat.half, prec, nrhs)
    y, z = torch.empty_like(x), torch.empty_like(x)
    D = lat.dslash_interleaved if interleaved else lat.dslash
    torch.cuda.synchronize()  # x was written on torch's stream
    with torch.cuda.stream(stream):
        for _ in range(3):
            D(1, y, x, prec, nrhs)
            D(0, z, y, prec, nrhs)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            D(1, y, x, prec, nrhs)
            D(0, z, y, prec, nrhs)
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
    lat = h.Lattice(DIMS, precs=(h.HISQ_F64, h.HISQ_F32, h.HISQ_F16, h.HISQ_DF64), stream=stream).load(fat, lng)
    half = lat.half
    b = torch.from_numpy(b_np).cuda()
    x = torch.zeros_like(b)
    torch.cuda.synchronize()  # b and x were written on torch's stream; the solves run on the library's
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
    t_max, tot_bytes = aggregate(t_ms, dbytes, dist, "cuda")
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

    # end to end through the C ABI with pinned host buffers (the library copies b and the initial x in
    # and x out on its stream, inside the timed region)
    b_pin = torch.from_numpy(np.ascontiguousarray(b_np)).pin_memory()
    x_pin = torch.zeros_like(b_pin).pin_memory()
    b_host, x_host = b_pin.numpy(), x_pin.numpy()
    barrier()
    t0 = time.perf_counter()
    e2e_bytes = 0.0
    for _ in range(args.steps):
        x_host[:] = 0
        rc, st = lat.cg(x_host, b_host, MASS, TOL, 20000, **opts)
        e2e_bytes += st["dslash_bytes"]
    barrier()
    t_e2e = time.perf_counter() - t0
    t_e2e, e2e_bytes = aggregate(t_e2e, e2e_bytes, dist, "cuda")
    vec_bytes = b_host.nbytes

    # roofline of the dominant kernel: the FP32 Dslash, timed live on its stream
    reps = 50
    ms_launch = time_dslash(torch, lat, h.HISQ_F32, 1, reps, stream)
    bytes_launch = lat.dslash_bytes(h.HISQ_F32, 1)
    peak, peak_src = peaks()
    achieved = bytes_launch / (ms_launch * 1e-3) / 1e9

    # time-to-1e-10 comparisons (mixed FP32, mixed FP16 with FP32 and with FP16 inner vectors, plain FP64)
    # at both masses, and the same with the double-float operator (plain CG, and FP32 inner with
    # double-float reliable updates); every solve is judged by its true residual
    cmp = {}
    sols = {}  # GPU solutions at the benchmark's mass, for their error against the oracle's solution
    for m in (0.01, 0.002):
        row = {}
        for name, o in (("mixed_f32", dict(inner_prec=h.HISQ_F32)), ("mixed_f16", dict(inner_prec=h.HISQ_F16)),
                        ("mixed_f16_spinor16", dict(inner_prec=h.HISQ_F16, spinor_prec=h.HISQ_F16)),
                        ("fp64", dict(inner_prec=h.HISQ_F64)), ("df64", dict(inner_prec=h.HISQ_DF64)),
                        ("mixed_f32_df64_reliable", dict(inner_prec=h.HISQ_F32, reliable_prec=h.HISQ_DF64))):
            xs = torch.zeros_like(b)
            torch.cuda.synchronize()
            lat.cg(xs, b, m, TOL, 20000, **o)  # first call tunes this variant's kernels
            xs.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, st = lat.cg(xs, b, m, TOL, 20000, **o)
            dt = time.perf_counter() - t0
            row[name] = {"s": round(dt, 4), "iters": st["iters"], "true_res": st["true_rel_residual"]}
            if name == "fp64":
                # the conditioning of this workload: Lanczos estimate from the FP64 solve's coefficients
                row["lanczos_A"] = lanczos_record(st)
            if m == MASS:
                sols[name] = xs.cpu().numpy()[0]
        cmp["m=%g" % m] = row
    # the same solves with compressed long links (two rows stored, third rebuilt in the kernel)
    lat.compress_long(-1.0 / 24.0).load(fat, lng)
    for m in (0.01, 0.002):
        for name, o in (("mixed_f32_comp12", dict(inner_prec=h.HISQ_F32)),
                        ("mixed_f16_comp12", dict(inner_prec=h.HISQ_F16)),
                        ("mixed_f16_spinor16_comp12", dict(inner_prec=h.HISQ_F16, spinor_prec=h.HISQ_F16))):
            xs = torch.zeros_like(b)
            torch.cuda.synchronize()
            lat.cg(xs, b, m, TOL, 20000, **o)  # first call tunes the compressed kernels
            xs.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, st = lat.cg(xs, b, m, TOL, 20000, **o)
            dt = time.perf_counter() - t0
            cmp["m=%g" % m][name] = {"s": round(dt, 4), "iters": st["iters"], "true_res": st["true_rel_residual"]}
            if m == MASS:
                sols[name] = xs.cpu().numpy()[0]
    ms_comp = time_dslash(torch, lat, h.HISQ_F32, 1, reps, stream)

    # the conditioning of the small plain-method workload (8^4, m = 0.1, FP64 CG to 1e-10), beside the
    # benchmark's own
    L8 = (8, 8, 8, 8)
    import hisq_inputs as hin
    small = h.Lattice(L8, precs=(h.HISQ_F64,), stream=stream).load(*hin.gen_links(L8, 1000, 0.3, 0.1))
    b8 = torch.from_numpy(hin.gen_source(2000, small.half, 1)).cuda()
    x8 = torch.zeros_like(b8)
    torch.cuda.synchronize()
    small.cg(x8, b8, 0.1, TOL, 20000, inner_prec=h.HISQ_F64)  # first call tunes and captures
    x8.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc, st8 = small.cg(x8, b8, 0.1, TOL, 20000, inner_prec=h.HISQ_F64)
    dt8 = time.perf_counter() - t0
    cmp["8^4 m=0.1"] = {"fp64": {"s": round(dt8, 5), "iters": st8["iters"], "true_res": st8["true_rel_residual"]},
                        "lanczos_A": lanczos_record(st8)}
    small.close()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle's FP64 CG on the same small workload, on the host's cores
        import oracle
        oracle.build()
        f8, l8 = hin.gen_links(L8, 1000, 0.3, 0.1)
        ff8, lf8 = oracle.fold_links(L8, f8.reshape(-1, 4, 3, 3), l8.reshape(-1, 4, 3, 3))
        b8h = hin.gen_source(2000, int(np.prod(L8)) // 2, 1)[0]
        t0 = time.perf_counter()
        _, it8 = oracle.cg(L8, ff8, lf8, 0.1, b8h, tol=TOL, maxiter=20000)
        cmp["8^4 m=0.1"]["oracle_fp64_cpu"] = {"s": round(time.perf_counter() - t0, 5), "iters": it8,
                                               "cores": omp_threads()}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        # the oracle's FP64 CG on the same source, to a 1e-12 relative residual: the timed baseline, and
        # the solution each GPU solve at this mass is compared with (final error per solve)
        gbs, dt, it, threads, x_or = oracle_solve(fat, lng, b_np)
        cpu = {"value": round(gbs, 4), "unit": "GB/s", "cores": threads, "kind": "oracle", "cpu_model": cpu_model(),
               "sample": "oracle FP64 CG on 48x48x48x12 m=%g to a 1e-12 relative residual: %d iterations "
                         "(%d Dslash) in %.1f s" % (MASS, it, 2 * (it + 1), dt)}
        if x_or is not None:
            nx = np.linalg.norm(x_or)
            for name, xg in sols.items():
                cmp["m=%g" % MASS][name]["final_err_vs_oracle"] = float("%.3g" % (np.linalg.norm(xg - x_or) / nx))
        # the same oracle on one host core
        all_threads = omp_threads()
        omp_threads(1)
        gbs1, dt1, it1, _ = oracle_sample(fat, lng, b_np, 5.0)
        omp_threads(all_threads)
        cpu["single_core"] = {"value": round(gbs1, 4), "unit": "GB/s", "cores": 1,
                              "sample": "%d iterations (%d Dslash) in %.1f s" % (it1, 2 * (it1 + 1), dt1)}
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t_max / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 inner / f64 reliable", "data": "synthetic",
        "config": {"workload": workload_name(), "lattice": list(DIMS), "mass": MASS, "tol": TOL,
                   "inner_prec": "f32", "reliable_period": 50, "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2: FP64+FP32+FP16+double-float links %.2f GB resident" % (
                       half * 16 * 18 * (8 + 4 + 2 + 8) / 1e9),
                   "iters_per_solve": iters[0][0], "reliable_updates": iters[0][1],
                   "worst_true_rel_residual": worst_res},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "peak_source": peak_src,
                     "kernel": "dslash_kernel<float,float,1,EPI_PLAIN> 48^3x12",
                     "us_per_launch": round(ms_launch * 1e3, 2), "bytes_per_launch": bytes_launch,
                     "us_per_launch_compressed_long_links": round(ms_comp * 1e3, 2),
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
        # double-float links are resident too where they fit beside the others (not at 144^3x36, where
        # FP64 + FP32 + FP16 + BF16 already take 248 GB)
        precs = (h.HISQ_F64, h.HISQ_F32, h.HISQ_F16, h.HISQ_BF16) + ((h.HISQ_DF64,) if L[0] < 144 else ())
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
                line = {"lattice": "x".join(map(str, L)), "prec": h.PREC_NAMES[p], "nrhs": nrhs,
                        "us": round(ms * 1e3, 2), "GB/s": round(by / ms / 1e6, 1),
                        "frac_hbm": round(by / ms / 1e6 / peak, 3),
                        "sites_per_s": round(nrhs * V / 2 / (ms * 1e-3), 1),
                        "GFLOP/s": round(1146 * nrhs * V / 2 / (ms * 1e-3) / 1e9, 1)}
                if nrhs == 1:
                    line["antiherm_rel"] = float("%.3g" % antiherm_rel(torch, lat, p))
                print(json.dumps(line), flush=True)
        # the tuner's choice per kernel: variant * 10000 + block
        print(json.dumps({"lattice": "x".join(map(str, L)), "tuned": h.hisq_tune_report(lat.ctx).splitlines()}),
              flush=True)
        lat.close()
        del lat
        torch.cuda.empty_cache()
        print(json.dumps(oracle_dslash_timing(hin, L)), flush=True)


def host_mem_available() -> float:
    """Bytes of host memory available now (MemAvailable), 0 if unknown."""
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return float(line.split()[1]) * 1024
    except OSError:
        pass
    return 0.0


def oracle_dslash_timing(hin, L, reps: int = 5):
    """The oracle's FP64 Dslash on the sweep lattice L, timed on the host beside the GPU: reps applies on all
    OpenMP threads and one on a single thread, when the full-lattice host arrays fit in memory (links as
    generated and as folded: 2304 bytes per site), else the reason it was skipped."""
    import oracle
    V = int(np.prod(L))
    need = 2304.0 * V * 1.25
    avail = host_mem_available()
    rec = {"lattice": "x".join(map(str, L)), "oracle_dslash": None}
    if avail and need > avail:
        rec["oracle_dslash"] = "skipped: needs %.0f GB of host memory, %.0f GB available" % (need / 1e9, avail / 1e9)
        return rec
    oracle.build()
    fat, lng = hin.gen_links(L, GAUGE_SEED, 0.3, 0.1)
    ff, lf = oracle.fold_links(L, fat.reshape(-1, 4, 3, 3), lng.reshape(-1, 4, 3, 3))
    del fat, lng
    v = hin.gen_source(SOURCE_SEED, V // 2, 1)[0]
    threads = omp_threads()
    oracle.dslash(L, ff, lf, 1, v)  # first touch
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.dslash(L, ff, lf, 1, v)
    dt = (time.perf_counter() - t0) / reps
    omp_threads(1)
    t0 = time.perf_counter()
    oracle.dslash(L, ff, lf, 1, v)
    dt1 = time.perf_counter() - t0
    omp_threads(threads)
    sites = V / 2
    rec["oracle_dslash"] = {"threads": threads, "cpu_model": cpu_model(), "reps": reps, "s_per_apply": round(dt, 4),
                            "sites_per_s": float("%.4g" % (sites / dt)), "GB/s": round(sites * 2400 / dt / 1e9, 2),
                            "single_thread_s_per_apply": round(dt1, 3),
                            "single_thread_sites_per_s": float("%.4g" % (sites / dt1))}
    return rec


# ----------------------------------------------------------------------------- other workloads
def _timed(torch, fn):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return time.perf_counter() - t0, out


def row_multirhs(h, torch, hin):
    """48^3x12: Dslash with 1-16 vectors per link read (FP16, FP64, FP32) and FP32 mixed CG on 1-16 sources."""
    L = (48, 48, 48, 12)
    fat, lng = hin.gen_links(L, 1002, 0.3, 0.1)
    stream = torch.cuda.Stream()
    lat = h.Lattice(L, precs=(h.HISQ_F64, h.HISQ_F32, h.HISQ_F16, h.HISQ_BF16, h.HISQ_DF64), stream=stream).load(fat, lng)
    peak, _ = peaks()
    dims = "x".join(map(str, L))
    # interleaved layout [cb][color][rhs], 16-bit storage: the tcgen05 tensor-core form against the
    # CUDA-core interleaved form, each forced; and the blocked CUDA-core form for reference
    for prec, name in ((h.HISQ_F16, "f16"), (h.HISQ_BF16, "bf16")):
        for n in (16, 32, 64):
            by = lat.dslash_bytes(prec, n)
            best = {}
            for path, form in ((1, "interleaved cuda-core"), (2, "interleaved tensor-core (tcgen05)")):
                h.hisq_tune_load(lat.ctx, "dslash_path_il/l%d/n%d %s -> %d\n" % (prec, n, dims, path))
                ms = time_dslash(torch, lat, prec, n, 10, stream, interleaved=True)
                best[path] = ms
                print(json.dumps({"row": "multirhs", "lattice": "48x48x48x12", "prec": name, "nrhs": n, "form": form,
                                  "dslash_us": round(ms * 1e3, 1), "dslash_GBps": round(by / ms / 1e6, 1),
                                  "dslash_frac_hbm": round(by / ms / 1e6 / peak, 3),
                                  "dslash_GFLOPs": round(1146 * n * lat.half / (ms * 1e-3) / 1e9, 1)}), flush=True)
            # keep the faster form, as the tuner would
            h.hisq_tune_load(lat.ctx, "dslash_path_il/l%d/n%d %s -> %d\n" % (prec, n, dims, min(best, key=best.get)))
    # FP32 storage: interleaved against blocked, n = 2 .. 16
    for n in (2, 4, 8, 16):
        by = lat.dslash_bytes(h.HISQ_F32, n)
        for il, form in ((False, "blocked"), (True, "interleaved")):
            ms = time_dslash(torch, lat, h.HISQ_F32, n, 10, stream, interleaved=il)
            print(json.dumps({"row": "multirhs", "lattice": "48x48x48x12", "prec": "f32", "nrhs": n, "form": form,
                              "dslash_us": round(ms * 1e3, 1), "dslash_frac_hbm": round(by / ms / 1e6 / peak, 3),
                              "dslash_GFLOPs": round(1146 * n * lat.half / (ms * 1e-3) / 1e9, 1)}), flush=True)
    # Dslash only at FP16 storage (FP32 arithmetic) and FP64
    for prec, name, ns in ((h.HISQ_F16, "f16", (1, 2, 4, 8, 16)), (h.HISQ_F64, "f64", (1, 2, 4, 8))):
        for n in ns:
            ms = time_dslash(torch, lat, prec, n, 20 if prec != h.HISQ_F64 else 5, stream)
            by = lat.dslash_bytes(prec, n)
            print(json.dumps({"row": "multirhs", "lattice": "48x48x48x12", "prec": name, "nrhs": n,
                              "dslash_us": round(ms * 1e3, 1), "dslash_GBps": round(by / ms / 1e6, 1),
                              "dslash_frac_hbm": round(by / ms / 1e6 / peak, 3),
                              "dslash_GFLOPs": round(1146 * n * lat.half / (ms * 1e-3) / 1e9, 1)}), flush=True)
    for n in (1, 2, 4, 8, 16):
        ms = time_dslash(torch, lat, h.HISQ_F32, n, 20, stream)
        by = lat.dslash_bytes(h.HISQ_F32, n)
        b = torch.from_numpy(hin.gen_source(2002, lat.half, n)).cuda()
        x = torch.zeros_like(b)
        torch.cuda.synchronize()  # inputs come from torch's stream, the solve runs on the library's
        lat.cg(x, b, 0.01, 1e-10, 5000, nrhs=n, inner_prec=h.HISQ_F32)  # warm-up / tuning
        x.zero_()
        dt, (rc, st) = _timed(torch, lambda: lat.cg(x, b, 0.01, 1e-10, 5000, nrhs=n, inner_prec=h.HISQ_F32))
        print(json.dumps({"row": "multirhs", "lattice": "48x48x48x12", "prec": "f32", "nrhs": n,
                          "dslash_us": round(ms * 1e3, 1), "dslash_GBps": round(by / ms / 1e6, 1),
                          "dslash_frac_hbm": round(by / ms / 1e6 / peak, 3),
                          "dslash_GFLOPs": round(1146 * n * lat.half / (ms * 1e-3) / 1e9, 1),
                          "cg_s": round(dt, 4), "cg_s_per_rhs": round(dt / n, 4), "cg_iters": st["iters"],
                          "worst_true_res": st["true_rel_residual"]}), flush=True)
        # the same solve with double-float reliable updates (the FP64 Dslash of n vectors is FP64-pipe bound)
        lat.cg(x, b, 0.01, 1e-10, 5000, nrhs=n, inner_prec=h.HISQ_F32, reliable_prec=h.HISQ_DF64)
        x.zero_()
        dt, (rc, st) = _timed(torch, lambda: lat.cg(x, b, 0.01, 1e-10, 5000, nrhs=n, inner_prec=h.HISQ_F32,
                                                    reliable_prec=h.HISQ_DF64))
        print(json.dumps({"row": "multirhs", "lattice": "48x48x48x12", "prec": "f32", "reliable": "df64", "nrhs": n,
                          "cg_s": round(dt, 4), "cg_s_per_rhs": round(dt / n, 4), "cg_iters": st["iters"],
                          "worst_true_res": st["true_rel_residual"]}), flush=True)
        # FP16 links and FP16 inner vectors (FP32 arithmetic, FP64 reliable updates)
        o16 = dict(nrhs=n, inner_prec=h.HISQ_F16, spinor_prec=h.HISQ_F16)
        lat.cg(x, b, 0.01, 1e-10, 5000, **o16)
        x.zero_()
        dt, (rc, st) = _timed(torch, lambda: lat.cg(x, b, 0.01, 1e-10, 5000, **o16))
        print(json.dumps({"row": "multirhs", "lattice": "48x48x48x12", "prec": "f16", "spinor": "f16", "nrhs": n,
                          "cg_s": round(dt, 4), "cg_s_per_rhs": round(dt / n, 4), "cg_iters": st["iters"],
                          "worst_true_res": st["true_rel_residual"]}), flush=True)
    # launch forms the tuner chose: key -> variant * 10000 + block (vectors per thread x threads per site)
    print(json.dumps({"row": "multirhs", "tuned": h.hisq_tune_report(lat.ctx).splitlines()}), flush=True)


def row_multishift(h, torch, hin):
    """48^3x12, m = 0.0025, 14 shifts log-spaced in [1e-5, 1], every shift to 1e-9."""
    L = (48, 48, 48, 12)
    fat, lng = hin.gen_links(L, 1002, 0.3, 0.1)
    lat = h.Lattice(L, precs=(h.HISQ_F64, h.HISQ_F32, h.HISQ_DF64), stream=torch.cuda.Stream()).load(fat, lng)
    shifts = np.logspace(-5, 0, 14)
    b = torch.from_numpy(hin.gen_source(2002, lat.half, 1)).cuda()
    x = torch.zeros((14, lat.half, 3), dtype=torch.complex128, device="cuda")
    torch.cuda.synchronize()  # inputs come from torch's stream, the solve runs on the library's
    for name, o in (("fp32_krylov+refine", dict(inner_prec=h.HISQ_F32)),
                    ("fp32_krylov+refine, df64 verification and reliable updates",
                     dict(inner_prec=h.HISQ_F32, reliable_prec=h.HISQ_DF64)),
                    ("fp64", dict(inner_prec=h.HISQ_F64))):
        lat.multishift_cg(x, b, shifts, 0.0025, 1e-9, 20000, **o)
        dt, (rc, st) = _timed(torch, lambda: lat.multishift_cg(x, b, shifts, 0.0025, 1e-9, 20000, **o))
        print(json.dumps({"row": "multishift", "variant": name, "s": round(dt, 4), "iters": st["iters"],
                          "shift_iters": st["shift_iters"], "max_true_res": max(st["shift_residual"]),
                          "converged": st["converged"], "kernel_launches": st["kernel_launches"]}), flush=True)
    # the rational function RHMC applies with these solves (f3): out = a0 b + sum_k a_k (A + sigma_k)^-1 b,
    # with synthetic coefficients (the paper gives none); its cost is the multi-shift solve plus one pass
    coeffs = np.logspace(-3, 0, 14)
    out = torch.empty_like(b)
    for name, o in (("rational apply (fp32 krylov+refine)", dict(inner_prec=h.HISQ_F32)),
                    ("rational apply (fp32 krylov+refine, df64 verification)",
                     dict(inner_prec=h.HISQ_F32, reliable_prec=h.HISQ_DF64))):
        h.hisq_rational_apply(lat.ctx, out, b, 0.5, shifts, coeffs, 0.0025, 1e-9, 20000, h.make_opts(**o))
        dt, st = _timed(torch, lambda: h.hisq_rational_apply(lat.ctx, out, b, 0.5, shifts, coeffs, 0.0025, 1e-9, 20000,
                                                             h.make_opts(**o)))
        print(json.dumps({"row": "multishift", "variant": name, "s": round(dt, 4), "iters": st["iters"],
                          "max_true_res": st["true_rel_residual"], "converged": st["converged"]}), flush=True)
    # reference point: 14 independent mixed-precision solves
    xs = torch.zeros((1, lat.half, 3), dtype=torch.complex128, device="cuda")
    t = 0.0
    for s_ in shifts:
        xs.zero_()
        dt, _ = _timed(torch, lambda: h.hisq_cg(lat.ctx, xs, b, 1, float(np.sqrt(0.0025 ** 2 + s_ / 4)), 1e-9,
                                                20000, h.make_opts(inner_prec=h.HISQ_F32)))
        t += dt
    print(json.dumps({"row": "multishift", "variant": "14 separate mixed CG", "s": round(t, 4)}), flush=True)


def row_batch(h, torch, hin):
    """64 lattices (32 x 16^4, 19 x 24^3x8, 13 x 32^3x8), per-lattice eps and mass, to 1e-10."""
    mix = hin.lattice_mix_64()
    batch = h.Batch([m["dims"] for m in mix], stream=torch.cuda.Stream())
    lats, bs = [], []
    for l, m in enumerate(mix):
        fat, lng = hin.gen_links(m["dims"], m["gauge_seed"], m["eps"], 0.1)
        batch.load(l, fat, lng)
        lats.append((fat, lng))
        bs.append(hin.gen_source(m["source_seed"], int(np.prod(m["dims"])) // 2, 1)[0])
    b = torch.from_numpy(np.concatenate([v.reshape(-1) for v in bs]).reshape(-1, 3)).cuda()
    masses = [m["mass"] for m in mix]
    x = torch.zeros_like(b)
    torch.cuda.synchronize()  # inputs come from torch's stream, the solve runs on the library's
    for name, prec in (("batched mixed f32/f64", h.HISQ_F32), ("batched fp64", h.HISQ_F64)):
        batch.cg(x, b, masses, 1e-10, 10000, inner_prec=prec)
        x.zero_()
        dt, (rc, st) = _timed(torch, lambda: batch.cg(x, b, masses, 1e-10, 10000, inner_prec=prec))
        print(json.dumps({"row": "batch", "variant": name, "lattices": 64, "s": round(dt, 4),
                          "max_iters": st["iters"], "cycles": st["reliable_updates"],
                          "max_true_res": max(st["lattice_residual"]), "converged": st["converged"],
                          "kernel_launches": st["kernel_launches"],
                          "dslash_GBps_whole_solve": round(st["dslash_bytes"] / dt / 1e9, 1)}), flush=True)
    # reference point: the same 64 solves one lattice at a time through hisq_cg; an FP64 solve of each
    # lattice (untimed) records its conditioning (Lanczos estimate from the CG coefficients)
    t = 0.0
    kappas = []
    for l, m in enumerate(mix):
        lat = h.Lattice(m["dims"], precs=(h.HISQ_F64, h.HISQ_F32)).load(*lats[l])
        bl = torch.from_numpy(bs[l]).reshape(1, -1, 3).cuda()
        xl = torch.zeros_like(bl)
        lat.cg(xl, bl, m["mass"], 1e-10, 10000, inner_prec=h.HISQ_F32)
        xl.zero_()
        dt, _ = _timed(torch, lambda: lat.cg(xl, bl, m["mass"], 1e-10, 10000, inner_prec=h.HISQ_F32))
        t += dt
        xl.zero_()
        _, (_, st64) = _timed(torch, lambda: lat.cg(xl, bl, m["mass"], 1e-10, 10000, inner_prec=h.HISQ_F64))
        rec = lanczos_record(st64)
        if rec:
            kappas.append((rec["kappa"], m["mass"], rec["lambda_min"], rec["lambda_max"]))
        lat.close()
    ks = sorted(k[0] for k in kappas)
    print(json.dumps({"row": "batch", "variant": "64 sequential single-lattice mixed CG", "s": round(t, 4),
                      "kappa_A": {"min": ks[0], "median": ks[len(ks) // 2], "max": ks[-1],
                                  "lambda_min_over_4m2": [float("%.4g" % (k[2] / (4 * k[1] ** 2)))
                                                          for k in sorted(kappas)[::16]]} if ks else None}),
          flush=True)


def row_learned(h, torch, hin, epochs=12, batch_pairs=16, lr=0.02):
    """32^3x8, m = 0.001, eps = 0.35: train the PTC net on 4 fields x 128 (source, solution) pairs,
    then flexible CG with it vs mixed-precision CG on 4 held-out fields, to 1e-10."""
    import oracle.ptc as optc
    L = (32, 32, 32, 8)
    mass = 0.001
    stream = torch.cuda.Stream()

    def field(seed):
        fat, lng = hin.gen_links(L, seed, 0.35, 0.1)
        return h.Lattice(L, precs=(h.HISQ_F64, h.HISQ_F32), stream=stream).load(fat, lng)

    train = [field(4000 + i) for i in range(4)]
    half = train[0].half
    t0 = time.perf_counter()
    pairs = []
    for i, lat in enumerate(train):
        b = torch.from_numpy(hin.gen_source(5000 + i, half, 128)).cuda()
        x = torch.zeros_like(b)
        torch.cuda.synchronize()  # inputs come from torch's stream, the solve runs on the library's
        for k in range(0, 128, 16):  # 16 sources per link read
            lat.cg(x[k:k + 16], b[k:k + 16], mass, 1e-10, 20000, nrhs=16, inner_prec=h.HISQ_F32)
        pairs.append((b.to(torch.complex64), x.to(torch.complex64)))
    t_data = time.perf_counter() - t0
    W1, _ = optc.init_weights(4000, scale=0.05)
    W1[0, 0, 0] = 1.0
    net = h.Ptc(train[0])
    net.set_tied(True)  # N = B^dag B: Hermitian positive semi-definite preconditioner
    net.set_weights(W1, optc.tie(W1))
    t0 = time.perf_counter()
    losses = []
    for ep in range(epochs):
        ep_loss = []
        for k in range(0, 128, batch_pairs):
            for i, lat in enumerate(train):
                net.bind(lat)
                b, x = pairs[i]
                loss, _, _ = net.train_step(b[k:k + batch_pairs].contiguous(), x[k:k + batch_pairs].contiguous(),
                                            batch_pairs, lr)
                ep_loss.append(loss)
        losses.append(float(np.mean(ep_loss)))
    t_train = time.perf_counter() - t0
    print(json.dumps({"row": "learned", "phase": "train", "pairs": 512, "epochs": epochs, "lr": lr,
                      "data_s": round(t_data, 2), "train_s": round(t_train, 2), "loss_per_epoch": losses}),
          flush=True)
    # one application of the trained network against one application of A (FP32, the FCG's operator),
    # device time on the library's stream
    lat0 = train[0]
    net.bind(lat0)
    r32 = torch.from_numpy(hin.gen_source(1, half, 1)).to(torch.complex64).cuda()
    z32 = torch.empty_like(r32)
    torch.cuda.synchronize()
    ms_net = _stream_ms(torch, stream, lambda: net.apply(z32, r32, 1), 50)
    ms_A = _stream_ms(torch, stream, lambda: lat0.apply_A(z32, r32, mass, h.HISQ_F32, 1), 50)
    print(json.dumps({"row": "learned", "phase": "apply", "lattice": "32x32x32x8", "network_us": round(ms_net * 1e3, 1),
                      "A_us": round(ms_A * 1e3, 1)}), flush=True)
    for i in range(4):
        lat = field(4100 + i)
        net.bind(lat)
        b = torch.from_numpy(hin.gen_source(6000 + i, half, 1)).cuda()
        x = torch.zeros_like(b)
        torch.cuda.synchronize()  # inputs come from torch's stream, the solve runs on the library's
        net.fcg(x, b, mass, 1e-10, 20000)
        x.zero_()
        dt_f, (rc_f, st_f) = _timed(torch, lambda: net.fcg(x, b, mass, 1e-10, 20000))
        x2 = torch.zeros_like(b)
        torch.cuda.synchronize()
        lat.cg(x2, b, mass, 1e-10, 20000, inner_prec=h.HISQ_F32)
        x2.zero_()
        dt_c, (rc_c, st_c) = _timed(torch, lambda: lat.cg(x2, b, mass, 1e-10, 20000, inner_prec=h.HISQ_F32))
        x3 = torch.zeros_like(b)
        dt_d, (rc_d, st_d) = _timed(torch, lambda: lat.cg(x3, b, mass, 1e-10, 20000, inner_prec=h.HISQ_F64))
        print(json.dumps({"row": "learned", "phase": "held-out", "field": 4100 + i,
                          "fcg": {"s": round(dt_f, 4), "iters": st_f["iters"], "true_res": st_f["true_rel_residual"]},
                          "mixed_cg": {"s": round(dt_c, 4), "iters": st_c["iters"],
                                       "true_res": st_c["true_rel_residual"]},
                          "fp64_cg": {"s": round(dt_d, 4), "iters": st_d["iters"],
                                      "true_res": st_d["true_rel_residual"]},
                          "lanczos_A": lanczos_record(st_d)}), flush=True)


SMEAR_LEVEL1 = dict(c1=1 / 8, c3=1 / 16, c5=1 / 64, c7=1 / 384)  # fat7
SMEAR_LEVEL2 = dict(c1=5 / 8, c3=1 / 16, c5=1 / 64, c7=1 / 384, cL=-1 / 16, cN=-1 / 24)  # asqtad-type
# one smearing level: 50 products of 3x3 complex matrices per site and direction (27 complex
# multiply-adds = 216 flops each); linear combinations are not counted
SMEAR_FLOPS_PER_SITE = 4 * 50 * 216


def _stream_ms(torch, stream, fn, reps):
    fn()  # workspaces
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def row_smear(h, torch, hin):
    """48^3x12 link smearing: one level with every path kind and the Naik product in FP64 and in
    double-float arithmetic, the U(3) projection, the two HISQ levels, and the oracle on sampled sites."""
    from oracle import smear as sm
    L = (48, 48, 48, 12)
    V = int(np.prod(L))
    Uh = hin.gen_thin(L, GAUGE_SEED, 0.3).reshape(V, 4, 3, 3)
    stream = torch.cuda.Stream()
    lat = h.Lattice(L, precs=(h.HISQ_F64,), stream=stream)
    U = torch.from_numpy(Uh).cuda()
    fat, lng = torch.empty_like(U), torch.empty_like(U)
    torch.cuda.synchronize()
    lname = "x".join(map(str, L))
    gpu_sites = {}
    for prec, name in ((h.HISQ_F64, "f64"), (h.HISQ_DF64, "df64")):
        ms = _stream_ms(torch, stream, lambda: lat.smear(fat, lng, U, SMEAR_LEVEL2, prec), 3)
        gf = SMEAR_FLOPS_PER_SITE * V / (ms * 1e-3) / 1e9
        line = {"row": "smear", "lattice": lname, "arith": name, "what": "one level, all paths + Naik",
                "ms": round(ms, 3), "GFLOP/s": round(gf, 1), "sites_per_s": round(V / (ms * 1e-3), 1)}
        if prec == h.HISQ_F64:
            line["frac_fp64_pipe"] = round(gf / (FP64_PIPE_TFLOPS * 1e3), 3)
        gpu_sites[name] = V / (ms * 1e-3)
        print(json.dumps(line), flush=True)
        ms = _stream_ms(torch, stream, lambda: lat.hisq_links(fat, lng, U, SMEAR_LEVEL1, SMEAR_LEVEL2, prec), 3)
        print(json.dumps({"row": "smear", "lattice": lname, "arith": name,
                          "what": "two HISQ levels (level 1, U(3) projection, level 2 + Naik)",
                          "ms": round(ms, 3)}), flush=True)
    ms = _stream_ms(torch, stream, lambda: h.hisq_project_u3(lat.ctx, fat, U), 5)
    by = 2 * V * 4 * 144
    print(json.dumps({"row": "smear", "lattice": lname, "what": "U(3) projection (FP64)", "ms": round(ms, 3),
                      "GB/s": round(by / (ms * 1e-3) / 1e9, 1)}), flush=True)
    # one level at the other sizes of the Dslash sweep that fit (inputs, outputs and workspaces take
    # 3 x 576 + 144 x 16 B per site: 96^3x24 needs 86 GB, 144^3x36 would need 433 GB)
    del lat, U, fat, lng
    torch.cuda.empty_cache()
    for Ls in ((32, 32, 32, 8), (64, 64, 64, 16), (96, 96, 96, 24)):
        Vs = int(np.prod(Ls))
        lat_s = h.Lattice(Ls, precs=(h.HISQ_F64,), stream=stream)
        Us = torch.from_numpy(hin.gen_thin(Ls, GAUGE_SEED, 0.3).reshape(Vs, 4, 3, 3)).cuda()
        fs, ls = torch.empty_like(Us), torch.empty_like(Us)
        torch.cuda.synchronize()
        for prec, name in ((h.HISQ_F64, "f64"), (h.HISQ_DF64, "df64")):
            ms = _stream_ms(torch, stream, lambda: lat_s.smear(fs, ls, Us, SMEAR_LEVEL2, prec), 2)
            gf = SMEAR_FLOPS_PER_SITE * Vs / (ms * 1e-3) / 1e9
            line = {"row": "smear", "lattice": "x".join(map(str, Ls)), "arith": name,
                    "what": "one level, all paths + Naik", "ms": round(ms, 3), "GFLOP/s": round(gf, 1),
                    "sites_per_s": round(Vs / (ms * 1e-3), 1)}
            if prec == h.HISQ_F64:
                line["frac_fp64_pipe"] = round(gf / (FP64_PIPE_TFLOPS * 1e3), 3)
            print(json.dumps(line), flush=True)
        del lat_s, Us, fs, ls
        torch.cuda.empty_cache()
    # the oracle (numpy, explicit path sums) on a sample of sites
    n = 2048
    sample = np.random.default_rng(3).choice(V, n, replace=False)
    t0 = time.perf_counter()
    sm.smear(L, Uh, **SMEAR_LEVEL2, sites=sample)
    dt = time.perf_counter() - t0
    print(json.dumps({"row": "smear", "lattice": lname, "what": "oracle, one level on %d sampled sites" % n,
                      "s": round(dt, 3), "sites_per_s": round(n / dt, 1),
                      "gpu_over_oracle": {k: round(v / (n / dt), 1) for k, v in gpu_sites.items()}}), flush=True)


def run_row(name):
    import torch

    import __graft_entry__
    import hisq_inputs as hin
    __graft_entry__.build()
    import paper_2111_10354_gb300 as h
    {"multirhs": row_multirhs, "multishift": row_multishift, "batch": row_batch,
     "learned": row_learned, "smear": row_smear}[name](h, torch, hin)


def run_kernel_case(name):
    """A handful of launches of one kernel on a modest case (inputs larger than L2), for ncu."""
    import torch

    import __graft_entry__
    import hisq_inputs as hin
    __graft_entry__.build()
    import paper_2111_10354_gb300 as h
    stream = torch.cuda.Stream()
    if name in ("dslash-f32-48", "dslash-f32-96", "dslash-f32-144"):
        # the FP32 Dslash on 48^3x12, 96^3x24 and 144^3x36 (FP64 + FP32 links resident, loaded slab by
        # slab): the tuner's choice, then each site order (cb order, the tiled walk) forced with the tuned
        # block size, for the DRAM traffic of launches whose input vector exceeds L2
        e = int(name.rsplit("-", 1)[1])
        L = (e, e, e, e // 4)
        lat = h.Lattice(L, precs=(h.HISQ_F64, h.HISQ_F32), stream=stream)
        nt = max(1, min(L[3], int(2e8 // (L[0] * L[1] * L[2] * 4 * 9 * 16))))
        for t0 in range(0, L[3], nt):
            n = min(nt, L[3] - t0)
            fat, lng = hin.gen_links(L, GAUGE_SEED, 0.3, 0.1, t0=t0, nt=n)
            h.hisq_load_links_slab(lat.ctx, t0, n, fat, lng)
        dims = "x".join(map(str, L))
        key = "dslash/l%d/s%d/nr1/e0/c0" % (h.HISQ_F32, h.HISQ_F32)
        ms = time_dslash(torch, lat, h.HISQ_F32, 1, 4, stream)
        tuned = [t for t in h.hisq_tune_report(lat.ctx).splitlines() if t.startswith(key + " ")][0]
        choice = int(tuned.rsplit(" ", 1)[1])
        out = {"case": name, "tuned": tuned, "us_tuned": round(ms * 1e3, 2), "bytes": lat.dslash_bytes(h.HISQ_F32, 1)}
        for vi, pol in ((0, "cb_order"), (1, "tiled_walk")):
            h.hisq_tune_load(lat.ctx, "%s %s -> %d\n" % (key, dims, vi * 10000 + choice % 10000))
            out["us_" + pol] = round(time_dslash(torch, lat, h.HISQ_F32, 1, 4, stream) * 1e3, 2)
        print(json.dumps(out))
    elif name.startswith("dslash"):
        L = (48, 48, 48, 12)
        fat, lng = hin.gen_links(L, 1001, 0.3, 0.1)
        lat = h.Lattice(L, precs=(h.HISQ_F64, h.HISQ_F32, h.HISQ_F16) + ((h.HISQ_DF64,) if name == "dslash-df64" else ()),
                        stream=stream)
        if name == "dslash-f32-comp":
            lat.compress_long(-1.0 / 24.0)
        lat.load(fat, lng)
        prec = {"dslash-f64": h.HISQ_F64, "dslash-df64": h.HISQ_DF64, "dslash-f16": h.HISQ_F16,
                "dslash-f32-comp": h.HISQ_F32, "dslash-f32-nr8": h.HISQ_F32, "dslash-f16-il64-tc": h.HISQ_F16,
                "dslash-f32-il8": h.HISQ_F32, "dslash-f32-il16": h.HISQ_F32,
                }[name]
        nrhs = 8 if name.endswith(("nr8", "il8")) else (16 if name.endswith("il16") else (64 if "il64" in name else 1))
        if name.endswith("-tc"):  # the tcgen05 tensor-core form, forced
            h.hisq_tune_load(lat.ctx, "dslash_path_il/l%d/n%d 48x48x48x12 -> 2\n" % (prec, nrhs))
        ms = time_dslash(torch, lat, prec, nrhs, 4, stream, interleaved="-il" in name)
        print(json.dumps({"case": name, "us": round(ms * 1e3, 2)}))
    elif name == "cg-f32-nr8":
        L = (48, 48, 48, 12)
        fat, lng = hin.gen_links(L, 1002, 0.3, 0.1)
        lat = h.Lattice(L, precs=(h.HISQ_F64, h.HISQ_F32), stream=stream).load(fat, lng)
        b = torch.from_numpy(hin.gen_source(2002, lat.half, 8)).cuda()
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        for _ in range(2):  # the first solve tunes and captures, the second replays
            x.zero_()
            torch.cuda.synchronize()
            rc, st = lat.cg(x, b, 0.01, 1e-10, 5000, nrhs=8, inner_prec=h.HISQ_F32)
        print(json.dumps({"case": name, "iters": st["iters"], "s": round(st["seconds"], 4)}))
    elif name in ("cg-f32", "multishift"):
        L = (48, 48, 48, 12)
        fat, lng = hin.gen_links(L, 1001 if name == "cg-f32" else 1002, 0.3, 0.1)
        lat = h.Lattice(L, precs=(h.HISQ_F64, h.HISQ_F32), stream=stream).load(fat, lng)
        b = torch.from_numpy(hin.gen_source(2001 if name == "cg-f32" else 2002, lat.half, 1)).cuda()
        torch.cuda.synchronize()
        for _ in range(2):  # the first solve tunes and captures, the second replays
            if name == "cg-f32":
                x = torch.zeros_like(b)
                torch.cuda.synchronize()
                rc, st = lat.cg(x, b, 0.01, 1e-10, 5000, inner_prec=h.HISQ_F32)
            else:
                shifts = np.logspace(-5, 0, 14)
                x = torch.zeros((14,) + tuple(b.shape[1:]), dtype=b.dtype, device="cuda")
                torch.cuda.synchronize()
                rc, st = lat.multishift_cg(x, b, shifts, 0.0025, 1e-9, 5000, inner_prec=h.HISQ_F32)
        print(json.dumps({"case": name, "iters": st["iters"], "s": round(st["seconds"], 4)}))
    elif name == "ptc":
        import oracle.ptc as optc
        L = (32, 32, 32, 8)
        fat, lng = hin.gen_links(L, 4000, 0.35, 0.1)
        lat = h.Lattice(L, precs=(h.HISQ_F64, h.HISQ_F32), stream=stream).load(fat, lng)
        net = h.Ptc(lat)
        W1, _ = optc.init_weights(4000, scale=0.05)
        net.set_tied(True)
        net.set_weights(W1, optc.tie(W1))
        r = torch.from_numpy(hin.gen_source(1, lat.half, 1)).to(torch.complex64).cuda()
        z = torch.empty_like(r)
        torch.cuda.synchronize()  # r comes from torch's stream, the network runs on the library's
        for _ in range(4):
            net.apply(z, r, 1)
        torch.cuda.synchronize()
        print(json.dumps({"case": name, "ok": True}))
    elif name == "fcg":
        # flexible CG with the (untrained, tied) PTC preconditioner: the launch mix of one solve
        import oracle.ptc as optc
        L = (32, 32, 32, 8)
        fat, lng = hin.gen_links(L, 4100, 0.35, 0.1)
        lat = h.Lattice(L, precs=(h.HISQ_F64, h.HISQ_F32), stream=stream).load(fat, lng)
        net = h.Ptc(lat)
        W1, _ = optc.init_weights(4000, scale=0.05)
        net.set_tied(True)
        net.set_weights(W1, optc.tie(W1))
        b = torch.from_numpy(hin.gen_source(6000, lat.half, 1)).cuda()
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        for _ in range(2):
            x.zero_()
            torch.cuda.synchronize()
            rc, st = h.hisq_fcg(lat.ctx, net.h, x, b, 0.001, 1e-10, 400, h.make_opts(), raise_on_error=False)
        print(json.dumps({"case": name, "status": rc, "iters": st["iters"], "s": round(st["seconds"], 4)}))
    elif name.startswith("smear"):
        L = (32, 32, 32, 8)
        V = int(np.prod(L))
        lat = h.Lattice(L, precs=(h.HISQ_F64,), stream=stream)
        U = torch.from_numpy(hin.gen_thin(L, GAUGE_SEED, 0.3).reshape(V, 4, 3, 3)).cuda()
        fat, lng = torch.empty_like(U), torch.empty_like(U)
        torch.cuda.synchronize()
        prec = h.HISQ_DF64 if name == "smear-df64" else h.HISQ_F64
        ms = _stream_ms(torch, stream, lambda: lat.smear(fat, lng, U, SMEAR_LEVEL2, prec), 1)
        print(json.dumps({"case": name, "ms": round(ms, 3)}))
    elif name == "batch":
        mix = hin.lattice_mix_64()[:16] + hin.lattice_mix_64()[32:40] + hin.lattice_mix_64()[51:55]
        batch = h.Batch([m["dims"] for m in mix], stream=stream)
        bs = []
        for l, m in enumerate(mix):
            fat, lng = hin.gen_links(m["dims"], m["gauge_seed"], m["eps"], 0.1)
            batch.load(l, fat, lng)
            bs.append(hin.gen_source(m["source_seed"], int(np.prod(m["dims"])) // 2, 1)[0])
        b = torch.from_numpy(np.concatenate([v.reshape(-1) for v in bs]).reshape(-1, 3)).cuda()
        x = torch.zeros_like(b)
        torch.cuda.synchronize()  # inputs come from torch's stream, the solve runs on the library's
        rc, st = batch.cg(x, b, [m["mass"] for m in mix], 1e-10, 10000, inner_prec=h.HISQ_F32)
        print(json.dumps({"case": name, "iters": st["iters"]}))


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.sweep:
        run_sweep()
        return
    if args.row:
        run_row(args.row)
        return
    if args.kernel_case:
        run_kernel_case(args.kernel_case)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
