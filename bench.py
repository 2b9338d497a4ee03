#!/usr/bin/env python
"""Benchmark of the sparse MTTKRP / CP-ALS hot path on GB300.

One *step* is one pass of the whole hot path over the workload: one CP-ALS
iteration (every mode: MTTKRP, Gram-Hadamard FP64 Cholesky solve, column
normalisation, then the fit) when the library has it, else the MTTKRP of
every mode.  The default workload is the 3-way power-law tensor
1,000,000 x 500,000 x 200,000 with 1e8 nonzeros (Zipf s=1.2 per mode),
rank 16, fp32 N(0,1) factors.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "MTTKRP nnz·R/s and % GB300 HBM peak (BF16 vs FP32 factors); CP-ALS iter/s"
UNIT = "nnz*R/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="zipf3d_1e6x5e5x2e5_nnz1e8")
    ap.add_argument("--dtype", default=None, help="factor storage (default: the workload's)")
    ap.add_argument("--scatter", default="sorted", choices=["atomic", "perm", "sorted"])
    ap.add_argument("--scale", type=float, default=1.0, help="shrink the workload (debug only)")
    ap.add_argument("--cpu-sample", type=int, default=4_000_000,
                    help="nonzeros of the oracle's bounded CPU sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--step-kind", default="auto", choices=["auto", "mttkrp", "cpals"])
    return ap.parse_args()


# ---------------------------------------------------------------- helpers
def algorithmic_bytes(scatter, P, d, R, s_f, I_n, W):
    """Bytes one mode-n MTTKRP must move (cache hits not deducted):
    value (4) + d coordinates (4 each) + d-1 gathered factor rows (R*s_f each)
    per nonzero, plus the output rows (R*4); the permuted traversal through
    perm_n adds 4 bytes per nonzero, the atomic scatter adds R*4 per nonzero
    (one read-modify-write per nonzero instead of one write per row)."""
    per = 4 + 4 * d + (d - 1) * R * s_f
    if scatter == "perm":
        per += 4
    if scatter == "atomic":
        per += R * 4
        return P * per + I_n * R * 4
    return P * per + W * R * 4 + I_n * R * 4


def compulsory_bytes(P, d, dims, n, R, s_f):
    """Every input byte read once and the output written once."""
    return P * (4 + 4 * d) + sum(dims[m] * R * s_f for m in range(d) if m != n) + dims[n] * R * 4


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during timing."""

    def __init__(self, dev_index: int):
        self.dev = dev_index
        self.proc = None
        self.lines = []

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def cpu_baseline(w, idx, vals, facs_np, dtype, R, sample):
    """The FP64 oracle as it stands, on the first `sample` nonzeros, every mode."""
    import oracle
    P_s = min(sample, idx.shape[1])
    si = np.ascontiguousarray(idx[:, :P_s])
    sv = vals[:P_s]
    A = [oracle.as_f64(f, dtype)[:, :R].copy() for f in facs_np]
    t0 = time.perf_counter()
    for n in range(len(w.dims)):
        oracle.mttkrp(si, sv, w.dims, A, n, R)
    dt = time.perf_counter() - t0
    return {"value": P_s * R * len(w.dims) / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {P_s} of {idx.shape[1]} nonzeros, MTTKRP of all {len(w.dims)} modes, "
                      f"FP64, single thread, {dt:.1f} s"}


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import synth
    w = synth.workload(args.workload, args.scale)
    dtype = args.dtype or w.factor_dtype
    R = w.R
    idx, vals = w.coo()
    facs = w.factors(R, dtype)
    import oracle
    A = [oracle.as_f64(f, dtype)[:, :R].copy() for f in facs]
    P_s = min(args.cpu_sample, idx.shape[1])
    si = np.ascontiguousarray(idx[:, :P_s])
    sv = vals[:P_s]
    times = []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for n in range(len(w.dims)):
            oracle.mttkrp(si, sv, w.dims, A, n, R)
        if it >= args.warmup:
            times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    v = P_s * R * len(w.dims) / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "R": R, "factors": dtype},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"first {P_s} nonzeros per step, MTTKRP of every mode"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_1809_09175_gb300 as P
    import synth

    w = synth.workload(args.workload, args.scale)
    if world > 1:  # independent problem per rank (weak scaling)
        w = synth.Workload(w.name, w.dims, w.nnz, w.s, w.R, w.factor_dist, w.seed + rank,
                           w.factor_dtype)
    dtype = args.dtype or w.factor_dtype
    R = w.R
    d = len(w.dims)
    ld = P.factor_ld(R)
    s_f = 4 if dtype == "f32" else 2
    idx, vals = w.coo()
    facs_np = w.factors(R, dtype)

    stream = torch.cuda.current_stream()
    t_ing = time.perf_counter()
    T = P.SparseTensor(idx, vals, w.dims)
    T.build_permutation(-1, index_only=(args.scatter == "perm"))
    torch.cuda.synchronize()
    ingest_s = time.perf_counter() - t_ing

    def dev_factor(f):
        if dtype == "f32":
            return torch.from_numpy(f).cuda()
        return torch.from_numpy(f.view(np.int16)).cuda().view(
            torch.bfloat16 if dtype == "bf16" else torch.float16)

    facs = [dev_factor(f) for f in facs_np]
    outs = [torch.empty((I, ld), dtype=torch.float32, device="cuda") for I in w.dims]
    scheds = []
    for n in range(d):
        s = P.mttkrp_default_schedule(T.handle, n, dtype, R)
        s.scatter = P.SCATTERS[args.scatter]
        scheds.append(s)

    has_cpals = hasattr(P.binding.lib(), "cp_als_step")
    kind = args.step_kind
    if kind == "auto":
        kind = "cpals" if has_cpals else "mttkrp"

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(d)]
    kern_ms = []

    def mttkrp_step(record):
        for n in range(d):
            if record:
                ev[n][0].record(stream)
            T.mttkrp(n, facs, R, out=outs[n], sched=scheds[n])
            if record:
                ev[n][1].record(stream)

    step = mttkrp_step
    launches_per_step = d

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    per_mode = [0.0] * d
    for _ in range(args.steps):
        step(True)
        torch.cuda.synchronize()
        for n in range(d):
            per_mode[n] += ev[n][0].elapsed_time(ev[n][1])
    t1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    T.check()
    total_ms = t0.elapsed_time(t1)
    if world > 1:
        tt = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
        dist.barrier()
    ms_step = total_ms / args.steps
    units = w.nnz * R * d  # nonzeros x rank per mode, every mode
    value = units * world / (ms_step / 1e3)

    # roofline of the dominant kernel (the MTTKRP launch), per mode averaged
    stats = []
    hbm_peak, peak_kind = measured_peaks()
    alg = 0.0
    comp = 0.0
    for n in range(d):
        W = w.dims[n]
        alg += algorithmic_bytes(args.scatter, w.nnz, d, R, s_f, w.dims[n], W)
        comp += compulsory_bytes(w.nnz, d, w.dims, n, R, s_f)
    mode_ms = [x / args.steps for x in per_mode]
    launch_ms = sum(mode_ms) / d
    achieved = (alg / d) / (launch_ms / 1e3) / 1e9
    comp_gbs = (comp / d) / (launch_ms / 1e3) / 1e9

    # end to end through the public API: factors H2D from pinned memory, the
    # step, results D2H, every step
    e2e = None
    if rank == 0 or world > 1:
        pin_f = [torch.from_numpy(f.view(np.int16) if dtype != "f32" else f).pin_memory() for f in facs_np]
        pin_o = [torch.empty(o.shape, dtype=o.dtype).pin_memory() for o in outs]
        h2d = sum(p.numel() * p.element_size() for p in pin_f)
        d2h = sum(p.numel() * p.element_size() for p in pin_o)
        torch.cuda.synchronize()
        e0 = time.perf_counter()
        for _ in range(args.steps):
            for f, p in zip(facs, pin_f):
                f.view(p.dtype).copy_(p, non_blocking=True)
            step(False)
            for o, p in zip(outs, pin_o):
                p.copy_(o, non_blocking=True)
            torch.cuda.synchronize()
        e_s = (time.perf_counter() - e0) / args.steps
        e2e = {"value": units / e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(w, idx, vals, facs_np, dtype, R, args.cpu_sample)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32-accumulate/" + dtype + "-factors",
        "data": "synthetic",
        "config": {"workload": w.name, "dims": w.dims, "nnz": w.nnz, "zipf_s": w.s, "R": R,
                   "factors": dtype, "factor_dist": w.factor_dist, "scatter": args.scatter,
                   "step": kind, "l2": "inputs larger than L2 (COO stream "
                   f"{w.nnz * 4 * (d + 1) / 1e9:.1f} GB per mode)"},
        "per_mode_ms": mode_ms,
        "per_mode_nnzR_per_s": [w.nnz * R / (m / 1e3) for m in mode_ms],
        "roofline": {"bound": "hbm", "kernel": "mttkrp_kernel", "achieved": achieved,
                     "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                     "peak_kind": peak_kind, "traffic": None,
                     "compulsory_GBps": comp_gbs, "compulsory_frac": comp_gbs / hbm_peak},
        "gpu_launches": launches_per_step * args.steps,
        "ingest_s": ingest_s,
        "clocks": clk,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    T.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
