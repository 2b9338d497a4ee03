#!/usr/bin/env python
"""Benchmark of the sparse MTTKRP / CP-ALS hot path on GB300.

One timed *step* is the MTTKRP of every mode of the workload (one kernel
launch per mode, the permuted traversal over mode-sorted copies by default).
The default workload is the 3-way power-law tensor 1,000,000 x 500,000 x
200,000 with 1e8 nonzeros (Zipf s=1.2 per mode, duplicates kept), rank 16,
fp32 N(0,1) factors.  After the timed region the line also reports the other
scatter strategies and bf16 factors on the same tensor, sampled-row errors
against the FP64 oracle, and CP-ALS iterations (captured CUDA graph) on the
coalesced tensor.

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
    ap.add_argument("--scatter", default="sorted", choices=["atomic", "perm", "sorted", "private"])
    ap.add_argument("--sched", default="tuned", choices=["default", "tuned"],
                    help="per-mode schedule: the library's exhaustive autotuner (set-up, untimed) "
                         "or its default rule")
    ap.add_argument("--npg", type=int, default=0, help="override the schedule's nonzeros per lane group")
    ap.add_argument("--scale", type=float, default=1.0, help="shrink the workload (debug only)")
    ap.add_argument("--cpu-sample", type=int, default=32_000_000,
                    help="nonzeros of the oracle's bounded CPU sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="skip the variants / CP-ALS extras")
    ap.add_argument("--slice-order", type=int, default=1,
                    help="1: build the mode-sorted copies with each slice ordered by the next modes")
    ap.add_argument("--l2-blocks", choices=["auto", "off"], default="auto",
                    help="auto: give a mode an L2-blocked copy where its largest other factor exceeds "
                         "twice --l2-block-mb (blocks of that many MB of the factor's rows)")
    ap.add_argument("--l2-block-mb", type=float, default=48.0)
    ap.add_argument("--full-parity-s", type=float, default=120.0,
                    help="whole-output parity against the all-core oracle when its estimated time "
                         "is within this many seconds (0: off)")
    ap.add_argument("--rank", type=int, default=0, help="override the workload's rank")
    ap.add_argument("--batched", type=int, default=0,
                    help="instead: the N-tensor batch, every mode in one persistent launch")
    ap.add_argument("--cpals", type=int, default=0,
                    help="instead: N CP-ALS iterations of the workload under the learned selector, "
                         "exhaustive autotune, default and paper schedules")
    ap.add_argument("--paper-sweep", action="store_true",
                    help="instead: the paper's 30K x 40K x 50K / 1e7-nonzero tensor, MTTKRP for R = 8..256 "
                         "step 8 with fp64, fp32 and bf16 factors, and 10 CP-ALS iterations at R = 128")
    ap.add_argument("--sweep-ranks", default="8:257:8", help="start:stop:step of the rank sweep")
    ap.add_argument("--shard-cpals", type=int, default=0,
                    help="time this many CP-ALS iterations with the nonzeros split across the ranks (NCCL)")
    ap.add_argument("--gather-probe", type=float, default=0,
                    help="time factor-row gathers for this many nonzeros (loads vs TMA) and exit")
    ap.add_argument("--weights", default=os.path.join(ROOT, "paper_1809_09175_gb300",
                                                       "selector_weights.npz"))
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


def l2_block_plan(args, dims, ld, s_f):
    """{mode: rows per block} for the modes whose largest other factor is
    more than twice the block budget (--l2-blocks auto)."""
    if args.l2_blocks == "off":
        return {}
    budget = args.l2_block_mb * 2 ** 20
    plan = {}
    for n in range(len(dims)):
        m = max((k for k in range(len(dims)) if k != n), key=lambda k: dims[k])
        if dims[m] * ld * s_f > 2 * budget:
            plan[n] = max(1, int(budget // (ld * s_f)))
    return plan


def build_l2_blocks(T, plan):
    for n, rows in plan.items():
        T.build_l2_blocks(n, -1, rows)
    return {str(n): list(T.l2_blocks(n)) for n in plan}


def kernel_traffic(nnz):
    """DRAM bytes per MTTKRP launch from the committed ncu capture, scaled to
    `nnz` nonzeros (the 16-byte nonzero record is ~3/4 of the traffic and
    grows with nnz), or None when the kernel sources changed since."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic_mttkrp_kernel_sorted_zipf3d_2e7nnz_R16.txt")
    if not os.path.exists(p):
        return None
    kv = {}
    for ln in open(p):
        if ":" in ln and not ln.startswith("#"):
            k, v = ln.split(":", 1)
            kv[k.strip()] = v.strip()
    h = hashlib.sha256()
    for f in ("mttkrp_kernel.cuh", "common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1809_09175_gb300", "csrc", f), "rb").read())
    if kv.get("kernel_source_sha256") != h.hexdigest():
        return None
    return float(kv["bytes_per_nonzero"]) * nnz


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def host_threads():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(w, idx, vals, facs_np, dtype, R, sample):
    """The FP64 oracle as it stands, on the first `sample` nonzeros, every
    mode: its all-core form (each host thread owns a range of output rows and
    walks every nonzero in storage order) as the baseline, the serial
    definition beside it."""
    import oracle
    P_s = min(sample, idx.shape[1])
    si = np.ascontiguousarray(idx[:, :P_s])
    sv = vals[:P_s]
    A = [oracle.as_f64(f, dtype)[:, :R].copy() for f in facs_np]
    T = host_threads()
    t0 = time.perf_counter()
    for n in range(len(w.dims)):
        oracle.mttkrp(si, sv, w.dims, A, n, R)
    dt1 = time.perf_counter() - t0
    t0 = time.perf_counter()
    for n in range(len(w.dims)):
        oracle.mttkrp_threads(si, sv, w.dims, A, n, R, T)
    dt = time.perf_counter() - t0
    units = P_s * R * len(w.dims)
    return {"value": units / dt, "unit": UNIT, "cores": T, "kind": "oracle",
            "sample": f"first {P_s} of {idx.shape[1]} nonzeros, MTTKRP of all {len(w.dims)} modes, "
                      f"FP64, {T} host threads, {dt:.1f} s",
            "single_thread": {"value": units / dt1, "unit": UNIT, "cores": 1, "seconds": dt1}}


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
    T = host_threads()
    times = []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for n in range(len(w.dims)):
            oracle.mttkrp_threads(si, sv, w.dims, A, n, R, T)
        if it >= args.warmup:
            times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    v = P_s * R * len(w.dims) / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "R": R, "factors": dtype},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": T, "kind": "oracle",
                             "sample": f"first {P_s} nonzeros per step, MTTKRP of every mode, "
                                       f"FP64, {T} host threads"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
def _dev_factor(torch, f, dtype):
    if dtype == "f32":
        return torch.from_numpy(f).cuda()
    return torch.from_numpy(f.view(np.int16)).cuda().view(
        torch.bfloat16 if dtype == "bf16" else torch.float16)


def sampled_rows(w, idx, n, R, count=24, seed=0):
    """Hottest rows of mode n plus uniformly drawn ones (oracle-checkable)."""
    cnt = np.bincount(idx[n], minlength=w.dims[n])
    hot = np.argsort(cnt)[::-1][: count // 2]
    rnd = np.random.default_rng(seed).integers(0, w.dims[n], count - hot.shape[0])
    return np.unique(np.concatenate([hot, rnd])).astype(np.int32)


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
    if args.rank:
        w = synth.Workload(w.name, w.dims, w.nnz, w.s, args.rank, w.factor_dist, w.seed, w.factor_dtype)
    from paper_1809_09175_gb300 import multi
    if world > 1:  # an independent problem per rank (weak scaling, no data-path collective)
        w = synth.Workload(w.name, w.dims, w.nnz, w.s, w.R, w.factor_dist,
                           multi.rank_seed(w.seed, rank), w.factor_dtype)
    dtype = args.dtype or w.factor_dtype
    R = w.R
    d = len(w.dims)
    ld = P.factor_ld(R)
    s_f = 4 if dtype == "f32" else 2
    idx, vals = w.coo()
    facs_np = w.factors(R, dtype)

    stream = torch.cuda.current_stream()
    sid = stream.cuda_stream
    t_ing = time.perf_counter()
    T = P.SparseTensor(idx, vals, w.dims)
    torch.cuda.synchronize()
    t_perm = time.perf_counter()
    T.build_permutation(-1, index_only=(args.scatter == "perm"), slice_order=bool(args.slice_order))
    plan = l2_block_plan(args, w.dims, ld, s_f) if args.scatter == "sorted" else {}
    l2_blocks = build_l2_blocks(T, plan)
    torch.cuda.synchronize()
    t_done = time.perf_counter()
    ingest_s, perm_s = t_perm - t_ing, t_done - t_perm

    facs = [_dev_factor(torch, f, dtype) for f in facs_np]
    outs = [torch.empty((I, ld), dtype=torch.float32, device="cuda") for I in w.dims]

    def sched_for(n, scatter, fdt):
        s = P.mttkrp_default_schedule(T.handle, n, fdt, R)
        s.scatter = P.SCATTERS[scatter]
        if args.npg:
            s.nnz_per_group = args.npg
        return s

    scheds = [sched_for(n, args.scatter, dtype) for n in range(d)]
    tune_s = None
    if args.sched == "tuned":  # the library's exhaustive autotuner, before the timed region
        t0 = time.perf_counter()
        for n in range(d):
            best, _, _ = P.mttkrp_autotune(T.handle, n, [f.data_ptr() for f in facs], dtype, R,
                                           ld, outs[n].data_ptr(), 2, sid)
            scheds[n] = best
        tune_s = time.perf_counter() - t0
    # one event pair per launch of the timed region (steps x modes)
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(d)] for _ in range(args.steps)]

    def step(k=None):
        for n in range(d):
            if k is not None:
                ev[k][n][0].record(stream)
            T.mttkrp(n, facs, R, out=outs[n], sched=scheds[n])
            if k is not None:
                ev[k][n][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed launches (ncu --nvtx-include timed/)
    t0.record(stream)
    for k in range(args.steps):
        step(k)
    t1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clk = clocks.stop()
    T.check()
    local_ms = t0.elapsed_time(t1)
    units = w.nnz * R * d  # per step, this rank
    # slowest rank's time, all ranks' units (timing reductions only)
    total_ms, all_units = multi.reduce_timing(local_ms, units * args.steps, device="cuda")
    if world > 1:
        dist.barrier()
    ms_step = total_ms / args.steps
    value = all_units / (total_ms / 1e3)
    mode_ms = [sum(ev[k][n][0].elapsed_time(ev[k][n][1]) for k in range(args.steps)) / args.steps
               for n in range(d)]

    hbm_peak, peak_kind = measured_peaks()
    # W (rows written) is bounded by I_n; the bound is used
    alg = sum(algorithmic_bytes(args.scatter, w.nnz, d, R, s_f, w.dims[n], w.dims[n])
              for n in range(d))
    comp = sum(compulsory_bytes(w.nnz, d, w.dims, n, R, s_f) for n in range(d))
    launch_ms = sum(mode_ms) / d
    alg_gbs = (alg / d) / (launch_ms / 1e3) / 1e9
    comp_gbs = (comp / d) / (launch_ms / 1e3) / 1e9
    # the fraction of HBM the kernel uses: DRAM bytes of one launch measured by
    # ncu (the committed record, scaled by nonzeros, while the kernel sources
    # match it) over the mean launch time of the timed region; without a
    # current record, the compulsory bytes (a lower bound) stand in
    traffic = (kernel_traffic(w.nnz) if args.scatter == "sorted" and dtype == "f32" and R == 16 and d == 3
               else None)
    dram_gbs = traffic / (launch_ms / 1e3) / 1e9 if traffic else comp_gbs
    roofline = {"bound": "hbm", "kernel": "mttkrp_kernel", "achieved": dram_gbs, "peak": hbm_peak,
                "unit": "GB/s", "frac": dram_gbs / hbm_peak, "peak_kind": peak_kind,
                "achieved_basis": ("ncu DRAM read+write bytes per launch / mean launch time" if traffic else
                                   "compulsory bytes per launch / mean launch time (no current ncu record)"),
                "traffic": traffic, "launch_ms": launch_ms,
                "algorithmic_bytes_per_launch": alg / d, "algorithmic_GBps": alg_gbs,
                "algorithmic_frac": alg_gbs / hbm_peak,
                "compulsory_bytes_per_launch": comp / d, "compulsory_GBps": comp_gbs,
                "compulsory_frac": comp_gbs / hbm_peak}

    # the metric's per-mode form: P R / t_mode with t_mode the median of 20
    # CUDA-graph replays of that mode's launch (after 3), beside the timed
    # region's whole-step figure
    graph_mode_ms = None
    try:
        graph_mode_ms = []
        for n in range(d):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, capture_error_mode="thread_local"):
                T.mttkrp(n, facs, R, out=outs[n], sched=scheds[n])
            for _ in range(3):
                g.replay()
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(20)]
            for a_, b_ in evs:
                a_.record(stream)
                g.replay()
                b_.record(stream)
            torch.cuda.synchronize()
            graph_mode_ms.append(statistics.median(a_.elapsed_time(b_) for a_, b_ in evs))
            del g
    except Exception as ex:  # reported, never fatal: the timed region above is the number
        graph_mode_ms = f"unavailable: {type(ex).__name__}: {ex}"[:200]
    T.check()

    # end to end through the public API: one mttkrp_from_host call per step
    # uploads the factors from pinned host memory, runs every mode's MTTKRP
    # (the timed region's schedules, recorded on the tensor) and downloads
    # every output, the copies overlapped with the kernels; the step ends
    # with the stream synchronised and the results in host memory
    ws = None
    try:
        tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[dtype]
        pin_f = [torch.from_numpy(f.view(np.int16) if dtype != "f32" else f).view(tdt).pin_memory()
                 for f in facs_np]
        pin_o = [torch.empty(o.shape, dtype=o.dtype).pin_memory() for o in outs]
        h2d = sum(p.numel() * p.element_size() for p in pin_f)
        d2h = sum(p.numel() * p.element_size() for p in pin_o)
        for n in range(d):
            P.tensor_set_schedule(T.handle, n, dtype, R, scheds[n])
        ws = torch.empty(P.mttkrp_from_host_workspace_size(T.handle, list(range(d)), dtype, R, ld),
                         dtype=torch.uint8, device="cuda")
        T.mttkrp_from_host(list(range(d)), pin_f, R, outs=pin_o, workspace=ws)  # warm-up
        torch.cuda.synchronize()
        e0 = time.perf_counter()
        for _ in range(args.steps):
            T.mttkrp_from_host(list(range(d)), pin_f, R, outs=pin_o, workspace=ws)
        e_s = (time.perf_counter() - e0) / args.steps
        e2e = {"value": units / e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
    except P.SptError as ex:  # reported, never fatal: the device-timed line stands
        e2e = {"value": None, "unit": UNIT, "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
               "error": str(ex)[:300]}
    finally:
        # a failed call still orders the stream after its queued copies: wait
        # for them before the workspace goes back to torch's allocator
        torch.cuda.current_stream().synchronize()
        del ws
        for n in range(d):  # the variants below pass their own schedules or take the default rule
            P.tensor_set_schedule(T.handle, n, dtype, R, None)

    extra = {}
    if rank == 0 and not args.quick:
        try:
            extra = measure_extras(args, P, torch, w, T, idx, vals, facs_np, dtype, R, d, ld, outs,
                                   sched_for, mode_ms)
        except Exception as ex:  # the headline above stands; say what the extras hit
            extra = {"extras_error": f"{type(ex).__name__}: {ex}"[:300]}
        # whole-output parity when the oracle's share of it fits the budget
        est_s = w.nnz * R * d * 2 / 6e8 * (16 / max(1, host_threads()))
        if args.full_parity_s > 0 and est_s <= args.full_parity_s:
            try:
                extra["full_parity"] = full_parity(args, P, torch, w, T, idx, vals, R, d, outs, sched_for)
            except Exception as ex:
                extra["full_parity"] = {"error": f"{type(ex).__name__}: {ex}"[:300]}
        else:
            extra["full_parity"] = {"skipped": f"estimated oracle time {est_s:.0f} s over the "
                                               f"--full-parity-s budget {args.full_parity_s} s"}
    if rank != 0:
        T.close()
        if world > 1:
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(w, idx, vals, facs_np, dtype, R, args.cpu_sample)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if dtype == "f64" else "f32",  # accumulation; 16-bit factors widen to fp32
        "data": "synthetic",
        "config": {"workload": w.name, "dims": w.dims, "nnz": w.nnz, "zipf_s": w.s, "R": R,
                   "factors": dtype, "factor_dist": w.factor_dist, "scatter": args.scatter,
                   "schedule": args.sched if args.sched == "default" else
                   "exhaustive autotune per mode (untimed set-up, %.1f s)" % tune_s,
                   "step": "MTTKRP of every mode (one launch per mode)",
                   "slice_order": bool(args.slice_order),
                   "l2_blocks": l2_blocks or "none",
                   "l2": "inputs larger than L2 (COO stream "
                   f"{w.nnz * 4 * (d + 1) / 1e9:.1f} GB per mode pass)"},
        "per_mode_ms": mode_ms,
        "per_mode_graph_median_ms": graph_mode_ms,
        "schedules": [s_.as_dict() for s_ in scheds],
        "per_mode_nnzR_per_s": [w.nnz * R / (m / 1e3) for m in mode_ms],
        "roofline": roofline,
        "gpu_launches": d * args.steps,
        "ingest_s": ingest_s, "permutation_s": perm_s,
        "clocks": clk,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    line.update(extra)
    print(json.dumps(line), flush=True)
    T.close()
    if world > 1:
        dist.destroy_process_group()


def full_parity(args, P, torch, w, T, idx, vals, R, d, outs, sched_for):
    """Relative Frobenius error of the whole output of every mode against the
    FP64 oracle (its all-core form, outside any timed region): the sorted,
    perm_n (over the coordinate arrays, and over the storage-order records),
    atomic and private scatters and the deterministic call, with fp32
    and with bf16 factors.  The gate compares with the oracle fed the same
    stored factor values (1e-5 for fp32, 2e-3 for bf16); for bf16 the error
    against the un-rounded fp32 factors (the quantisation included) is
    reported beside it."""
    import oracle
    th = host_threads()
    t0 = time.perf_counter()
    res = {"gate": {"f32": 1e-5, "bf16": 2e-3}, "metric": "||V_gpu - V_oracle||_F / ||V_oracle||_F per mode",
           "oracle": f"oracle_mttkrp_threads on {th} host threads, FP64"}
    ref32 = None
    for fdt in ["f32", "bf16"]:
        fnp = w.factors(R, fdt)
        fd = [_dev_factor(torch, f, fdt) for f in fnp]
        A64 = [oracle.as_f64(f, fdt)[:, :R].copy() for f in fnp]
        errs = {}
        quant = []
        for n in range(d):
            ref = oracle.mttkrp_threads(idx, vals, w.dims, A64, n, R, th)
            den = np.linalg.norm(ref)
            for sc in ["sorted", "perm", "perm_rec", "atomic", "private", "deterministic"]:
                if sc in ("sorted", "perm", "deterministic") and args.scatter == "perm" and sc != "perm":
                    continue
                try:
                    if sc == "perm_rec":  # perm_n over the storage-order records
                        T.storage_records(True)
                    s = sched_for(n, {"deterministic": "sorted", "perm_rec": "perm"}.get(sc, sc), fdt)
                    if sc == "deterministic" and s.lanes_per_nnz * s.chunks * 4 < R:
                        s = None
                    T.mttkrp(n, fd, R, out=outs[n], sched=s, deterministic=(sc == "deterministic"))
                except P.SptError:  # private: this mode's output copy does not fit a cluster
                    errs.setdefault(sc, []).append(None)
                    continue
                finally:
                    if sc == "perm_rec":
                        T.storage_records(False)
                got = outs[n][:, :R].double().cpu().numpy()
                errs.setdefault(sc, []).append(float(np.linalg.norm(got - ref) / den))
                if fdt == "bf16" and sc == "sorted":
                    quant.append(float(np.linalg.norm(got - ref32[n]) / np.linalg.norm(ref32[n])))
            if fdt == "f32":
                ref32 = (ref32 or []) + [ref]
        res[fdt] = errs
        if fdt == "bf16":
            res["bf16_vs_unrounded_f32_factors"] = {"sorted": quant}
        del fd
    worst = {fdt: max((e for v in res[fdt].values() for e in v if e is not None), default=None)
             for fdt in ("f32", "bf16")}
    res["worst"] = worst
    res["within_gate"] = all(worst[f] is not None and worst[f] <= res["gate"][f] for f in worst)
    res["seconds"] = time.perf_counter() - t0
    T.check()
    return res


def measure_extras(args, P, torch, w, T, idx, vals, facs_np, dtype, R, d, ld, outs, sched_for,
                   mode_ms):
    """Variants (scatter x factor precision), CP-ALS iterations and sampled
    errors against the oracle -- reported beside the headline number."""
    import oracle
    stream = torch.cuda.current_stream()
    out = {}
    # ---- scatter x precision, MTTKRP only, ms per mode
    var = {}
    for fdt in ["f32", "bf16"]:
        fnp = w.factors(R, fdt)
        fd = [_dev_factor(torch, f, fdt) for f in fnp]
        for sc in (["sorted"] if args.scatter != "perm" else []) + ["perm", "perm_rec", "atomic", "private"]:
            ms = []
            T.storage_records(sc == "perm_rec")  # perm_rec: perm_n over the storage-order records
            for n in range(d):
                s = sched_for(n, "perm" if sc == "perm_rec" else sc, fdt)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                try:
                    T.mttkrp(n, fd, R, out=outs[n], sched=s)
                except P.SptError:  # private: this mode's output copy does not fit a cluster
                    if sc != "private":
                        raise
                    ms.append(None)
                    continue
                e0.record(stream)
                for _ in range(3):
                    T.mttkrp(n, fd, R, out=outs[n], sched=s)
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1) / 3)
            # sampled-row error against the oracle (same stored factor values)
            errs = []
            A64 = [oracle.as_f64(f, fdt)[:, :R].copy() for f in fnp]
            if sc in ("sorted", "atomic", "private"):
                for n in range(d):
                    if ms[n] is None:
                        errs.append(None)
                        continue
                    rows = sampled_rows(w, idx, n, R)
                    T.mttkrp(n, fd, R, out=outs[n], sched=sched_for(n, sc, fdt))
                    got = outs[n][torch.from_numpy(rows).long().cuda(), :R].double().cpu().numpy()
                    ref = oracle.mttkrp_rows(idx, vals, w.dims, A64, n, R, rows)
                    errs.append(float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
            T.storage_records(False)
            ran = [m for m in ms if m is not None]
            var[f"{sc}/{fdt}"] = {"ms_per_mode": ms,
                                  "nnzR_per_s": w.nnz * R * len(ran) / (sum(ran) / 1e3) if ran else None,
                                  "rel_err_sampled_rows": errs or None}
        del fd
    out["variants"] = var
    # ---- deterministic sums (per-warp boundary slots and a fix-up kernel in
    # place of the boundary rows' atomics): ms per mode, bit-identical repeats
    if args.scatter == "sorted" and R <= 256:
        fnp = w.factors(R, dtype)
        fd = [_dev_factor(torch, f, dtype) for f in fnp]
        A64 = [oracle.as_f64(f, dtype)[:, :R].copy() for f in fnp]
        ms, errs, same = [], [], True
        for n in range(d):
            s = sched_for(n, "sorted", dtype)
            if s is not None and s.lanes_per_nnz * s.chunks * 4 < R:
                s = None
            T.mttkrp(n, fd, R, out=outs[n], sched=s, deterministic=True)
            first = outs[n].clone()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                T.mttkrp(n, fd, R, out=outs[n], sched=s, deterministic=True)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1) / 3)
            iv = torch.int64 if first.dtype == torch.float64 else torch.int32
            same = same and torch.equal(first.view(iv), outs[n].view(iv))
            rows = sampled_rows(w, idx, n, R)
            got = outs[n][torch.from_numpy(rows).long().cuda(), :R].double().cpu().numpy()
            ref = oracle.mttkrp_rows(idx, vals, w.dims, A64, n, R, rows)
            errs.append(float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
        out["deterministic"] = {"ms_per_mode": ms, "nnzR_per_s": w.nnz * R * d / (sum(ms) / 1e3),
                                "vs_default_ms": sum(ms) / sum(mode_ms), "bit_identical_repeats": same,
                                "rel_err_sampled_rows": errs}
        del fd
    # ---- generalised CP gradient (one fused launch per mode + the Poisson
    # dense term), beside the plain MTTKRP of the same schedule
    if args.scatter != "perm" and d >= 2:
        fnp = w.factors(R, dtype)
        fd = [_dev_factor(torch, f, dtype) for f in fnp]
        if w.factor_dist == "normal":  # keep the model positive for the Poisson loss
            fd = [f.abs() + 0.01 * (torch.arange(f.shape[1], device="cuda") < R).to(f.dtype) for f in fd]
        gcp = {}
        for loss in ["poisson", "bernoulli", "gaussian"]:
            ms = []
            for n in range(d):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                T.gcp_gradient(n, fd, R, loss, out=outs[n])
                e0.record(stream)
                for _ in range(3):
                    T.gcp_gradient(n, fd, R, loss, out=outs[n])
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1) / 3)
            gcp[loss] = {"ms_per_mode": ms, "nnzR_per_s": w.nnz * R * d / (sum(ms) / 1e3)}
        out["gcp_gradient"] = gcp
        del fd
    # ---- CP-ALS iterations on the coalesced tensor (duplicates summed)
    Tc = P.SparseTensor(idx, vals, w.dims, coalesce=True)
    t0 = time.perf_counter()
    Tc.build_permutation()  # plain copies: over a few iterations the slice order's longer build does not pay
    build_l2_blocks(Tc, l2_block_plan(args, w.dims, ld, 4 if dtype == "f32" else 2))
    torch.cuda.synchronize()
    sort_s = time.perf_counter() - t0
    fc = [_dev_factor(torch, f, dtype) for f in facs_np]
    tuned = args.sched == "tuned"
    if tuned:  # the autotuner's schedule per mode, recorded on the tensor for cp_als_step
        for n in range(d):
            best, _, _ = P.mttkrp_autotune(Tc.handle, n, [f.data_ptr() for f in fc], dtype, R, ld,
                                           outs[n].data_ptr(), 2, stream.cuda_stream)
            P.tensor_set_schedule(Tc.handle, n, dtype, R, best)
    lam = torch.zeros(R, dtype=torch.float64, device="cuda")
    fit = torch.zeros(1, dtype=torch.float64, device="cuda")
    ws = Tc.cp_als_workspace(R, ld)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        for _ in range(2):
            Tc.cp_als_step(fc, R, lam, fit, ws)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(side)
        iters = 5
        torch.cuda.nvtx.range_push("cpals")  # the timed iterations' launches (ncu --nvtx-include cpals/)
        for _ in range(iters):
            Tc.cp_als_step(fc, R, lam, fit, ws)
        torch.cuda.nvtx.range_pop()
        e1.record(side)
    torch.cuda.synchronize()
    it_ms = e0.elapsed_time(e1) / iters
    out["cp_als"] = {"nnz_coalesced": Tc.nnz, "ms_per_iter": it_ms, "iter_per_s": 1e3 / it_ms,
                     "schedules": "autotuned per mode" if tuned else "default rule",
                     "fit": float(fit.item()), "graph": True,
                     "permutation_build_s": sort_s,
                     "permutation_cost_in_iterations": sort_s * 1e3 / it_ms}
    Tc.close()
    return out


def run_cpals(args):
    """CP-ALS iterations (captured graphs) of one workload under four sources
    of per-mode MTTKRP schedules; the tensor is coalesced (duplicates summed)."""
    import torch
    import oracle
    import paper_1809_09175_gb300 as P
    import paper_1809_09175_gb300.selector as S
    import synth

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    w = synth.workload(args.workload, args.scale)
    if args.rank:
        w = synth.Workload(w.name, w.dims, w.nnz, w.s, args.rank, w.factor_dist, w.seed, w.factor_dtype)
    fdt = args.dtype or w.factor_dtype
    R, d = w.R, len(w.dims)
    ld = P.factor_ld(R)
    t0 = time.perf_counter()
    idx_d, vals_d = synth.coo_zipf_device(w.dims, w.nnz, w.s, w.seed)
    T = P.SparseTensor(idx_d, vals_d, w.dims, coalesce=True)
    del idx_d, vals_d
    torch.cuda.synchronize()
    t_ingest = time.perf_counter() - t0
    t0 = time.perf_counter()
    T.build_permutation()
    l2_blocks = build_l2_blocks(T, l2_block_plan(args, w.dims, ld, 4 if fdt == "f32" else 2))
    torch.cuda.synchronize()
    t_perm = time.perf_counter() - t0
    facs_np = w.factors(R, fdt)
    def fresh():
        return [(torch.from_numpy(f).cuda() if fdt == "f32" else
                 torch.from_numpy(f.view(np.int16)).cuda().view(torch.bfloat16)) for f in facs_np]
    facs = fresh()
    ptrs = [f.data_ptr() for f in facs]
    st = torch.cuda.current_stream().cuda_stream
    scheds = {"default": [P.mttkrp_default_schedule(T.handle, n, fdt, R) for n in range(d)],
              "paper_rule": [P.mttkrp_paper_schedule(R, fdt, "perm") for n in range(d)]}
    t0 = time.perf_counter()
    auto, auto_ms, auto_times = [], [], []
    for n in range(d):
        out = torch.empty((w.dims[n], ld), device="cuda")
        best, bms, times = P.mttkrp_autotune(T.handle, n, ptrs, fdt, R, ld, out.data_ptr(), 2, st)
        auto.append(best)
        auto_ms.append(bms)
        auto_times.append(times)
        del out
    t_tune = time.perf_counter() - t0
    scheds["exhaustive"] = auto
    t_select = t_verify = None
    sel_info = {}
    if os.path.exists(args.weights):
        net = S.Net.load(args.weights)
        t0 = time.perf_counter()
        chosen = [net.choose(T, n, R, fdt) for n in range(d)]
        t_select = time.perf_counter() - t0
        scheds["selector"] = [c[0] for c in chosen]
        ranks, sel_mode_ms, kept = [], [], []
        for n in range(d):
            cands, valid = P.mttkrp_candidates(T.handle, n, R)
            order = [q for q in np.argsort(chosen[n][1]) if valid[q]]
            tt = np.array(auto_times[n])
            ranks.append(order.index(int(np.argmin(np.where(tt > 0, tt, np.inf)))))
            out = torch.empty((w.dims[n], ld), device="cuda")
            sel_mode_ms.append(P.mttkrp_time_schedule(T.handle, n, ptrs, fdt, R, ld, out.data_ptr(),
                                                      chosen[n][0], 3, st))
            kept.append(chosen[n][0].as_dict() == scheds["default"][n].as_dict())
            del out
        t0 = time.perf_counter()
        ver = []
        for n in range(d):
            out = torch.empty((w.dims[n], ld), device="cuda")
            ver.append(net.choose_verified(T, n, R, fdt, facs, out, k=3))
            del out
        t_verify = time.perf_counter() - t0
        scheds["selector_verified"] = [v[0] for v in ver]
        sel_info = {"rank_of_exhaustive_best_in_network_order": ranks,
                    "selector_mttkrp_ms_per_mode": sel_mode_ms,
                    "selector_kept_default_per_mode": kept, "anchor_margin": net.anchor_margin,
                    "exhaustive_mttkrp_ms_per_mode": auto_ms,
                    "verified_mttkrp_ms_per_mode": [v[1] for v in ver],
                    "verify_s": t_verify}
    res = {}
    side = torch.cuda.Stream()
    for name, sc in scheds.items():
        for n in range(d):
            try:
                P.tensor_set_schedule(T.handle, n, fdt, R, sc[n])
            except P.SptError:
                P.tensor_set_schedule(T.handle, n, fdt, R, None)
        f = fresh()
        lam = torch.zeros(R, dtype=torch.float64, device="cuda")
        fit = torch.zeros(1, dtype=torch.float64, device="cuda")
        ws = T.cp_als_workspace(R, ld)
        fits, ms = [], []
        with torch.cuda.stream(side):
            for it in range(args.cpals):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(side)
                T.cp_als_step(f, R, lam, fit, ws)
                e1.record(side)
                side.synchronize()
                ms.append(e0.elapsed_time(e1))
                fits.append(float(fit.item()))
        P.cp_als_status(ws.data_ptr(), side.cuda_stream)
        steady = ms[2:] if len(ms) > 4 else ms  # first replay includes graph capture
        res[name] = {"ms_per_iter": float(np.median(steady)), "iter_per_s": 1e3 / float(np.median(steady)),
                     "fit_first": fits[0], "fit_last": fits[-1],
                     "fit_nondecreasing": bool(all(b >= a - 1e-6 for a, b in zip(fits, fits[1:])))}
        del ws, f
    line = {"metric": METRIC, "workload": w.name, "dims": w.dims, "nnz_generated": w.nnz,
            "nnz_coalesced": T.nnz, "R": R, "factors": fdt, "iterations": args.cpals,
            "ingest_coalesce_s": t_ingest, "permutation_s": t_perm, "l2_blocks": l2_blocks or "none",
            "autotune_s": t_tune,
            "select_s": t_select, "autotune_best_ms_per_mode": auto_ms, "selector_detail": sel_info,
            "cp_als": res,
            "schedules": {k: [s_.as_dict() for s_ in v] for k, v in scheds.items()}}
    for k in ("selector", "selector_verified"):
        if k in res:
            line[k + "_vs_exhaustive_time_ratio"] = res[k]["ms_per_iter"] / res["exhaustive"]["ms_per_iter"]
    print(json.dumps(line), flush=True)
    T.close()


def run_batched(args):
    """The many-tensor batch (order 3-4, dims 1e3-1e6, nnz 1e4-5e6, Zipf s in
    [0, 1.5), R in {16, 32, 64}): every mode of every tensor in one persistent
    launch (captured graph), against one launch per (tensor, mode); schedules
    from the autotuner."""
    import torch
    import paper_1809_09175_gb300 as P
    import synth

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    from paper_1809_09175_gb300 import multi
    fdt = args.dtype or "f32"
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    specs = multi.shard(synth.batched_specs(args.batched), rank, world)
    Ts, facs_all, outs_all, items, tuned = [], [], [], [], []
    t0 = time.perf_counter()
    for w in specs:
        idx, vals = synth.coo_zipf_device(w.dims, w.nnz, w.s, w.seed)
        T = P.SparseTensor(idx, vals, w.dims)
        del idx, vals
        T.build_permutation()
        ld = P.factor_ld(w.R)
        g = torch.Generator(device="cuda")
        g.manual_seed(w.seed)
        facs = []
        for I in w.dims:
            f = torch.zeros((I, ld), device="cuda")
            f[:, :w.R] = torch.rand((I, w.R), generator=g, device="cuda")
            facs.append(f if fdt == "f32" else f.to(torch.bfloat16))
        outs = [torch.empty((I, ld), device="cuda") for I in w.dims]
        sc = []
        for n in range(len(w.dims)):  # best schedule among the sorted-traversal candidates
            cands, valid = P.mttkrp_candidates(T.handle, n, w.R)
            best, bms = None, 1e30
            for c, v in zip(cands, valid):
                if not v or c.scatter != P.SPT_SCATTER_SORTED:
                    continue
                ms = P.mttkrp_time_schedule(T.handle, n, [f.data_ptr() for f in facs], fdt, w.R, ld,
                                            outs[n].data_ptr(), c, 1)
                if ms < bms:
                    best, bms = c, ms
            sc.append(best)
        Ts.append(T); facs_all.append(facs); outs_all.append(outs); tuned.append(sc)
        items.append({"tensor": T.handle, "mode": -1, "rank": w.R, "ld": ld,
                      "factors": [f.data_ptr() for f in facs], "outs": [o.data_ptr() for o in outs],
                      "scheds": sc})
    setup_s = time.perf_counter() - t0
    b, keep = P.mttkrp_batch_create(items, fdt)
    ntask, nitem, blocks = P.mttkrp_batch_info(b)
    side = torch.cuda.Stream()
    units = sum(w.nnz * w.R * len(w.dims) for w in specs)
    with torch.cuda.stream(side):
        for _ in range(args.warmup):
            P.mttkrp_batch_run(b, side.cuda_stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(side)
        for _ in range(args.steps):
            P.mttkrp_batch_run(b, side.cuda_stream)
        e1.record(side)
    torch.cuda.synchronize()
    P.mttkrp_batch_check(b)
    batch_ms = e0.elapsed_time(e1) / args.steps
    # one launch per (tensor, mode) with the same schedules
    def singles():
        for T, facs, outs, sc, w in zip(Ts, facs_all, outs_all, tuned, specs):
            for n in range(len(w.dims)):
                T.mttkrp(n, facs, w.R, out=outs[n], sched=sc[n])
    for _ in range(args.warmup):
        singles()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        singles()
    e1.record()
    torch.cuda.synchronize()
    single_ms = e0.elapsed_time(e1) / args.steps
    # each task's kernel alone (fastest of 3 launches, output zeroing included)
    task_ms = 0.0
    for T, facs, outs, sc, w in zip(Ts, facs_all, outs_all, tuned, specs):
        for n in range(len(w.dims)):
            task_ms += P.mttkrp_time_schedule(T.handle, n, [f.data_ptr() for f in facs], fdt, w.R,
                                              facs[0].shape[1], outs[n].data_ptr(), sc[n], 3)
    # bytes: the survey's algorithmic figure (sorted traversal, cache hits not
    # deducted) and a compulsory one: every output written once, every record
    # read once, and each factor's distinct touched rows (at most min(I_m, P))
    # read once
    s_f = 4 if fdt == "f32" else 2
    alg = comp = 0
    for w in specs:
        d_ = len(w.dims)
        ld_ = P.factor_ld(w.R)
        for n in range(d_):
            alg += algorithmic_bytes("sorted", w.nnz, d_, w.R, s_f, w.dims[n], w.dims[n])
            comp += (w.dims[n] * ld_ * 4 + w.nnz * 4 * {2: 4, 3: 4, 4: 6, 5: 6}[d_]
                     + sum(min(w.dims[m], w.nnz) * ld_ * s_f for m in range(d_) if m != n))
    peak, peak_kind = measured_peaks()
    line = {"metric": METRIC, "workload": f"batched{len(specs)}", "tensors": len(specs),
            "total_nnz": int(sum(w.nnz for w in specs)), "tasks": ntask, "work_items": nitem,
            "persistent_ctas": blocks, "factors": fdt, "setup_s": setup_s,
            "batched_ms": batch_ms, "batched_nnzR_per_s": units / (batch_ms / 1e3),
            "per_task_launches_ms": single_ms, "per_task_nnzR_per_s": units / (single_ms / 1e3),
            "sum_of_task_kernel_ms": task_ms,
            "speedup": single_ms / batch_ms, "launches_per_run": 1 + len({(s_.chunks, len(w.dims) == 5) for w, sc in zip(specs, tuned) for s_ in sc}),
            "graph": True,
            "bytes": {"algorithmic": alg, "compulsory": comp,
                      "algorithmic_GBps": alg / (batch_ms / 1e3) / 1e9,
                      "compulsory_GBps": comp / (batch_ms / 1e3) / 1e9,
                      "compulsory_frac": comp / (batch_ms / 1e3) / 1e9 / peak, "peak": peak,
                      "peak_kind": peak_kind}}
    print(json.dumps(line), flush=True)
    P.mttkrp_batch_destroy(b)
    for T in Ts:
        T.close()


def run_paper_sweep(args):
    """The paper's synthetic study (Sec. 7): MTTKRP of every mode of the
    30K x 40K x 50K tensor with 1e7 uniformly random nonzeros for R = 8..256
    in steps of 8, in the sorted (Fig. MTTKRP-C) and atomic (Fig. MTTKRP-B)
    traversals, with fp64 (the paper's precision), fp32 and bf16 factors;
    then 10 CP-ALS iterations at R = 128 (the paper's speed-up experiment).
    Reported per point: nnz*R/s, the paper's bandwidth model
    ((d R + 3) s_r + d s_o) P / t over the measured copy bandwidth, and for
    fp64 the fp64 operations (d per nonzero and column) over the measured
    fp64 FMA rate."""
    import torch
    import oracle
    import paper_1809_09175_gb300 as P
    import synth

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    w = synth.workload("uniform3d_30kx40kx50k_nnz1e7", args.scale)
    d = len(w.dims)
    idx, vals = w.coo()
    T = P.SparseTensor(idx, vals, w.dims)
    T.build_permutation()
    st = torch.cuda.current_stream()
    peak_gbs, peak_kind = measured_peaks()

    def ev_time(fn, reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        fn()
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    # fp64 / fp32 FMA throughput of this device (the fp64 path's roofline)
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    fma = {}
    for dt, iters in (("f64", 1 << 13), ("f32", 1 << 16)):
        flops = P.spt_fma_probe(dt, iters, sink.data_ptr(), st.cuda_stream)
        fma[dt] = flops / (ev_time(lambda: P.spt_fma_probe(dt, iters, sink.data_ptr(), st.cuda_stream), 3) / 1e3)

    a, b, c = (int(x) for x in args.sweep_ranks.split(":"))
    s_o = 4
    rows = []
    g = torch.Generator(device="cuda")
    for R in range(a, b, c):
        ld = P.factor_ld(R)
        for dt in ("f64", "f32", "bf16"):
            g.manual_seed(R)
            facs = []
            for I in w.dims:
                f = torch.zeros((I, ld), dtype=torch.float64, device="cuda")
                f[:, :R] = torch.rand((I, R), generator=g, dtype=torch.float64, device="cuda")
                facs.append(f.to({"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dt]))
            out = torch.empty((max(w.dims), ld), device="cuda",
                              dtype=torch.float64 if dt == "f64" else torch.float32)
            s_r = {"f64": 8, "f32": 4, "bf16": 2}[dt]
            for sc in ("sorted", "atomic"):
                ms = []
                for n in range(d):
                    sch = P.mttkrp_default_schedule(T.handle, n, dt, R)
                    sch.scatter = P.SCATTERS[sc]
                    o = out[: w.dims[n]]
                    ms.append(ev_time(lambda: T.mttkrp(n, facs, R, out=o, sched=sch), 3))
                t = sum(ms) / d / 1e3
                row = {"R": R, "factors": dt, "scatter": sc, "ms_per_mode": ms,
                       "nnzR_per_s": w.nnz * R * d / (sum(ms) / 1e3),
                       "paper_model_GBps": ((d * R + 3) * s_r + d * s_o) * w.nnz / t / 1e9}
                row["paper_model_frac_of_peak"] = row["paper_model_GBps"] / peak_gbs
                if dt == "f64":
                    row["fp64_frac_of_fma_peak"] = w.nnz * R * d / t / fma["f64"]
                rows.append(row)
            del facs, out
    # 10 CP-ALS iterations at R = 128 on the coalesced tensor (captured graph)
    Tc = P.SparseTensor(idx, vals, w.dims, coalesce=True)
    Tc.build_permutation()
    cp = {}
    R = 128
    ld = P.factor_ld(R)
    for dt in ("f32", "bf16"):
        fnp = synth.factor_matrices(w.dims, R, 11, "uniform", dtype=dt)
        facs = [_dev_factor(torch, f, dt) for f in fnp]
        lam = torch.zeros(R, dtype=torch.float64, device="cuda")
        fit = torch.zeros(1, dtype=torch.float64, device="cuda")
        ws = Tc.cp_als_workspace(R, ld)
        side = torch.cuda.Stream()
        with torch.cuda.stream(side):
            Tc.cp_als_step(facs, R, lam, fit, ws)  # capture
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(side)
            for _ in range(10):
                Tc.cp_als_step(facs, R, lam, fit, ws)
            e1.record(side)
        torch.cuda.synchronize()
        P.cp_als_status(ws.data_ptr(), side.cuda_stream)
        cp[dt] = {"s_per_10_iterations": e0.elapsed_time(e1) / 1e3, "fit": float(fit.item())}
    # the FP64 oracle's MTTKRP on one host core, sampled and scaled to the tensor
    sample = min(w.nnz, 1_000_000)
    A64 = [np.random.default_rng(m).random((I, R)) for m, I in enumerate(w.dims)]
    t0 = time.perf_counter()
    for n in range(d):
        oracle.mttkrp(idx[:, :sample], vals[:sample], w.dims, A64, n, R)
    t_or = (time.perf_counter() - t0) * w.nnz / sample
    best = {}
    for r in rows:
        k = (r["factors"], r["scatter"])
        best[k] = max(best.get(k, 0.0), r["paper_model_frac_of_peak"])
    line = {"metric": "paper sweep: MTTKRP nnz*R/s and bandwidth model vs R; CP-ALS 10 iterations",
            "workload": w.name, "dims": w.dims, "nnz": w.nnz, "nnz_coalesced": Tc.nnz,
            "hbm_peak_GBps": peak_gbs, "peak_kind": peak_kind,
            "fma_probe_flops": fma, "sweep": rows, "cp_als_R128": cp,
            "oracle_mttkrp_s_per_iteration_1core": t_or,
            "speedup_vs_1core_oracle_mttkrp": {dt: 10 * t_or / v["s_per_10_iterations"] for dt, v in cp.items()},
            "best_paper_model_frac": {f"{k[0]}/{k[1]}": v for k, v in best.items()}}
    print(json.dumps(line), flush=True)
    Tc.close()
    T.close()


def run_shard_cpals(args):
    """CP-ALS with the nonzeros split across the ranks (one per GPU, NCCL):
    every rank holds a contiguous range of each mode's permutation and owns
    the rows it reaches first; the rows shared at the cuts are completed by
    one small all-reduce, the Grams and column norms all-reduced, and each
    rank's factor rows broadcast (paper Sec. 8 future work).  The workload's
    tensor is coalesced; `--shard-cpals K` timed iterations after --warmup,
    the slowest rank's time.  With one rank, cp_als_step on the same GPU is
    timed beside it (the cost of the split and of the collectives' calls)."""
    import socket
    import torch
    import torch.distributed as dist
    import paper_1809_09175_gb300 as P
    from paper_1809_09175_gb300 import shard as S
    import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if "MASTER_ADDR" not in os.environ:  # one rank started without torchrun
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        so = socket.socket()
        so.bind(("127.0.0.1", 0))
        os.environ["MASTER_PORT"] = str(so.getsockname()[1])
        so.close()
    dist.init_process_group("nccl", rank=rank, world_size=world, device_id=torch.device("cuda", local))
    w = synth.workload(args.workload, args.scale)
    fdt = args.dtype or w.factor_dtype
    R, d = w.R, len(w.dims)
    ld = P.factor_ld(R)
    idx, vals = synth.coo_zipf_device(w.dims, w.nnz, w.s, w.seed)
    T = P.SparseTensor(idx, vals, w.dims, coalesce=True)
    del idx, vals
    T.build_permutation()
    shards = S.make_shards(T, world, rank)
    facs_np = w.factors(R, fdt)
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16}[fdt]
    facs = [torch.from_numpy(f.view(np.int16) if fdt != "f32" else f).cuda().view(tdt) for f in facs_np]
    drv = S.ShardedCPALS(S.DeviceOps(T, shards, R, fdt, ld), w.dims, R, ld)
    F = drv.replicated_factors(facs)
    lam = torch.zeros(R, dtype=torch.float64, device="cuda")
    fit = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        drv.step(F, lam, fit)
    torch.cuda.synchronize()
    dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.shard_cpals):
        drv.step(F, lam, fit)
    e1.record()
    torch.cuda.synchronize()
    dist.barrier()
    t = torch.tensor([e0.elapsed_time(e1) / args.shard_cpals], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    s_f = 4 if fdt == "f32" else 2
    comm = drv.collective_bytes(s_f)
    line = {"metric": "sharded CP-ALS iter/s", "workload": w.name, "n_gpus": world, "nnz_coalesced": T.nnz,
            "R": R, "factors": fdt, "iterations": args.shard_cpals, "warmup": args.warmup,
            "ms_per_iter": ms, "iter_per_s": 1e3 / ms, "fit": float(fit.item()),
            "collective_bytes_per_rank_per_iter": comm,
            "collectives": "per mode: all-reduce of the rows shared at the cuts (world x ld fp32), of the "
                           "column norms and of the R x R FP64 Gram, one broadcast of each rank's factor rows"}
    if world == 1:  # the unsplit iteration on the same GPU
        g = [torch.from_numpy(f.view(np.int16) if fdt != "f32" else f).cuda().view(tdt) for f in facs_np]
        ws = T.cp_als_workspace(R, ld)
        side = torch.cuda.Stream()
        with torch.cuda.stream(side):
            for _ in range(args.warmup):
                T.cp_als_step(g, R, lam, fit, ws)
            e0.record(side)
            for _ in range(args.shard_cpals):
                T.cp_als_step(g, R, lam, fit, ws)
            e1.record(side)
        torch.cuda.synchronize()
        line["cp_als_step_ms_per_iter"] = e0.elapsed_time(e1) / args.shard_cpals
    if rank == 0:
        print(json.dumps(line), flush=True)
    for s_ in shards:
        s_.close()
    T.close()
    dist.destroy_process_group()


def run_gather_probe(args):
    """The ceiling of the MTTKRP's gather step: 64-byte factor rows (fp32,
    R = 16) of the 3-way 1e8 workload's mode-1 and mode-2 factors (5e5 and
    2e5 rows, Zipf s = 1.2 row streams) brought to the SMs by 16-byte loads
    (the kernel's way), by TMA tile::gather4 and by 1-D bulk copies, each
    into a product, without the nonzero records or the scatter."""
    import torch
    import paper_1809_09175_gb300 as P
    import synth

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    n = int(args.gather_probe) // 64 * 64
    dims = (500_000, 200_000)
    idx, _ = synth.coo_zipf_device(dims, n, 1.2, 5)
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    F = [torch.rand((I, 16), generator=g, device="cuda") for I in dims]
    sink = torch.zeros(1, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream()
    out = {"metric": "factor-row gather rate (64-byte rows, two per nonzero)", "nonzeros": n,
           "rows": list(dims), "zipf_s": 1.2, "unit": "rows/s", "methods": {}}
    # the same rows, ordered by (row of F1, row of F2) within segments of
    # `seg` nonzeros, as a slice's nonzeros would be if the mode-sorted copy
    # ordered each slice by the other modes
    def sorted_within(seg):
        key = idx[0].long() * dims[1] + idx[1].long()
        if seg >= n:
            order = torch.argsort(key, stable=True)
        else:
            base = (torch.arange(n, device="cuda") // seg) * (dims[0] * dims[1])
            order = torch.argsort(base + key, stable=True)
        return idx[0][order].contiguous(), idx[1][order].contiguous()
    streams = {"random order": (idx[0], idx[1])}
    for seg in (184, 4096, n):
        streams[f"sorted within {seg}"] = sorted_within(seg)
    runs = [(0, "ld.global 16 B per lane", "random order"), (1, "TMA tile::gather4", "random order"),
            (2, "1-D cp.async.bulk per row", "random order")]
    for sname in list(streams)[1:]:
        runs += [(0, "ld.global 16 B per lane", sname), (3, "ld.global, groups on consecutive nonzeros", sname)]
    for m, mname, sname in runs:
        name = f"{mname} / {sname}"
        r1, r2 = streams[sname]

        def launch():
            P.spt_row_gather_probe(m, F[0].data_ptr(), dims[0], F[1].data_ptr(), dims[1], r1.data_ptr(),
                                   r2.data_ptr(), n, sink.data_ptr(), status.data_ptr(), st.cuda_stream)
        launch()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(5):
            launch()
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 5
        out["methods"][name] = {"ms": ms, "rows_per_s": 2 * n / (ms / 1e3), "ms_per_1e8_nonzeros": ms * 1e8 / n}
    out["status"] = int(status.item())
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.gather_probe:
        run_gather_probe(a)
    elif a.shard_cpals:
        run_shard_cpals(a)
    elif a.paper_sweep:
        run_paper_sweep(a)
    elif a.cpals:
        run_cpals(a)
    elif a.batched:
        run_batched(a)
    else:
        run_ours(a)
