"""Build the learned selector's timing dataset and train it on the GPU.

For each generated training tensor (order 3-5, Zipf skew 0-2, R 8-128,
dims log-uniform in [1e2, 1e6], nnz log-uniform in [nnz_lo, nnz_hi]) and
every mode, the exhaustive autotuner times all candidate schedules; the
paper's Tab. "sizes" rule and the library's default rule are timed too.
The network is trained on the first (1 - holdout) of the tensors (plus
``--large`` extra tensors with more nonzeros) with the library's own
forward/backward/Adam kernels, and evaluated on the held-out rest.

    python -m paper_1809_09175_gb300.train_selector --count 500 --out DIR

writes DIR/selector_dataset.npz, DIR/selector_weights.npz and
DIR/selector_report.json;

    python -m paper_1809_09175_gb300.train_selector --extend OLD/selector_dataset.npz \
        --large 40 --nnz-hi 3e7 --large-hi 3e8 --out DIR

appends 40 more training tensors with 3e7..3e8 nonzeros to a saved dataset
and trains on the union (the held-out tensors stay the same).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

from . import binding as B  # noqa: E402
from . import selector as S  # noqa: E402
from .tensor import SparseTensor, factor_ld  # noqa: E402


def device_factors(dims, R, fdt, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    ld = factor_ld(R)
    out = []
    for I in dims:
        f = torch.zeros((I, ld), device="cuda")
        f[:, :R] = torch.rand((I, R), generator=g, device="cuda")
        out.append(f if fdt == "f32" else f.to(torch.bfloat16))
    return out


def order5_specs(count: int, seed0: int = 40_000):
    """Large order-5 power-law tensors like the 5-way CP-ALS workload: mode
    lengths log-uniform around 5e5, 2e5, 5e4, 5e3, 5e2 (a factor 3 either
    way), 1e8..3e8 nonzeros, Zipf s in [0.9, 1.3], R in {16, 32, 64}."""
    out = []
    for t in range(count):
        rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed0 + t, 13])))
        dims = [int(round(c * np.exp(rng.uniform(-np.log(3), np.log(3))))) for c in (5e5, 2e5, 5e4, 5e3, 5e2)]
        nnz = int(round(np.exp(rng.uniform(np.log(1e8), np.log(3e8)))))
        out.append(synth.Workload(f"o5_{t}", dims, nnz, float(rng.uniform(0.9, 1.3)),
                                  int(rng.choice([16, 32, 64])), "uniform", seed0 + t))
    return out


def measure_tensor(w, fdt, reps, coalesce=False):
    """Rows (features, candidate times, paper-rule time, default-rule time);
    coalesce: duplicates summed and the nonzeros in lexicographic order, as
    CP-ALS keeps them."""
    torch.cuda.empty_cache()
    idx, vals = synth.coo_zipf_device(w.dims, w.nnz, w.s, w.seed)
    T = SparseTensor(idx, vals, w.dims, coalesce=coalesce)
    del idx, vals
    T.build_permutation()
    facs = device_factors(w.dims, w.R, fdt, w.seed)
    ld = facs[0].shape[1]
    ptrs = [f.data_ptr() for f in facs]
    st = torch.cuda.current_stream().cuda_stream
    rows = []
    for n in range(T.order):
        out = torch.empty((w.dims[n], ld), device="cuda")
        feat = B.tensor_mode_features(T.handle, n, w.R, fdt)
        _, _, times = B.mttkrp_autotune(T.handle, n, ptrs, fdt, w.R, ld, out.data_ptr(), reps, st)
        paper = B.mttkrp_paper_schedule(w.R, fdt, "perm")
        try:
            t_paper = B.mttkrp_time_schedule(T.handle, n, ptrs, fdt, w.R, ld, out.data_ptr(), paper,
                                             reps, st)
        except B.SptError:  # the table's block does not fit this kernel's shared memory
            paper.nnz_per_group = 32
            t_paper = B.mttkrp_time_schedule(T.handle, n, ptrs, fdt, w.R, ld, out.data_ptr(), paper,
                                             reps, st)
        dflt = B.mttkrp_default_schedule(T.handle, n, fdt, w.R)
        t_dflt = B.mttkrp_time_schedule(T.handle, n, ptrs, fdt, w.R, ld, out.data_ptr(), dflt, reps, st)
        rows.append((np.array(feat, np.float32), np.array(times, np.float32), t_paper, t_dflt))
        del out
    T.close()
    return rows


def evaluate(pred, times, t_paper, t_dflt, margin=S.ANCHOR_MARGIN):
    """Selected schedule's time (the anchored rule of mttkrp_select) vs the
    exhaustive best and the two fixed rules."""
    sel = np.array([S.pick(pred[b], times[b], t_dflt[b], margin) for b in range(times.shape[0])])
    best = np.array([times[b][times[b] > 0].min() for b in range(times.shape[0])])
    return {
        "samples": int(times.shape[0]),
        "total_ms_selected": float(sel.sum()),
        "total_ms_best": float(best.sum()),
        "total_ms_paper_rule": float(np.sum(t_paper)),
        "total_ms_default_rule": float(np.sum(t_dflt)),
        "regret_total": float(sel.sum() / best.sum() - 1.0),
        "regret_mean": float(np.mean(sel / best - 1.0)),
        "regret_p90": float(np.quantile(sel / best - 1.0, 0.9)),
        "speedup_vs_paper_rule": float(np.sum(t_paper) / sel.sum()),
        "speedup_vs_default_rule": float(np.sum(t_dflt) / sel.sum()),
        "selected_default": float(np.mean([s_ == d_ for s_, d_ in zip(sel, t_dflt)])),
        "worse_than_default": float(np.mean(sel > np.asarray(t_dflt) * 1.02)),
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=500)
    ap.add_argument("--nnz-lo", type=float, default=1e5)
    ap.add_argument("--nnz-hi", type=float, default=1e7)
    ap.add_argument("--large", type=int, default=0, help="extra tensors with nnz in [nnz_hi, large_hi]")
    ap.add_argument("--large-hi", type=float, default=1.5e8)
    ap.add_argument("--order5", type=int, default=0,
                    help="extra training tensors like the 5-way CP-ALS workload (order5_specs)")
    ap.add_argument("--extend", default=None,
                    help="append --large, --count and --order5 new training tensors (other seeds) to "
                         "this saved dataset")
    ap.add_argument("--coalesce", action="store_true",
                    help="with --extend: the new tensors are coalesced (lexicographic order, as CP-ALS uses)")
    ap.add_argument("--holdout", type=float, default=0.1)
    ap.add_argument("--epochs", type=int, default=4000)
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--out", default=".")
    ap.add_argument("--dataset", default=None, help="train from a saved selector_dataset.npz")
    ap.add_argument("--weighting", default="sqrt", choices=["sqrt", "none"])
    ap.add_argument("--margin", type=float, default=S.ANCHOR_MARGIN,
                    help="selection keeps the default rule unless a candidate is predicted this much "
                         "faster (log time); stored with the weights")
    a = ap.parse_args()
    os.makedirs(a.out, exist_ok=True)
    if a.dataset:
        z = np.load(a.dataset)
        return train_and_report(a, z["X"], z["times"], z["t_paper"], z["t_default"], z["meta"],
                                int(z["n_train_tensors"]) if "n_train_tensors" in z else None, 0.0,
                                z["train_mask"] if "train_mask" in z else None,
                                z["coalesced_ids"] if "coalesced_ids" in z else None)
    if a.extend:
        z = np.load(a.extend)
        meta0 = z["meta"]
        mask0 = z["train_mask"] if "train_mask" in z else meta0[:, 0] < int(z["n_train_tensors"])
        big = (synth.selector_specs(a.large, seed0=30_000, nnz_lo=a.nnz_hi, nnz_hi=a.nnz_hi,
                                    large=a.large, large_hi=a.large_hi) if a.large else [])
        big += synth.selector_specs(a.count, seed0=50_000, nnz_lo=a.nnz_lo, nnz_hi=a.nnz_hi) if a.count else []
        big += order5_specs(a.order5, seed0=41_000)
        X, TT, TP, TD, meta = [list(z[k]) for k in ("X", "times", "t_paper", "t_default", "meta")]
        coalesced_ids = list(z["coalesced_ids"]) if "coalesced_ids" in z else []
        base = int(meta0[:, 0].max()) + 1
        t0 = time.time()
        for i, w in enumerate(big):
            fdt = "bf16" if i % 2 else "f32"
            for n, (f, t, tp, td) in enumerate(measure_tensor(w, fdt, a.reps, a.coalesce)):
                X.append(f); TT.append(t); TP.append(tp); TD.append(td)
                meta.append(np.array((base + i, n, w.R, 0 if fdt == "f32" else 1, w.nnz, len(w.dims))))
            if a.coalesce:
                coalesced_ids.append(base + i)
            print(f"{i + 1}/{len(big)} extra tensors, {time.time() - t0:.0f} s", flush=True)
        X = np.array(X, np.float32); TT = np.array(TT, np.float32)
        TP = np.array(TP, np.float32); TD = np.array(TD, np.float32); meta = np.array(meta, np.int64)
        mask = np.concatenate([mask0, np.ones(len(meta) - len(meta0), bool)])
        np.savez(os.path.join(a.out, "selector_dataset.npz"), X=X, times=TT, t_paper=TP, t_default=TD,
                 meta=meta, train_mask=mask, coalesced_ids=np.array(coalesced_ids, np.int64))
        return train_and_report(a, X, TT, TP, TD, meta, None, time.time() - t0, mask, coalesced_ids)
    specs = synth.selector_specs(a.count, nnz_lo=a.nnz_lo, nnz_hi=a.nnz_hi)
    # larger tensors join the training part only (the held-out part keeps the base recipe)
    big = synth.selector_specs(a.large, seed0=20_000, nnz_lo=a.nnz_hi, nnz_hi=a.nnz_hi,
                               large=a.large, large_hi=a.large_hi) if a.large else []
    big += order5_specs(a.order5)
    specs = specs[: int(round(len(specs) * (1 - a.holdout)))] + big + \
        specs[int(round(len(specs) * (1 - a.holdout))):]
    X, TT, TP, TD, meta = [], [], [], [], []
    t0 = time.time()
    for i, w in enumerate(specs):
        fdt = "bf16" if i % 2 else "f32"
        for n, (f, t, tp, td) in enumerate(measure_tensor(w, fdt, a.reps)):
            X.append(f); TT.append(t); TP.append(tp); TD.append(td)
            meta.append((i, n, w.R, 0 if fdt == "f32" else 1, w.nnz, len(w.dims)))
        if (i + 1) % 50 == 0:
            print(f"{i + 1}/{len(specs)} tensors, {time.time() - t0:.0f} s", flush=True)
    X = np.array(X, np.float32); TT = np.array(TT, np.float32)
    TP = np.array(TP, np.float32); TD = np.array(TD, np.float32); meta = np.array(meta, np.int64)
    n_train_tensors = int(round(a.count * (1 - a.holdout))) + len(big)
    np.savez(os.path.join(a.out, "selector_dataset.npz"), X=X, times=TT, t_paper=TP, t_default=TD,
             meta=meta, n_train_tensors=n_train_tensors)
    train_and_report(a, X, TT, TP, TD, meta, n_train_tensors, time.time() - t0)


def train_and_report(a, X, TT, TP, TD, meta, n_train_tensors, dataset_s, train_mask=None, coalesced_ids=None):
    if train_mask is not None:
        tr = np.asarray(train_mask, bool)
        n_train_tensors = int(len(np.unique(meta[tr, 0])))
    else:
        if n_train_tensors is None:  # datasets saved before the split was recorded: 450 + 30 large
            n_train_tensors = int(meta[:, 0].max() + 1) - 50
        tr = meta[:, 0] < n_train_tensors
    te = ~tr
    mean, std = S.fit_scaling(X[tr])
    net = S.Net.init(0, mean=mean, std=std)
    net.anchor_margin = a.margin
    T, M = S.targets(TT, TD, a.weighting)
    hist = net.train(X[tr], T[tr], M[tr], epochs=a.epochs, lr=3e-3, log_every=500)
    net.save(os.path.join(a.out, "selector_weights.npz"))
    rep = {"dataset_s": dataset_s, "tensors": int(meta[:, 0].max() + 1), "samples": int(X.shape[0]),
           "train_tensors": n_train_tensors, "weighting": a.weighting, "anchor_margin": a.margin,
           "targets": "log(candidate time / default-rule time)", "loss": hist,
           "train": evaluate(net.predict(X[tr]), TT[tr], TP[tr], TD[tr], a.margin),
           "holdout": evaluate(net.predict(X[te]), TT[te], TP[te], TD[te], a.margin)}
    o5 = (meta[:, 5] == 5) & (meta[:, 4] >= 1e8)
    if o5.any():  # the large order-5 training tensors (like the 5-way CP-ALS workload)
        rep["order5_large"] = evaluate(net.predict(X[o5]), TT[o5], TP[o5], TD[o5], a.margin)
    if coalesced_ids is not None and len(coalesced_ids):
        co = np.isin(meta[:, 0], np.asarray(coalesced_ids))
        rep["coalesced"] = evaluate(net.predict(X[co]), TT[co], TP[co], TD[co], a.margin)
    with open(os.path.join(a.out, "selector_report.json"), "w") as f:
        json.dump(rep, f, indent=1)
    print(json.dumps({k: rep[k] for k in ("tensors", "samples", "train", "holdout")}), flush=True)


if __name__ == "__main__":
    main()
