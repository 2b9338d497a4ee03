"""Learned MTTKRP schedule selector (not in the paper).

The paper fixes its launch shape by a rule of the rank (Tab. "sizes",
Sec. 5).  Here the exhaustive autotuner (``mttkrp_autotune``) times every
candidate schedule of a (tensor, mode, rank, dtype); those timings train a
small network (``mlp_*`` kernels: forward, back-propagation, Adam, all in
``libspt.so``) that maps the mode's features (``tensor_mode_features``) to
the predicted log time of each candidate relative to the library's own
choice (``mttkrp_default_schedule``), and ``mttkrp_select`` picks the
candidate with the smallest prediction -- keeping the library's choice unless
a candidate is predicted to beat it by more than ``ANCHOR_MARGIN`` -- using
the network's fused inference kernel.  This module only marshals data between those entry points.
"""
from __future__ import annotations

import math
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import binding as B

F = B.SPT_NUM_FEATURES
K = B.SPT_NUM_CANDIDATES
H1 = 64
H2 = 64


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def collect(T, factors: List[torch.Tensor], rank: int, fdt: str, reps: int = 1):
    """Autotune every mode of a tensor; returns [(features, times_ms)]."""
    ld = factors[0].shape[1]
    rows = []
    ptrs = [f.data_ptr() for f in factors]
    for n in range(T.order):
        out = torch.empty((T.dims[n], ld), dtype=torch.float32, device="cuda")
        feat = B.tensor_mode_features(T.handle, n, rank, fdt)
        _, _, times = B.mttkrp_autotune(T.handle, n, ptrs, fdt, rank, ld, out.data_ptr(), reps,
                                        _stream())
        rows.append((np.array(feat, np.float32), np.array(times, np.float32)))
        del out
    return rows


# The network's outputs are log(candidate time / time of the library's own
# choice, mttkrp_default_schedule), so a negative output is a predicted gain
# over running without the selector; mttkrp_select keeps the library's
# choice unless some candidate is predicted to beat it by more than this.
ANCHOR_MARGIN = 0.02


def targets(times: np.ndarray, t_default: np.ndarray, weighting: str = "sqrt"):
    """Regression targets: log(time / default-rule time) of each valid
    candidate; mask 0 where a candidate could not run.  With weighting
    "sqrt" a sample's mask is sqrt(its best time / the mean best time), so
    the fit favours the tensors that dominate total run time over
    launch-overhead noise of tiny ones; "none" weighs every sample alike."""
    times = np.asarray(times, np.float64)
    t_default = np.asarray(t_default, np.float64)
    valid = times > 0
    T = np.zeros(times.shape, np.float32)
    M = valid.astype(np.float32)
    best = np.ones(times.shape[0])
    for b in range(times.shape[0]):
        v = valid[b]
        if v.any():
            best[b] = times[b, v].min()
            T[b, v] = np.log(times[b, v] / t_default[b])
    if weighting == "sqrt":
        M *= np.sqrt(best / best.mean()).astype(np.float32)[:, None]
    return T, M


def pick(pred: np.ndarray, times: np.ndarray, t_default: float, margin: float) -> float:
    """Time of the schedule the anchored rule selects for one sample: the
    best-predicted valid candidate if it is predicted to beat the default by
    more than `margin`, else the default."""
    v = times > 0
    if not v.any():
        return float(t_default)
    y = np.where(v, pred, np.inf)
    q = int(np.argmin(y))
    return float(times[q]) if (margin < 0 or y[q] < -margin) else float(t_default)


class Net:
    """Parameters (device, packed as the kernels expect) and feature scaling."""

    def __init__(self, params: torch.Tensor, mean: np.ndarray, std: np.ndarray,
                 h1: int = H1, h2: int = H2, anchor_margin: float = ANCHOR_MARGIN):
        self.params = params
        self.mean = np.ascontiguousarray(mean, np.float32)
        self.std = np.ascontiguousarray(std, np.float32)
        self.h1, self.h2 = h1, h2
        self.anchor_margin = float(anchor_margin)

    @staticmethod
    def init(seed: int = 0, h1: int = H1, h2: int = H2, mean=None, std=None):
        rng = np.random.default_rng(seed)
        parts = [rng.standard_normal((h1, F)) * math.sqrt(2.0 / F), np.zeros(h1),
                 rng.standard_normal((h2, h1)) * math.sqrt(2.0 / h1), np.zeros(h2),
                 rng.standard_normal((K, h2)) * math.sqrt(1.0 / h2), np.zeros(K)]
        flat = np.concatenate([p.reshape(-1) for p in parts]).astype(np.float32)
        assert flat.size == B.mlp_param_count(F, h1, h2, K)
        return Net(torch.from_numpy(flat).cuda(), np.zeros(F) if mean is None else mean,
                   np.ones(F) if std is None else std, h1, h2)

    def unpack(self):
        """Host float64 copies (W1, b1, W2, b2, W3, b3)."""
        p = self.params.double().cpu().numpy()
        shapes = [(self.h1, F), (self.h1,), (self.h2, self.h1), (self.h2,), (K, self.h2), (K,)]
        out, o = [], 0
        for s in shapes:
            n = int(np.prod(s))
            out.append(p[o:o + n].reshape(s))
            o += n
        return out

    def normalise(self, X: np.ndarray) -> np.ndarray:
        return ((np.asarray(X, np.float32) - self.mean) / self.std).astype(np.float32)

    def train(self, X: np.ndarray, T: np.ndarray, M: np.ndarray, epochs: int = 3000,
              lr: float = 3e-3, log_every: int = 0) -> List[float]:
        """Full-batch Adam on the masked MSE, on the GPU kernels."""
        Bn = X.shape[0]
        x = torch.from_numpy(self.normalise(X)).cuda()
        t = torch.from_numpy(np.ascontiguousarray(T, np.float32)).cuda()
        m = torch.from_numpy(np.ascontiguousarray(M, np.float32)).cuda()
        n = self.params.numel()
        grads = torch.zeros(n, device="cuda")
        m1 = torch.zeros(n, device="cuda")
        v1 = torch.zeros(n, device="cuda")
        loss = torch.zeros(1, device="cuda")
        work = torch.empty(B.mlp_workspace_floats(Bn, F, self.h1, self.h2, K), device="cuda")
        hist = []
        st = _stream()
        for e in range(1, epochs + 1):
            B.mlp_loss_grad(Bn, F, self.h1, self.h2, K, x.data_ptr(), self.params.data_ptr(),
                            t.data_ptr(), m.data_ptr(), grads.data_ptr(), loss.data_ptr(),
                            work.data_ptr(), st)
            B.mlp_adam(n, self.params.data_ptr(), grads.data_ptr(), m1.data_ptr(), v1.data_ptr(),
                       lr, 0.9, 0.999, 1e-8, e, st)
            if log_every and (e % log_every == 0 or e == 1):
                hist.append(float(loss.item()))
        hist.append(float(loss.item()))
        return hist

    def predict(self, X: np.ndarray) -> np.ndarray:
        Bn = X.shape[0]
        x = torch.from_numpy(self.normalise(X)).cuda()
        y = torch.empty((Bn, K), device="cuda")
        work = torch.empty(B.mlp_workspace_floats(Bn, F, self.h1, self.h2, K), device="cuda")
        B.mlp_forward(Bn, F, self.h1, self.h2, K, x.data_ptr(), self.params.data_ptr(),
                      y.data_ptr(), work.data_ptr(), _stream())
        return y.cpu().numpy()

    def selector(self) -> B.spt_selector:
        self._keep = (np.ascontiguousarray(self.mean, np.float32),
                      np.ascontiguousarray(self.std, np.float32))
        fp = B.C.POINTER(B.C.c_float)
        return B.spt_selector(F, self.h1, self.h2, K, self.params.data_ptr(),
                              self._keep[0].ctypes.data_as(fp), self._keep[1].ctypes.data_as(fp),
                              self.anchor_margin)

    def choose(self, T, mode: int, rank: int, fdt: str):
        """The selector's schedule for (tensor, mode, rank, dtype)."""
        return B.mttkrp_select(T.handle, mode, fdt, rank, self.selector(), _stream())

    def choose_verified(self, T, mode: int, rank: int, fdt: str, factors, out, k: int = 3,
                        reps: int = 2, with_default: bool = True):
        """Time the network's k best-ranked valid candidates (instead of all
        SPT_NUM_CANDIDATES), and the library's default rule unless
        with_default is False, and return (schedule, ms) of the fastest."""
        _, pred = self.choose(T, mode, rank, fdt)
        cands, valid = B.mttkrp_candidates(T.handle, mode, rank)
        trial = [cands[q] for q in [q for q in np.argsort(pred) if valid[q]][:k]]
        if with_default:
            dflt = B.mttkrp_default_schedule(T.handle, mode, fdt, rank)
            if all(c.as_dict() != dflt.as_dict() for c in trial):
                trial.append(dflt)
        ld = factors[0].shape[1]
        ptrs = [f.data_ptr() for f in factors]
        best, bms = None, float("inf")
        for c in trial:
            ms = B.mttkrp_time_schedule(T.handle, mode, ptrs, fdt, rank, ld, out.data_ptr(),
                                        c, reps, _stream())
            if ms < bms:
                best, bms = c, ms
        return best, bms

    def save(self, path: str):
        np.savez(path, params=self.params.cpu().numpy(), mean=self.mean, std=self.std,
                 h1=self.h1, h2=self.h2, anchor_margin=self.anchor_margin)

    @staticmethod
    def load(path: str) -> "Net":
        z = np.load(path)
        h1, h2 = int(z["h1"]), int(z["h2"])
        want = B.mlp_param_count(F, h1, h2, K)
        if z["params"].size != want or z["mean"].size != F or z["std"].size != F:
            raise ValueError(f"{path}: a network for {z['params'].size} parameters, this library's "
                             f"candidate list needs {want} ({K} outputs); retrain it")
        # weights saved without a margin predict log(time / best time): no anchor
        margin = float(z["anchor_margin"]) if "anchor_margin" in z else -1.0
        return Net(torch.from_numpy(z["params"]).cuda(), z["mean"], z["std"], h1, h2, margin)


def fit_scaling(X: np.ndarray):
    mean = X.mean(axis=0)
    std = X.std(axis=0)
    std[std < 1e-6] = 1.0
    return mean.astype(np.float32), std.astype(np.float32)
