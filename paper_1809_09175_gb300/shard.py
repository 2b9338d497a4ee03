"""CP-ALS over a tensor whose nonzeros are split across the ranks of a
``torch.distributed`` group -- the multi-GPU distribution that the paper
names as its first piece of future work (Sec. 8).

Every rank holds, for each mode n, the nonzeros at one contiguous range of
the mode-n permutation (``tensor_create_shard``), so its rows of V are mostly
its own, and a full copy of every factor matrix.  One mode update:

1. partial V = the mode-n MTTKRP of the rank's nonzeros (all I_n rows);
2. **reduce-scatter** of V by row blocks: rank r receives the summed rows
   ``[r B, (r+1) B)``, ``B = ceil(I_n / G)`` (V padded to ``G B`` rows);
3. ``H^-1`` from the replicated FP64 Grams, ``A32 = V_r H^-1`` on the rank's
   rows and their column sums of squares, **all-reduced** into lambda;
4. the normalised rows ``A_r = A32 / lambda``, their Gram ``A_r^T A_r``
   **all-reduced** into G_n (R x R FP64);
5. **all-gather** of the rows ``A_r`` into the replicated ``A^(n)``.

After the last mode the fit's ``<X, M>`` (from the last V's rows) and, once,
``||X||^2`` (from the mode-0 shards) are all-reduced.  The steps of 1 and
3-5 run in the library's CUDA kernels through the C ABI (:class:`DeviceOps`);
this module only moves buffers between them and the collectives.  The
collectives are ``torch.distributed`` calls (NCCL between GPUs).
"""
from __future__ import annotations

from typing import List, Optional, Sequence

import torch
import torch.distributed as dist

from . import binding as B
from .tensor import SparseTensor


def shard_bounds(nnz: int, world: int, rank: int):
    """Rank ``rank``'s range ``[begin, end)`` of perm_n positions: contiguous
    ranges of (nearly) equal length, in rank order."""
    return nnz * rank // world, nnz * (rank + 1) // world


def row_block(I: int, world: int):
    """Rows per rank of the reduce-scatter (V and the factors are padded to
    ``world * B`` rows)."""
    return (I + world - 1) // world


class DeviceOps:
    """The local steps of a mode update on this rank's GPU, through the C ABI."""

    acc_dtype = torch.float32  # V and the unnormalised rows A32

    def __init__(self, tensor: SparseTensor, shards: Sequence[SparseTensor], rank_: int, fdt: str, ld: int):
        self.T = tensor
        self.shards = list(shards)
        self.R = rank_
        self.fdt = fdt
        self.ld = ld
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.status = torch.zeros(1, dtype=torch.int32, device=self.dev)
        self.hinv = torch.empty((rank_, rank_), dtype=torch.float32, device=self.dev)

    @staticmethod
    def _s() -> int:
        return torch.cuda.current_stream().cuda_stream

    def partial_mttkrp(self, mode: int, factors: List[torch.Tensor], V: torch.Tensor):
        """V[:I_n] = MTTKRP of this rank's mode-n shard (rows past I_n zero)."""
        I = self.T.dims[mode]
        V[I:].zero_()
        self.shards[mode].mttkrp(mode, factors, self.R, out=V[:I])

    def gram(self, A: torch.Tensor, rows: int, G: torch.Tensor):
        G.zero_()
        B.cp_als_gram(A.data_ptr(), rows, self.ld, self.R, self.fdt, G.data_ptr(), self._s())

    def solve_rows(self, mode: int, Grams: torch.Tensor, Vr: torch.Tensor, rows: int, A32: torch.Tensor,
                   colsq: torch.Tensor):
        B.cp_als_hinv(Grams.data_ptr(), self.T.order, mode, self.R, self.hinv.data_ptr(), self.status.data_ptr(),
                      self._s())
        colsq.zero_()
        B.cp_als_apply(Vr.data_ptr(), rows, self.ld, self.R, self.hinv.data_ptr(), A32.data_ptr(), colsq.data_ptr(),
                       self._s())

    def normalize_rows(self, A32: torch.Tensor, rows: int, colsq: torch.Tensor, Ar: torch.Tensor,
                       lam: torch.Tensor, Vr: Optional[torch.Tensor], inner: Optional[torch.Tensor]):
        if inner is not None:
            inner.zero_()
        B.cp_als_normalize(A32.data_ptr(), Vr.data_ptr() if Vr is not None else 0, rows, self.ld, self.R,
                           colsq.data_ptr(), Ar.data_ptr(), self.fdt, lam.data_ptr(),
                           inner.data_ptr() if inner is not None else 0, self._s())

    def fit(self, Grams: torch.Tensor, lam: torch.Tensor, inner: torch.Tensor, xnorm2: float, fit: torch.Tensor):
        B.cp_als_fit(Grams.data_ptr(), self.T.order, self.R, lam.data_ptr(), inner.data_ptr(), xnorm2,
                     fit.data_ptr(), self._s())

    def check(self):
        h = int(self.status.item())
        if h:
            raise B.SptError(B.SPT_ESINGULAR, "a Gram-Hadamard matrix was not positive definite")

    def xnorm2(self) -> float:
        return self.shards[0].norm2()


def make_shards(T: SparseTensor, world: int, rank: int, stream: Optional[int] = None) -> List[SparseTensor]:
    """This rank's shard of every mode: perm_n positions shard_bounds(...)
    (needs T.build_permutation())."""
    st = torch.cuda.current_stream().cuda_stream if stream is None else stream
    out = []
    for n in range(T.order):
        b, e = shard_bounds(T.nnz, world, rank)
        S = SparseTensor.from_handle(B.tensor_create_shard(T.handle, n, b, e, st), T.dims)
        S.build_permutation(n)  # the shard's own mode takes the sorted traversal
        out.append(S)
    return out


class ShardedCPALS:
    """CP-ALS iterations over nonzeros split across a process group.

    ``ops`` performs the rank's local steps (:class:`DeviceOps` on a GPU);
    ``factors`` are the replicated factor matrices (I_m x ld each, padded
    here to ``world * B_m`` rows so that the collectives see equal blocks).
    All collective arguments are torch tensors on the ops' device."""

    def __init__(self, ops, dims: Sequence[int], rank_: int, ld: int, group=None):
        self.ops = ops
        self.dims = [int(x) for x in dims]
        self.d = len(self.dims)
        self.R = rank_
        self.ld = ld
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        self.x2 = None

    def _pad(self, I: int) -> int:
        return self.world * row_block(I, self.world)

    def padded_factors(self, factors: Sequence[torch.Tensor]) -> List[torch.Tensor]:
        """Copies of the factors padded with zero rows to world * B_m rows (the
        iteration updates them in place; row I_m and beyond stay zero)."""
        out = []
        for m, f in enumerate(factors):
            p = torch.zeros((self._pad(self.dims[m]), f.shape[1]), dtype=f.dtype, device=f.device)
            p[: self.dims[m]].copy_(f)
            out.append(p)
        return out

    def step(self, F: List[torch.Tensor], lam: torch.Tensor, fit: Optional[torch.Tensor] = None):
        """One iteration over every mode in order; F are the padded factors
        (updated in place), lam receives lambda (rank doubles)."""
        dev = F[0].device
        f64 = dict(dtype=torch.float64, device=dev)
        d, R, ld, w, r = self.d, self.R, self.ld, self.world, self.rank
        Grams = torch.zeros((d, R, R), **f64)
        for m in range(d):  # each rank's rows, summed over the ranks
            Bm = row_block(self.dims[m], w)
            rows = max(0, min(Bm, self.dims[m] - r * Bm))
            self.ops.gram(F[m][r * Bm:], rows, Grams[m])
        dist.all_reduce(Grams, group=self.group)
        colsq = torch.zeros(R, **f64)
        inner = torch.zeros(1, **f64)
        for n in range(d):
            In = self.dims[n]
            Bn = row_block(In, w)
            rows = max(0, min(Bn, In - r * Bn))
            V = torch.empty((w * Bn, ld), dtype=self.ops.acc_dtype, device=dev)
            self.ops.partial_mttkrp(n, [f[: self.dims[m]] for m, f in enumerate(F)], V)
            Vr = torch.empty((Bn, ld), dtype=self.ops.acc_dtype, device=dev)
            dist.reduce_scatter_tensor(Vr, V, group=self.group)
            A32 = torch.zeros((Bn, ld), dtype=self.ops.acc_dtype, device=dev)
            self.ops.solve_rows(n, Grams, Vr, rows, A32, colsq)
            dist.all_reduce(colsq, group=self.group)
            Ar = torch.zeros((Bn, ld), dtype=F[n].dtype, device=dev)
            last = n == d - 1
            self.ops.normalize_rows(A32, rows, colsq, Ar, lam, Vr if last else None, inner if last else None)
            self.ops.gram(Ar, rows, Grams[n])
            dist.all_reduce(Grams[n], group=self.group)
            dist.all_gather_into_tensor(F[n], Ar, group=self.group)
        dist.all_reduce(inner, group=self.group)
        if self.x2 is None:
            x2 = torch.tensor([self.ops.xnorm2()], **f64)
            dist.all_reduce(x2, group=self.group)
            self.x2 = float(x2.item())
        if fit is not None:
            self.ops.fit(Grams, lam, inner, self.x2, fit)
        self.ops.check()
        return Grams


__all__ = ["DeviceOps", "ShardedCPALS", "make_shards", "shard_bounds", "row_block"]
