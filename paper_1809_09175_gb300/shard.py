"""CP-ALS over a tensor whose nonzeros are split across the ranks of a
``torch.distributed`` group -- the multi-GPU distribution that the paper
names as its first piece of future work (Sec. 8).

Every rank holds, for each mode n, the nonzeros at one contiguous range of
the mode-n permutation (``tensor_create_shard``), and a full copy of every
factor matrix.  The permutation is sorted by the mode-n coordinate, so a
rank's nonzeros cover one run of rows [first_r, last_r], and two ranks share
at most the row at the cut between them.  Rank r owns the rows after the
previous ranks' last rows up to its own last row (the last rank also owns
the rows after it, which hold no nonzeros), so every row has one owner and a
shared row belongs to the lowest rank whose nonzeros reach it.  One mode update:

1. partial V = the mode-n MTTKRP of the rank's nonzeros;
2. the **boundary rows**: each rank puts its partial of the row it shares
   with a lower rank into that owner's slot of a G x ld buffer, and its own
   last row into its slot; one **all-reduce** of that buffer, and each owner
   takes its slot back as the full row of V.  No other row of V has a
   partial on another rank, so V is never reduced as a whole;
3. ``H^-1`` from the replicated FP64 Grams, ``A32 = V_r H^-1`` on the owned
   rows and their column sums of squares, **all-reduced** into lambda;
4. the normalised rows ``A_r = A32 / lambda`` written into the rank's rows
   of the factor, their Gram ``A_r^T A_r`` **all-reduced** into G_n;
5. one **broadcast** per rank of its rows of the factor.

Per mode a rank then sends its rows of the new factor and R + R^2 + G ld
numbers, where a reduce-scatter of V by row blocks would also move I_n x R
fp32 partial sums.  After the last mode the fit's ``<X, M>`` (from the owned
rows of the last V) and, once, ``||X||^2`` (from the mode-0 shards) are
all-reduced.  The steps of 1 and 3-4 run in the library's CUDA kernels
through the C ABI (:class:`DeviceOps`); this module only moves buffers
between them and the collectives (``torch.distributed``, NCCL between GPUs).
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

import torch
import torch.distributed as dist

from . import binding as B
from .tensor import SparseTensor


def shard_bounds(nnz: int, world: int, rank: int):
    """Rank ``rank``'s range ``[begin, end)`` of perm_n positions: contiguous
    ranges of (nearly) equal length, in rank order."""
    return nnz * rank // world, nnz * (rank + 1) // world


def owned_rows(lasts: Sequence[int], I: int) -> List[Tuple[int, int]]:
    """Row range ``[lo, hi)`` of every rank from the ranks' last rows in rank
    order (-1 for a rank without nonzeros): rank r owns the rows after the
    largest last row of the ranks before it, up to and including its own
    last row; the last rank also owns the rows up to I.  A rank whose
    nonzeros all lie in a row owned by a lower rank owns nothing (lo == hi)."""
    out = []
    prev = -1
    G = len(lasts)
    for r in range(G):
        cur = max(prev, int(lasts[r]))
        lo = prev + 1
        hi = I if r == G - 1 else cur + 1
        out.append((lo, max(lo, hi)))
        prev = cur
    return out


def row_owner(own: Sequence[Tuple[int, int]], row: int) -> int:
    """The rank whose range of ``own`` holds ``row``."""
    for r, (lo, hi) in enumerate(own):
        if lo <= row < hi:
            return r
    raise ValueError(f"row {row} is outside every rank's range")


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

    def row_span(self, mode: int) -> Tuple[int, int]:
        """First and last mode-n row of this rank's mode-n shard, (-1, -1)
        if it holds no nonzeros (the shard keeps the permutation's order, so
        they are its first and last coordinates)."""
        S = self.shards[mode]
        if S.nnz == 0:
            return -1, -1
        idx, _ = S.coo()
        return int(idx[mode, 0].item()), int(idx[mode, -1].item())

    def partial_mttkrp(self, mode: int, factors: List[torch.Tensor], V: torch.Tensor):
        """V (I_n rows) = MTTKRP of this rank's mode-n shard."""
        self.shards[mode].mttkrp(mode, factors, self.R, out=V)

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
    ``factors`` are the replicated factor matrices (I_m x ld each).  All
    collective arguments are torch tensors on the ops' device."""

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
        self.spans = None  # per mode: every rank's (first, last) row
        self.own = None    # per mode: every rank's owned rows [lo, hi)

    def replicated_factors(self, factors: Sequence[torch.Tensor]) -> List[torch.Tensor]:
        """Copies of the factors for the iteration to update in place."""
        return [f.clone() for f in factors]

    def _partition(self, dev):
        """Every rank's row span and owned rows of every mode (once: the
        shards do not change between iterations)."""
        if self.own is not None:
            return
        mine = torch.tensor([v for n in range(self.d) for v in self.ops.row_span(n)], dtype=torch.int64,
                            device=dev)
        every = [torch.empty_like(mine) for _ in range(self.world)]
        dist.all_gather(every, mine, group=self.group)
        every = [e.cpu().tolist() for e in every]
        self.spans = [[(e[2 * n], e[2 * n + 1]) for e in every] for n in range(self.d)]
        self.own = [owned_rows([sp[1] for sp in self.spans[n]], self.dims[n]) for n in range(self.d)]

    def _boundary_rows(self, n: int, V: torch.Tensor):
        """Complete the rows of V that a rank shares with the rank owning
        them: one all-reduce of a world x ld buffer (step 2)."""
        w, r = self.world, self.rank
        own, (first, last) = self.own[n], self.spans[n][r]
        lo, hi = own[r]
        Z = torch.zeros((w, V.shape[1]), dtype=V.dtype, device=V.device)
        owns_last = first >= 0 and lo <= last < hi
        if owns_last:
            Z[r].copy_(V[last])
        if first >= 0:
            o = row_owner(own, first)
            if o != r:
                Z[o].copy_(V[first])
        dist.all_reduce(Z, group=self.group)
        if owns_last:
            V[last].copy_(Z[r])

    def step(self, F: List[torch.Tensor], lam: torch.Tensor, fit: Optional[torch.Tensor] = None):
        """One iteration over every mode in order; F are the replicated
        factors (updated in place), lam receives lambda (rank doubles)."""
        dev = F[0].device
        f64 = dict(dtype=torch.float64, device=dev)
        d, R, ld, w, r = self.d, self.R, self.ld, self.world, self.rank
        self._partition(dev)
        Grams = torch.zeros((d, R, R), **f64)
        for m in range(d):  # each rank's owned rows, summed over the ranks
            lo, hi = self.own[m][r]
            self.ops.gram(F[m][lo:hi], hi - lo, Grams[m])
        dist.all_reduce(Grams, group=self.group)
        colsq = torch.zeros(R, **f64)
        inner = torch.zeros(1, **f64)
        for n in range(d):
            lo, hi = self.own[n][r]
            rows = hi - lo
            V = torch.empty((self.dims[n], ld), dtype=self.ops.acc_dtype, device=dev)
            self.ops.partial_mttkrp(n, [f[: self.dims[m]] for m, f in enumerate(F)], V)
            self._boundary_rows(n, V)
            Vr = V[lo:hi]
            A32 = torch.zeros((max(rows, 1), ld), dtype=self.ops.acc_dtype, device=dev)
            self.ops.solve_rows(n, Grams, Vr, rows, A32, colsq)
            dist.all_reduce(colsq, group=self.group)
            Ar = F[n][lo:hi]  # the rank's rows of the factor, written in place
            last = n == d - 1
            self.ops.normalize_rows(A32, rows, colsq, Ar, lam, Vr if last else None, inner if last else None)
            self.ops.gram(Ar, rows, Grams[n])
            dist.all_reduce(Grams[n], group=self.group)
            for s, (slo, shi) in enumerate(self.own[n]):
                if shi > slo:
                    dist.broadcast(F[n][slo:shi], src=s, group=self.group)
        dist.all_reduce(inner, group=self.group)
        if self.x2 is None:
            x2 = torch.tensor([self.ops.xnorm2()], **f64)
            dist.all_reduce(x2, group=self.group)
            self.x2 = float(x2.item())
        if fit is not None:
            self.ops.fit(Grams, lam, inner, self.x2, fit)
        self.ops.check()
        return Grams

    def collective_bytes(self, factor_bytes: int) -> int:
        """Bytes of the buffers one iteration passes to its collectives: per
        mode the shared-row buffer, the factor's rows (every rank's, through
        the broadcasts), the column norms and the Gram; then the first
        Grams and the fit's scalar (the one-time spans and ||X||^2 left out)."""
        acc = torch.tensor([], dtype=self.ops.acc_dtype).element_size()
        R, w, ld = self.R, self.world, self.ld
        per_mode = sum(w * ld * acc + I * ld * factor_bytes + R * 8 + R * R * 8 for I in self.dims)
        return per_mode + self.d * R * R * 8 + 8


__all__ = ["DeviceOps", "ShardedCPALS", "make_shards", "shard_bounds", "owned_rows", "row_owner"]
