"""Torch-tensor convenience layer over the C ABI (argument marshalling only).

``SparseTensor`` owns a library tensor handle; its methods pass torch device
pointers and the current CUDA stream to the entry points of
:mod:`.binding`.  No arithmetic of the method happens here.
"""
from __future__ import annotations

from typing import List, Optional, Sequence

import numpy as np
import torch

from . import binding as B

_TORCH_DT = {torch.float32: "f32", torch.bfloat16: "bf16", torch.float16: "f16", torch.float64: "f64"}


def factor_ld(R: int) -> int:
    """Row stride (elements) the library expects for rank R: a multiple of 8."""
    return max(8, (R + 7) // 8 * 8)


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


class SparseTensor:
    """A COO tensor resident on the current CUDA device.

    ``idx`` is (d, P) int32 and ``vals`` (P,) float32, either numpy arrays
    (host; copied by the library) or CUDA torch tensors (device; copied)."""

    def __init__(self, idx, vals, dims: Sequence[int], coalesce: bool = False):
        self.dims = [int(x) for x in dims]
        d = len(self.dims)
        flags = B.SPT_COALESCE if coalesce else 0
        if isinstance(idx, torch.Tensor):
            assert idx.is_cuda and idx.dtype == torch.int32 and vals.dtype == torch.float32
            idx = idx.contiguous()
            vals = vals.contiguous()
            ptrs = [idx[m].data_ptr() for m in range(d)]
            vptr = vals.data_ptr()
            flags |= B.SPT_DEVICE_PTRS
            keep = (idx, vals)
        else:
            idx = np.ascontiguousarray(idx, dtype=np.int32)
            vals = np.ascontiguousarray(vals, dtype=np.float32)
            ptrs = [idx[m].ctypes.data for m in range(d)]
            vptr = vals.ctypes.data
            keep = (idx, vals)
        nnz = int(vals.shape[0])
        self.handle = B.tensor_create_coo(d, self.dims, nnz, ptrs, vptr, flags, _stream())
        del keep
        _, _, self.nnz, fl = B.tensor_info(self.handle)
        self.coalesced = bool(fl & B.SPT_COALESCE)
        self.order = d

    @classmethod
    def from_handle(cls, handle: int, dims: Sequence[int]) -> "SparseTensor":
        """Wrap a library tensor handle (e.g. from tensor_create_shard); the
        wrapper owns it and destroys it on close()."""
        self = cls.__new__(cls)
        self.handle = handle
        self.dims = [int(x) for x in dims]
        self.order, _, self.nnz, fl = B.tensor_info(handle)
        self.coalesced = bool(fl & B.SPT_COALESCE)
        return self

    def close(self):
        if getattr(self, "handle", None):
            B.tensor_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build_permutation(self, mode: int = -1, index_only: bool = False, slice_order: bool = False):
        """perm_n and (unless index_only) the mode-sorted copy; slice_order
        orders each slice of the copy by the next modes (SPT_PERM_SLICE_ORDER)."""
        flags = (B.SPT_PERM_INDEX_ONLY if index_only else 0) | (B.SPT_PERM_SLICE_ORDER if slice_order else 0)
        B.build_mode_permutation(self.handle, mode, flags, _stream())

    def storage_records(self, keep: bool = True):
        """Pack (or drop) the storage-order records the perm_n traversal reads."""
        B.tensor_storage_records(self.handle, keep, _stream())

    def build_l2_blocks(self, mode: int, blocked_mode: int = -1, block_rows: int = -1):
        """The mode's L2-blocked copy (build_mode_l2_blocks); block_rows = 0 drops it."""
        B.build_mode_l2_blocks(self.handle, mode, blocked_mode, block_rows, _stream())

    def l2_blocks(self, mode: int):
        """(blocked mode or -1, rows per block, groups) of the mode's L2-blocked copy."""
        return B.tensor_l2_blocks(self.handle, mode)

    def permutation(self, mode: int) -> torch.Tensor:
        out = torch.empty(self.nnz, dtype=torch.int32, device="cuda")
        B.tensor_get_permutation(self.handle, mode, out.data_ptr(), _stream())
        return out

    def coo(self):
        idx = torch.empty((self.order, self.nnz), dtype=torch.int32, device="cuda")
        vals = torch.empty(self.nnz, dtype=torch.float32, device="cuda")
        B.tensor_get_coo(self.handle, [idx[m].data_ptr() for m in range(self.order)],
                         vals.data_ptr(), _stream())
        return idx, vals

    def norm2(self) -> float:
        return B.tensor_norm2(self.handle)

    def check(self):
        B.tensor_check(self.handle, _stream())

    def mttkrp(self, mode: int, factors: List[Optional[torch.Tensor]], rank: int,
               lam: Optional[torch.Tensor] = None, out: Optional[torch.Tensor] = None,
               sched: Optional[B.spt_schedule] = None, deterministic: bool = False) -> torch.Tensor:
        """Mode-n MTTKRP into out (allocated if None).  deterministic=True
        runs mttkrp_deterministic: bit-identical results from call to call
        (needs build_permutation)."""
        f0 = next(f for m, f in enumerate(factors) if m != mode and f is not None) \
            if self.order > 1 else None
        ld = f0.shape[1] if f0 is not None else factor_ld(rank)
        fdt = _TORCH_DT[f0.dtype] if f0 is not None else "f32"
        if out is None:  # float64 output for fp64 factors, float32 otherwise
            out = torch.empty((self.dims[mode], ld), device="cuda",
                              dtype=torch.float64 if fdt == "f64" else torch.float32)
        ptrs = [0 if (m == mode or f is None) else f.data_ptr() for m, f in enumerate(factors)]
        fn = B.mttkrp_deterministic if deterministic else B.mttkrp
        fn(self.handle, mode, ptrs, fdt, rank, ld,
           lam.data_ptr() if lam is not None else 0, out.data_ptr(), sched, _stream())
        return out

    def mttkrp_from_host(self, modes: Sequence[int], factors: List[Optional[torch.Tensor]], rank: int,
                         outs: Optional[List[torch.Tensor]] = None, lam: Optional[torch.Tensor] = None,
                         workspace: Optional[torch.Tensor] = None, sync: bool = True) -> List[torch.Tensor]:
        """MTTKRP of `modes` from host memory (mttkrp_from_host): factors are
        CPU torch tensors (pinned ones let the copies overlap the kernels),
        outs CPU tensors (allocated pinned if None).  With sync=False the
        results are valid once the current stream has completed."""
        f0 = next(f for f in factors if f is not None)
        ld = f0.shape[1]
        fdt = _TORCH_DT[f0.dtype]
        odt = torch.float64 if fdt == "f64" else torch.float32
        if outs is None:
            outs = [torch.empty((self.dims[n], ld), dtype=odt).pin_memory() for n in modes]
        for m, f in enumerate(factors):  # the library copies dims[m] x ld elements
            if f is not None and (f.is_cuda or f.dtype != f0.dtype or not f.is_contiguous()
                                  or f.shape != (self.dims[m], ld)):
                raise ValueError(f"factor {m}: a contiguous host tensor of shape ({self.dims[m]}, {ld}) "
                                 f"and dtype {f0.dtype} is required")
        for q, n in enumerate(modes):
            o = outs[q]
            if o.is_cuda or o.dtype != odt or not o.is_contiguous() or o.shape != (self.dims[n], ld):
                raise ValueError(f"outs[{q}]: a contiguous host tensor of shape ({self.dims[n]}, {ld}) "
                                 f"and dtype {odt} is required")
        need = B.mttkrp_from_host_workspace_size(self.handle, list(modes), fdt, rank, ld)
        if workspace is None or workspace.numel() < need:
            workspace = torch.empty(need, dtype=torch.uint8, device="cuda")
        B.mttkrp_from_host(self.handle, list(modes), [f.data_ptr() if f is not None else 0 for f in factors],
                           fdt, rank, ld, lam.data_ptr() if lam is not None else 0,
                           [o.data_ptr() for o in outs], workspace.data_ptr(), workspace.numel(), _stream())
        if sync:
            torch.cuda.current_stream().synchronize()
        return outs

    def gcp_gradient(self, mode: int, factors: List[torch.Tensor], rank: int, loss: str,
                     out: Optional[torch.Tensor] = None):
        """Generalised CP loss gradient with respect to factors[mode] (all d
        factors are read); returns (grad, F) with F a 1-element float64 tensor."""
        ld = factors[0].shape[1]
        fdt = _TORCH_DT[factors[0].dtype]
        if out is None:
            out = torch.empty((self.dims[mode], ld), dtype=torch.float32, device="cuda")
        F = torch.zeros(1, dtype=torch.float64, device="cuda")
        B.gcp_gradient(self.handle, mode, [f.data_ptr() for f in factors], fdt, rank, ld, loss,
                       out.data_ptr(), F.data_ptr(), _stream())
        return out, F

    def cp_als_workspace(self, rank: int, ld: int) -> torch.Tensor:
        nbytes = B.cp_als_workspace_size(self.handle, rank, ld)
        return torch.empty(nbytes, dtype=torch.uint8, device="cuda")

    def cp_als_step(self, factors: List[torch.Tensor], rank: int, lam: torch.Tensor,
                    fit: Optional[torch.Tensor], workspace: torch.Tensor):
        ld = factors[0].shape[1]
        fdt = _TORCH_DT[factors[0].dtype]
        B.cp_als_step(self.handle, [f.data_ptr() for f in factors], fdt, rank, ld,
                      lam.data_ptr(), fit.data_ptr() if fit is not None else 0,
                      workspace.data_ptr(), workspace.numel(), _stream())
