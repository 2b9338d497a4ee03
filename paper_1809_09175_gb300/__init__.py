"""GB300 (sm_103a) sparse COO MTTKRP and CP-ALS.

Method: Phipps & Kolda, arXiv 1809.09175 -- the mode-n MTTKRP of a COO sparse
tensor (Sec. 3 eq. mttkrp), its atomic and permuted-traversal scatters
(Secs. 4-6) and the CP-ALS iteration around it (Sec. 3).  The compute runs
in ``libspt.so`` (hand-written CUDA for sm_103a behind the C ABI of
``include/spt.h``); :mod:`.binding` marshals arguments to it and
:mod:`.tensor` adds a thin torch-tensor convenience layer.
"""
from . import binding  # noqa: F401  (fails loudly if libspt.so is missing)
from .binding import *  # noqa: F401,F403
from .tensor import SparseTensor, factor_ld  # noqa: F401
from . import shard  # noqa: F401  (nonzero-sharded CP-ALS over a process group)

__all__ = ["binding", "shard", "SparseTensor", "factor_ld"] + list(binding.EXPORTED)
