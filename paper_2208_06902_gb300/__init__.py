"""GB300-native learned sort: the learned partitioning pass of IPLS
(In-Place Parallel Learned Sort, arxiv 2208.06902) as hand-written sm_103a
CUDA kernels behind a C ABI (include/ipls.h), with this thin binding.
"""
from . import build
from .ipls import (F32, F64, U32, U64, Context, IPLSError, iplsCreate, iplsDefaultConfig,
                   iplsDestroy, iplsGetStats, iplsGetTrace, iplsLastError, iplsPoll,
                   iplsScratchBytes, iplsSort, iplsSortHost, iplsSortHostBatch, iplsSortSegmented, iplsSubmit, iplsWait,
                   iplsGetKernelStats, iplsGetTraceKnots, iplsPL2LossGrad, iplsSortBatch, iplsGetBatchLog, load)

__all__ = ["build", "load", "Context", "IPLSError", "F64", "F32", "U64", "U32",
           "iplsDefaultConfig", "iplsCreate", "iplsDestroy", "iplsScratchBytes", "iplsSort",
           "iplsSortSegmented", "iplsSortHost", "iplsSortHostBatch", "iplsSubmit", "iplsPoll", "iplsWait",
           "iplsGetStats", "iplsGetKernelStats", "iplsGetTrace", "iplsGetTraceKnots",
           "iplsPL2LossGrad", "iplsSortBatch", "iplsGetBatchLog", "iplsLastError"]
