"""ctypes binding of the C ABI in include/ipls.h (argument marshalling only).

Every function here forwards to the CUDA library libipls.so; nothing is
computed in Python.  Loading fails loudly when the library is missing: there
is no CPU fallback.  Tensors are torch CUDA tensors (device memory, streams);
the raw ``iplsXxx`` functions take plain integers (pointers) like the C ABI.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

F64, F32, U64, U32 = 0, 1, 2, 3
IPLS_OK, IPLS_PENDING = 0, 1
STATUS_NAMES = {0: "IPLS_OK", 1: "IPLS_PENDING", -1: "IPLS_ERR_ARG", -2: "IPLS_ERR_OOM",
                -3: "IPLS_ERR_CUDA", -4: "IPLS_ERR_TIMEOUT", -5: "IPLS_ERR_BUDGET",
                -6: "IPLS_ERR_INTERNAL"}


class iplsConfig(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("cutoff", ctypes.c_int32),
                ("root_sample", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("sync", ctypes.c_int32), ("exact_only", ctypes.c_int32),
                ("spin_limit", ctypes.c_int64), ("trace_cap", ctypes.c_int64),
                ("budget_bytes", ctypes.c_int64), ("profile", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("pl2_leaves", ctypes.c_int32), ("serve_slots", ctypes.c_int32),
                ("pl2_depth", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]

FLAG_THRESHOLD_INDEX = 1
FLAG_GRAPH = 2


class iplsKernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double), ("bytes", ctypes.c_int64)]


class iplsBatchRec(ctypes.Structure):
    _fields_ = [("first_ticket", ctypes.c_uint64), ("requests", ctypes.c_int32),
                ("slot", ctypes.c_int32), ("keys", ctypes.c_int64), ("dtype", ctypes.c_int32),
                ("status", ctypes.c_int32), ("start_ms", ctypes.c_double), ("end_ms", ctypes.c_double)]


class iplsLevelStat(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int32), ("pad", ctypes.c_int32), ("launches", ctypes.c_int64),
                ("keys", ctypes.c_int64), ("grid_ms", ctypes.c_double), ("bytes", ctypes.c_int64)]


class iplsTraceRec(ctypes.Structure):
    _fields_ = [("off", ctypes.c_int64), ("n", ctypes.c_int64), ("level", ctypes.c_int32),
                ("kind", ctypes.c_int32), ("capped", ctypes.c_int32),
                ("nbuckets", ctypes.c_int32), ("S", ctypes.c_int64), ("D", ctypes.c_int64),
                ("A", ctypes.c_double), ("Bc", ctypes.c_double), ("ud", ctypes.c_double),
                ("xlo_bits", ctypes.c_uint64), ("nsplit", ctypes.c_int32),
                ("where", ctypes.c_int32), ("counts", ctypes.c_int64 * 256)]


class iplsStats(ctypes.Structure):
    _fields_ = [("calls", ctypes.c_int64), ("grid_levels", ctypes.c_int64),
                ("grid_passes", ctypes.c_int64), ("keys_partitioned", ctypes.c_int64),
                ("resident_groups", ctypes.c_int64), ("fallback_passes", ctypes.c_int64),
                ("algorithmic_bytes", ctypes.c_int64), ("scratch_bytes", ctypes.c_int64),
                ("trace_records", ctypes.c_int64), ("max_bucket_frac", ctypes.c_double),
                ("slow_tasks", ctypes.c_int64), ("slow_passes", ctypes.c_int64),
                ("sweep_tasks", ctypes.c_int64)]


_lib = None
SYMBOLS = ["iplsDefaultConfig", "iplsCreate", "iplsDestroy", "iplsScratchBytes", "iplsSort",
           "iplsSortSegmented", "iplsSortHost", "iplsSortHostBatch", "iplsSubmit", "iplsPoll", "iplsWait",
           "iplsGetStats", "iplsGetKernelStats", "iplsGetLevelStats", "iplsGetTrace",
           "iplsGetTraceKnots",
           "iplsPL2LossGrad", "iplsSortSmallNoAlloc", "iplsSortBatch", "iplsGetBatchLog",
           "iplsLastError"]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libipls.so (building it with nvcc if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libipls.so not found at {path}: build it with "
                           "paper_2208_06902_gb300.build.build()")
    L = ctypes.CDLL(path)
    c = ctypes
    P = c.c_void_p
    L.iplsDefaultConfig.argtypes = [c.POINTER(iplsConfig)]
    L.iplsCreate.argtypes = [c.POINTER(P), c.POINTER(iplsConfig), P, P, P, P]
    L.iplsDestroy.argtypes = [P]
    L.iplsScratchBytes.argtypes = [P, c.c_int64, c.c_int, c.POINTER(c.c_size_t)]
    L.iplsSort.argtypes = [P, P, c.c_int64, c.c_int]
    L.iplsSortSegmented.argtypes = [P, P, P, c.c_int64, c.c_int]
    L.iplsSortHost.argtypes = [P, P, c.c_int64, c.c_int]
    L.iplsSortBatch.argtypes = [P, P, P, c.c_int64, c.c_int]
    L.iplsSortHostBatch.argtypes = [P, P, P, c.c_int64, c.c_int]
    L.iplsGetBatchLog.argtypes = [P, c.POINTER(iplsBatchRec), c.c_int64, c.POINTER(c.c_int64)]
    L.iplsSortSmallNoAlloc.argtypes = [P, c.c_int64, c.c_int, c.POINTER(iplsConfig), P]
    L.iplsGetKernelStats.argtypes = [P, c.POINTER(iplsKernelStat), c.c_int32,
                                     c.POINTER(c.c_int32), c.c_int32]
    L.iplsGetLevelStats.argtypes = [P, c.POINTER(iplsLevelStat), c.c_int32,
                                    c.POINTER(c.c_int32), c.c_int32]
    L.iplsSubmit.argtypes = [P, P, c.c_int64, c.c_int, c.POINTER(c.c_uint64)]
    L.iplsPoll.argtypes = [P, c.c_uint64]
    L.iplsWait.argtypes = [P, c.c_uint64, c.c_int64]
    L.iplsGetStats.argtypes = [P, c.POINTER(iplsStats)]
    L.iplsGetTrace.argtypes = [P, P, c.c_int64, c.POINTER(c.c_int64)]
    L.iplsGetTraceKnots.argtypes = [P, P, c.c_int64, c.POINTER(c.c_int64)]
    L.iplsPL2LossGrad.argtypes = [P, c.c_int64, c.c_int, c.c_int32, P, P, P]
    L.iplsLastError.restype = c.c_char_p
    for name in SYMBOLS:
        if name != "iplsLastError":
            getattr(L, name).restype = c.c_int
    _lib = L
    return L


class IPLSError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = load().iplsLastError().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} ({msg})")
        self.status = status


def _check(st: int, where: str) -> int:
    if st < 0:
        raise IPLSError(st, where)
    return st


# ---- raw C-ABI functions (same names, integer pointers) -------------------
def iplsDefaultConfig() -> iplsConfig:
    cfg = iplsConfig()
    _check(load().iplsDefaultConfig(ctypes.byref(cfg)), "iplsDefaultConfig")
    return cfg


def iplsCreate(cfg: iplsConfig | None = None, stream: int = 0) -> int:
    ctx = ctypes.c_void_p()
    _check(load().iplsCreate(ctypes.byref(ctx), ctypes.byref(cfg) if cfg is not None else None,
                             None, None, None, ctypes.c_void_p(stream)), "iplsCreate")
    return ctx.value


def iplsDestroy(ctx: int) -> None:
    _check(load().iplsDestroy(ctypes.c_void_p(ctx)), "iplsDestroy")


def iplsScratchBytes(ctx: int | None, n: int, dtype: int) -> int:
    b = ctypes.c_size_t()
    _check(load().iplsScratchBytes(ctypes.c_void_p(ctx), n, dtype, ctypes.byref(b)),
           "iplsScratchBytes")
    return b.value


def iplsSort(ctx: int | None, keys_ptr: int, n: int, dtype: int) -> int:
    return _check(load().iplsSort(ctypes.c_void_p(ctx), ctypes.c_void_p(keys_ptr), n, dtype),
                  "iplsSort")


def iplsSortSmallNoAlloc(keys_ptr: int, n: int, dtype: int, cfg: iplsConfig | None = None,
                         stream: int = 0) -> int:
    """Sorts at most 8192 device keys in place without allocating memory
    (one block, the library's static status block as its only scratch)."""
    return _check(load().iplsSortSmallNoAlloc(ctypes.c_void_p(keys_ptr), n, dtype,
                                              ctypes.byref(cfg) if cfg is not None else None,
                                              ctypes.c_void_p(stream)), "iplsSortSmallNoAlloc")


def iplsSortSegmented(ctx: int | None, keys_ptr: int, offsets_ptr: int, nseg: int,
                      dtype: int) -> int:
    return _check(load().iplsSortSegmented(ctypes.c_void_p(ctx), ctypes.c_void_p(keys_ptr),
                                           ctypes.c_void_p(offsets_ptr), nseg, dtype),
                  "iplsSortSegmented")


def iplsSortBatch(ctx: int | None, ptrs, sizes, dtype: int) -> int:
    """Sorts len(ptrs) separate device arrays in place, each ptrs[i] holding
    sizes[i] keys (one batched sort, each array in its own memory)."""
    m = len(ptrs)
    P = (ctypes.c_void_p * max(m, 1))(*[ctypes.c_void_p(p) for p in ptrs])
    N = (ctypes.c_int64 * max(m, 1))(*[int(x) for x in sizes])
    return _check(load().iplsSortBatch(ctypes.c_void_p(ctx), P, N, m, dtype), "iplsSortBatch")


def iplsSortHostBatch(ctx: int | None, ptrs, sizes, dtype: int) -> int:
    """Sorts len(ptrs) separate host arrays in place, each ptrs[i] holding
    sizes[i] keys, with the copies in and out overlapped with the sorts."""
    m = len(ptrs)
    P = (ctypes.c_void_p * max(m, 1))(*[ctypes.c_void_p(p) for p in ptrs])
    N = (ctypes.c_int64 * max(m, 1))(*[int(x) for x in sizes])
    return _check(load().iplsSortHostBatch(ctypes.c_void_p(ctx), P, N, m, dtype), "iplsSortHostBatch")


def iplsGetBatchLog(ctx: int, cap: int = 65536) -> list:
    out = (iplsBatchRec * max(cap, 1))()
    cnt = ctypes.c_int64()
    _check(load().iplsGetBatchLog(ctypes.c_void_p(ctx), out, cap, ctypes.byref(cnt)), "iplsGetBatchLog")
    return [dict(first_ticket=r.first_ticket, requests=r.requests, slot=r.slot, keys=r.keys,
                 dtype=r.dtype, status=r.status, start_ms=r.start_ms, end_ms=r.end_ms)
            for r in out[: cnt.value]]


def iplsSortHost(ctx: int | None, host_ptr: int, n: int, dtype: int) -> int:
    return _check(load().iplsSortHost(ctypes.c_void_p(ctx), ctypes.c_void_p(host_ptr), n, dtype),
                  "iplsSortHost")


def iplsGetKernelStats(ctx: int, reset: bool = False) -> list:
    out = (iplsKernelStat * 32)()
    cnt = ctypes.c_int32()
    _check(load().iplsGetKernelStats(ctypes.c_void_p(ctx), out, 32, ctypes.byref(cnt),
                                     1 if reset else 0), "iplsGetKernelStats")
    return [dict(name=r.name.decode(), launches=r.launches, total_ms=r.total_ms,
                 bytes=r.bytes) for r in out[: cnt.value]]


def iplsGetLevelStats(ctx: int, reset: bool = False) -> list:
    out = (iplsLevelStat * 16)()
    cnt = ctypes.c_int32()
    _check(load().iplsGetLevelStats(ctypes.c_void_p(ctx), out, 16, ctypes.byref(cnt),
                                    1 if reset else 0), "iplsGetLevelStats")
    return [dict(level=r.level, launches=r.launches, keys=r.keys, grid_ms=r.grid_ms,
                 bytes=r.bytes) for r in out[: cnt.value]]


def iplsSubmit(ctx: int, keys_ptr: int, n: int, dtype: int) -> int:
    t = ctypes.c_uint64()
    _check(load().iplsSubmit(ctypes.c_void_p(ctx), ctypes.c_void_p(keys_ptr), n, dtype,
                             ctypes.byref(t)), "iplsSubmit")
    return t.value


def iplsPoll(ctx: int, ticket: int) -> int:
    return _check(load().iplsPoll(ctypes.c_void_p(ctx), ticket), "iplsPoll")


def iplsWait(ctx: int, ticket: int, timeout_us: int = -1) -> int:
    return _check(load().iplsWait(ctypes.c_void_p(ctx), ticket, timeout_us), "iplsWait")


def iplsGetStats(ctx: int) -> iplsStats:
    s = iplsStats()
    _check(load().iplsGetStats(ctypes.c_void_p(ctx), ctypes.byref(s)), "iplsGetStats")
    return s


TRACE_DTYPE = None


def trace_dtype():
    """numpy structured dtype with the layout of iplsTraceRec."""
    import numpy as np
    global TRACE_DTYPE
    if TRACE_DTYPE is None:
        TRACE_DTYPE = np.dtype(iplsTraceRec)
    return TRACE_DTYPE


def iplsGetTrace(ctx: int, cap: int, as_array: bool = False):
    """The trace records of the last sort: a list of iplsTraceRec, or with
    as_array a numpy structured array of that layout."""
    import numpy as np
    out = np.zeros(max(cap, 1), trace_dtype())
    cnt = ctypes.c_int64()
    _check(load().iplsGetTrace(ctypes.c_void_p(ctx), ctypes.c_void_p(out.ctypes.data), cap,
                               ctypes.byref(cnt)), "iplsGetTrace")
    arr = out[: cnt.value]
    if as_array:
        return arr
    return [iplsTraceRec.from_buffer_copy(r.tobytes()) for r in arr]


def iplsGetTraceKnots(ctx: int, cap: int, leaves: int):
    """PL2 knots of the grid-level trace records: array (records, leaves + 1)."""
    import numpy as np
    out = np.zeros((max(cap, 1), leaves + 1), np.float32)
    cnt = ctypes.c_int64()
    _check(load().iplsGetTraceKnots(ctypes.c_void_p(ctx), ctypes.c_void_p(out.ctypes.data), cap,
                                    ctypes.byref(cnt)), "iplsGetTraceKnots")
    return out[: cnt.value]


def iplsPL2LossGrad(sample_ptr: int, S: int, dtype: int, leaves: int, knots_ptr: int,
                    out_ptr: int, stream: int = 0) -> int:
    """Device PL2 loss and gradient (see include/ipls.h); all pointers are
    device pointers, out holds 2*(leaves+1)+2 floats."""
    return _check(load().iplsPL2LossGrad(ctypes.c_void_p(sample_ptr), S, dtype, leaves,
                                         ctypes.c_void_p(knots_ptr), ctypes.c_void_p(out_ptr),
                                         ctypes.c_void_p(stream)), "iplsPL2LossGrad")


def iplsLastError() -> str:
    return load().iplsLastError().decode(errors="replace")


# ---- tensor conveniences ---------------------------------------------------
def dtype_code(t) -> int:
    import torch
    m = {torch.float64: F64, torch.float32: F32, torch.uint64: U64, torch.uint32: U32,
         torch.int64: U64, torch.int32: U32}
    if t.dtype not in m:
        raise TypeError(f"unsupported dtype {t.dtype}")
    return m[t.dtype]


class Context:
    """Owns an iplsCtx bound to a CUDA stream (default: torch's current)."""

    def __init__(self, *, k: int = 256, cutoff: int = 32, root_sample: int = 0, seed: int = 0,
                 exact_only: bool = False, trace_cap: int = 0, spin_limit: int | None = None,
                 stream=None, budget_bytes: int = 0, profile: bool = False, flags: int = 0,
                 max_batch: int = 0, pl2_leaves: int = 0, serve_slots: int = 0,
                 pl2_depth: int = 1):
        import torch
        cfg = iplsDefaultConfig()
        cfg.k, cfg.cutoff, cfg.root_sample, cfg.seed = k, cutoff, root_sample, seed
        cfg.exact_only = 1 if exact_only else 0
        cfg.trace_cap = trace_cap
        cfg.budget_bytes = budget_bytes
        cfg.profile = 1 if profile else 0
        cfg.flags = flags
        cfg.max_batch = max_batch
        cfg.pl2_leaves = pl2_leaves
        cfg.serve_slots = serve_slots
        cfg.pl2_depth = pl2_depth
        if spin_limit is not None:
            cfg.spin_limit = spin_limit
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        self.ctx = iplsCreate(cfg, s.cuda_stream)
        self.trace_cap = trace_cap
        self.pl2_leaves = pl2_leaves

    def submit_ptr(self, ptr: int, n: int, dtype: int) -> int:
        """Queues an asynchronous sort of n device keys; returns its ticket."""
        return iplsSubmit(self.ctx, ptr, n, dtype)

    def poll(self, ticket: int) -> int:
        """PENDING (1) while the request runs, then 0 (errors raise)."""
        return iplsPoll(self.ctx, ticket)

    def wait(self, ticket: int, timeout_us: int = -1) -> int:
        return iplsWait(self.ctx, ticket, timeout_us)

    def sort_(self, keys) -> None:
        """Sorts a contiguous CUDA tensor in place."""
        assert keys.is_cuda and keys.is_contiguous()
        iplsSort(self.ctx, keys.data_ptr(), keys.numel(), dtype_code(keys))

    def sort_ptr(self, ptr: int, n: int, dtype: int) -> None:
        iplsSort(self.ctx, ptr, n, dtype)

    def sort_segmented_(self, keys, offsets) -> None:
        """Sorts keys[offsets[i]:offsets[i+1]] for each i (offsets: int64 CUDA tensor)."""
        import torch
        assert offsets.is_cuda and offsets.dtype == torch.int64 and offsets.is_contiguous()
        iplsSortSegmented(self.ctx, keys.data_ptr(), offsets.data_ptr(), offsets.numel() - 1,
                          dtype_code(keys))

    def sort_batch_ptrs(self, ptrs, sizes, dtype: int) -> None:
        iplsSortBatch(self.ctx, ptrs, sizes, dtype)

    def batch_log(self) -> list:
        return iplsGetBatchLog(self.ctx)

    def sort_host_ptr(self, host_ptr: int, n: int, dtype: int) -> None:
        iplsSortHost(self.ctx, host_ptr, n, dtype)

    def sort_host_batch_ptrs(self, ptrs, sizes, dtype: int) -> None:
        iplsSortHostBatch(self.ctx, ptrs, sizes, dtype)

    def stats(self) -> iplsStats:
        return iplsGetStats(self.ctx)

    def kernel_stats(self, reset: bool = False) -> list:
        return iplsGetKernelStats(self.ctx, reset)

    def level_stats(self, reset: bool = False) -> list:
        return iplsGetLevelStats(self.ctx, reset)

    def trace(self, as_array: bool = False):
        return iplsGetTrace(self.ctx, self.trace_cap, as_array)

    def trace_knots(self):
        return iplsGetTraceKnots(self.ctx, self.trace_cap, self.pl2_leaves)

    def close(self) -> None:
        if getattr(self, "ctx", None):
            iplsDestroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
