"""Serial CPU oracle of IPLS (arxiv 2208.06902) -- test infrastructure only.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and
the oracle never imports the product library: the two share no code.

The oracle itself is plain serial C++ (``ipls_oracle.cpp``); this module
builds it with g++ and wraps its C entry points with ctypes.  Every function
cites the passage of the paper it follows; the C++ file lists the readings
taken where the paper is silent.

Parity status of each function (what pins it, in ``tests/test_oracle_pins.py``):
  * ``sort``                  -- std::sort under totalOrder, brute force over
                                 all permutations (n <= 7), multiset hash.
  * ``classify``              -- the worked example of Ch.4 (golden file),
                                 monotonicity property, NaN/inf/-0 cases.
  * ``fmcd``                  -- written from the definition; the one-walk
                                 O(S) search gives the same D, closed form on
                                 arithmetic progressions, conflict-degree
                                 bound.
  * ``partition_pass``        -- histogram sums, permutation, bucket ordering,
                                 the splitter fallback's progress guarantee.
  * ``sample_indices``        -- parity unpinned by the paper (it names no
                                 random generator); pinned only against the
                                 published SplitMix64 reference outputs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ipls_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libipls_oracle.so")
_lock = threading.Lock()
_lib = None

F64, F32, U64, U32 = 0, 1, 2, 3
_NP = {F64: np.float64, F32: np.float32, U64: np.uint64, U32: np.uint32}
_CODE = {np.dtype(np.float64): F64, np.dtype(np.float32): F32,
         np.dtype(np.uint64): U64, np.dtype(np.uint32): U32}

KIND_LINEAR, KIND_SPLITTER = 0, 1


class Cfg(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("cutoff", ctypes.c_int32),
                ("root_sample", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("pl2_leaves", ctypes.c_int32), ("pl2_depth", ctypes.c_int32)]


class Model(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("capped", ctypes.c_int32),
                ("S", ctypes.c_int64), ("D", ctypes.c_int64),
                ("A", ctypes.c_double), ("Bc", ctypes.c_double),
                ("xlo", ctypes.c_double), ("xlo_bits", ctypes.c_uint64),
                ("B", ctypes.c_double), ("ud", ctypes.c_double),
                ("nsplit", ctypes.c_int32), ("nbuckets", ctypes.c_int32),
                ("split", ctypes.c_uint64 * 128),
                ("pl2_sh", ctypes.c_int32), ("pl2_rho", ctypes.c_int32),
                ("pl2_x0", ctypes.c_int64)]


class Trace(ctypes.Structure):
    _fields_ = [("off", ctypes.c_int64), ("n", ctypes.c_int64),
                ("level", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("model", Model), ("counts", ctypes.c_int64 * 512)]


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (no FMA contraction, no fast-math)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        c = ctypes
        L.oracle_record_sizes.argtypes = [c.POINTER(c.c_int64), c.POINTER(c.c_int64)]
        L.oracle_mix64.restype = c.c_uint64
        L.oracle_mix64.argtypes = [c.c_uint64]
        L.oracle_sample_indices.restype = None
        L.oracle_sample_indices.argtypes = [c.c_uint64, c.c_int64, c.c_int64, c.c_int32,
                                            c.c_int64, c.c_void_p]
        L.oracle_sample_size.restype = c.c_int64
        L.oracle_sample_size.argtypes = [c.c_int64, c.c_int32, c.c_int32, c.c_int64]
        L.oracle_total_order.argtypes = [c.c_int, c.c_void_p, c.c_int64, c.c_void_p]
        L.oracle_fmcd.argtypes = [c.c_int, c.c_void_p, c.c_int64, c.c_int32, c.POINTER(Model)]
        L.oracle_fmcd_incremental.argtypes = [c.c_int, c.c_void_p, c.c_int64, c.c_int32,
                                              c.POINTER(Model)]
        L.oracle_classify.argtypes = [c.c_int, c.c_void_p, c.c_int64, c.POINTER(Model),
                                      c.c_void_p]
        L.oracle_partition_with_model.argtypes = [c.c_int, c.c_void_p, c.c_int64,
                                                  c.POINTER(Model), c.c_void_p, c.c_void_p]
        L.oracle_partition_pass.argtypes = [c.c_int, c.c_void_p, c.c_int64, c.c_int64,
                                            c.c_int32, c.POINTER(Cfg), c.c_void_p,
                                            c.c_void_p, c.POINTER(Model)]
        L.oracle_sort.argtypes = [c.c_int, c.c_void_p, c.c_int64, c.POINTER(Cfg),
                                  c.POINTER(Trace), c.c_int64, c.POINTER(c.c_int64),
                                  c.POINTER(c.c_int32)]
        L.oracle_sort_segments.argtypes = [c.c_int, c.c_void_p, c.c_void_p, c.c_int64,
                                           c.POINTER(Cfg), c.POINTER(Trace), c.c_int64,
                                           c.POINTER(c.c_int64), c.POINTER(c.c_int32)]
        L.oracle_std_sort.argtypes = [c.c_int, c.c_void_p, c.c_int64]
        L.oracle_pl2_fit.argtypes = [c.c_int, c.c_void_p, c.c_int64, c.c_int32, c.c_int32,
                                     c.POINTER(Model), c.c_void_p, c.c_void_p]
        L.oracle_pl2_classify.argtypes = [c.c_int, c.c_void_p, c.c_int64, c.POINTER(Model),
                                          c.c_void_p, c.c_void_p]
        L.oracle_pl2_loss_grad.argtypes = [c.c_int, c.c_void_p, c.c_int64, c.POINTER(Model),
                                           c.c_void_p, c.POINTER(c.c_double), c.c_void_p,
                                           c.c_void_p]
        L.oracle_pl2_fit_f64.argtypes = [c.c_int, c.c_void_p, c.c_int64, c.c_int32, c.c_int32,
                                         c.POINTER(Model), c.c_void_p, c.c_void_p]
        L.oracle_sort_knots.argtypes = [c.c_int, c.c_void_p, c.c_int64, c.POINTER(Cfg),
                                        c.c_void_p, c.c_int64, c.POINTER(c.c_int64),
                                        c.POINTER(c.c_int32), c.c_void_p]
        L.oracle_multiset_hash.restype = None
        L.oracle_multiset_hash.argtypes = [c.c_int, c.c_void_p, c.c_int64,
                                           c.POINTER(c.c_uint64), c.POINTER(c.c_uint64)]
        mb, tb = c.c_int64(), c.c_int64()
        L.oracle_record_sizes(c.byref(mb), c.byref(tb))
        if mb.value != c.sizeof(Model) or tb.value != c.sizeof(Trace):
            raise RuntimeError("oracle record layout mismatch")
        _lib = L
    return _lib


def _code(a: np.ndarray) -> int:
    return _CODE[a.dtype]


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def cfg(k: int = 256, cutoff: int = 32, root_sample: int = 0, seed: int = 0,
        pl2_leaves: int = 0, pl2_depth: int = 1) -> Cfg:
    return Cfg(k, cutoff, root_sample, seed, pl2_leaves, pl2_depth)


def mix64(z: int) -> int:
    """SplitMix64 finaliser (Steele, Lea and Flood 2014)."""
    return int(lib().oracle_mix64(ctypes.c_uint64(z & (2**64 - 1))))


def sample_size(n: int, level: int, k: int = 256, root_sample: int = 0) -> int:
    """S = alpha*k - 1 with alpha = 0.2*floor(log2 n) (Ch.4), at least 3."""
    return int(lib().oracle_sample_size(n, level, k, root_sample))


def sample_indices(seed: int, off: int, n: int, level: int, S: int) -> np.ndarray:
    """Sampling phase (Ch.2 IPS4o; Ch.3): S indices in [off, off+n), with replacement."""
    out = np.empty(S, np.int64)
    lib().oracle_sample_indices(seed, off, n, level, S, _ptr(out))
    return out


def total_order(keys: np.ndarray) -> np.ndarray:
    keys = np.ascontiguousarray(keys)
    out = np.empty(keys.size, np.uint64)
    lib().oracle_total_order(_code(keys), _ptr(keys), keys.size, _ptr(out))
    return out


def fmcd(sorted_sample: np.ndarray, K: int = 256) -> Model:
    """FMCD (Ch.3 "Linear Models") from its definition, binary64: the smallest
    D whose windows of D+1 sample points all span u_d(D)."""
    s = np.ascontiguousarray(sorted_sample)
    m = Model()
    if lib().oracle_fmcd(_code(s), _ptr(s), s.size, K, ctypes.byref(m)) != 0:
        raise ValueError("FMCD needs N >= 3 and K >= 3")
    return m


def fmcd_incremental(sorted_sample: np.ndarray, K: int = 256) -> Model:
    """FMCD by one walk over the window starts (the O(S) search of Ch.3);
    must equal fmcd()."""
    s = np.ascontiguousarray(sorted_sample)
    m = Model()
    if lib().oracle_fmcd_incremental(_code(s), _ptr(s), s.size, K, ctypes.byref(m)) != 0:
        raise ValueError("FMCD needs N >= 3 and K >= 3")
    return m


def linear_model(A: float, Bc: float, k: int, xlo_bits: int = 0) -> Model:
    """A linear partition model given directly (kind 0)."""
    m = Model()
    m.kind, m.A, m.Bc, m.nbuckets, m.xlo_bits = KIND_LINEAR, A, Bc, k, xlo_bits
    return m


def classify(keys: np.ndarray, m: Model) -> np.ndarray:
    """Bucket of every key: the model equation of Ch.3 (or the splitter tree,
    or a PL2 model from pl2_fit, which carries its knots)."""
    keys = np.ascontiguousarray(keys)
    out = np.empty(keys.size, np.int32)
    if m.kind == 2:
        y = np.ascontiguousarray(m.knots, np.float32)
        rc = lib().oracle_pl2_classify(_code(keys), _ptr(keys), keys.size, ctypes.byref(m),
                                       _ptr(y), _ptr(out))
    else:
        rc = lib().oracle_classify(_code(keys), _ptr(keys), keys.size, ctypes.byref(m), _ptr(out))
    if rc != 0:
        raise RuntimeError(f"oracle classify failed ({rc})")
    return out


def partition_with_model(keys: np.ndarray, m: Model):
    keys = np.ascontiguousarray(keys)
    dst = np.empty_like(keys)
    counts = np.zeros(m.nbuckets, np.int64)
    lib().oracle_partition_with_model(_code(keys), _ptr(keys), keys.size, ctypes.byref(m),
                                      _ptr(dst), _ptr(counts))
    return dst, counts


def partition_pass(keys: np.ndarray, off: int = 0, level: int = 0, k: int = 256,
                   root_sample: int = 0, seed: int = 0):
    """One IPLS pass: sample, sort, FMCD, classify, scan, stable scatter."""
    keys = np.ascontiguousarray(keys)
    dst = np.empty_like(keys)
    counts = np.zeros(512, np.int64)
    m = Model()
    c = Cfg(k, 1, root_sample, seed, 0, 0)
    rc = lib().oracle_partition_pass(_code(keys), _ptr(keys), keys.size, off, level,
                                     ctypes.byref(c), _ptr(dst), _ptr(counts),
                                     ctypes.byref(m))
    if rc != 0:
        raise ValueError(f"partition_pass failed ({rc})")
    return dst, counts[: m.nbuckets].copy(), m


TRACE_DTYPE = np.dtype(Trace)


def sort(keys: np.ndarray, k: int = 256, cutoff: int = 32, root_sample: int = 0,
         seed: int = 0, trace_cap: int = 0, pl2_leaves: int = 0, as_array: bool = False,
         knots: bool = False, pl2_depth: int = 1):
    """Whole IPLS sort (returns a sorted copy, the trace records and the depth).
    pl2_leaves > 0: subproblems above 8192 keys at levels below pl2_depth
    (0: every level) use the PL2 model.
    as_array: the trace as a numpy structured array (TRACE_DTYPE) instead of a
    list of records (for large traces).  knots: also return the PL2 knots of
    every record, an array of shape (records, pl2_leaves + 1)."""
    out = np.array(keys, copy=True)
    c = Cfg(k, cutoff, root_sample, seed, pl2_leaves, pl2_depth)
    # np.zeros leaves untouched pages unallocated: a generous cap costs nothing
    tr = np.zeros(max(trace_cap, 1), TRACE_DTYPE)
    kn = np.zeros((max(trace_cap, 1), pl2_leaves + 1), np.float32) if knots else None
    cnt = ctypes.c_int64(0)
    lv = ctypes.c_int32(0)
    rc = lib().oracle_sort_knots(_code(out), _ptr(out), out.size, ctypes.byref(c),
                                 _ptr(tr) if trace_cap > 0 else None, trace_cap,
                                 ctypes.byref(cnt), ctypes.byref(lv),
                                 _ptr(kn) if kn is not None else None)
    if rc != 0:
        raise RuntimeError(f"oracle_sort failed ({rc})")
    arr = tr[: cnt.value] if trace_cap > 0 else tr[:0]
    recs = arr if as_array else [Trace.from_buffer_copy(r.tobytes()) for r in arr]
    if knots:
        return out, recs, lv.value, kn[: cnt.value]
    return out, recs, lv.value


def sort_segments(keys: np.ndarray, offsets, k: int = 256, cutoff: int = 32,
                  root_sample: int = 0, seed: int = 0, trace_cap: int = 0, pl2_leaves: int = 0,
                  as_array: bool = False, pl2_depth: int = 1):
    """IPLS on each segment keys[off[i]:off[i+1]], each a level-0 subproblem
    keyed by its own offset (returns sorted copy, trace records, depth).
    as_array: the trace as a numpy structured array (TRACE_DTYPE)."""
    out = np.array(keys, copy=True)
    off = np.ascontiguousarray(offsets, np.int64)
    c = Cfg(k, cutoff, root_sample, seed, pl2_leaves, pl2_depth)
    tr = np.zeros(max(trace_cap, 1), TRACE_DTYPE)
    cnt = ctypes.c_int64(0)
    lv = ctypes.c_int32(0)
    rc = lib().oracle_sort_segments(_code(out), _ptr(out), _ptr(off), off.size - 1,
                                    ctypes.byref(c), ctypes.cast(_ptr(tr), ctypes.POINTER(Trace))
                                    if trace_cap > 0 else None, trace_cap, ctypes.byref(cnt),
                                    ctypes.byref(lv))
    if rc != 0:
        raise RuntimeError(f"oracle_sort_segments failed ({rc})")
    arr = tr[: cnt.value] if trace_cap > 0 else tr[:0]
    recs = arr if as_array else [Trace.from_buffer_copy(r.tobytes()) for r in arr]
    return out, recs, lv.value


PL2_STEPS = 8


def pl2_fit(sorted_sample: np.ndarray, M: int = 64, K: int = 256):
    """PL2 fitted on a sorted sample: (model, loss after each training step),
    or None when the sample's range cannot be used."""
    s = np.ascontiguousarray(sorted_sample)
    m = Model()
    losses = np.zeros(PL2_STEPS + 1, np.float64)
    knots = np.zeros(M + 1, np.float32)
    if lib().oracle_pl2_fit(_code(s), _ptr(s), s.size, M, K, ctypes.byref(m), _ptr(losses),
                            _ptr(knots)) != 0:
        return None
    m.knots = knots
    return m, losses


def pl2_knots(m: Model) -> np.ndarray:
    """The knot values y_0..y_M of a PL2 model from pl2_fit (binary32)."""
    return np.array(m.knots, np.float32)


def pl2_loss_grad(sorted_sample: np.ndarray, m: Model, y: np.ndarray, with_abs: bool = False):
    """The PL2 loss and its gradient in the knot values y (for m's leaves),
    binary64.  with_abs: also the per-knot sum of the magnitudes of the
    gradient's terms."""
    s = np.ascontiguousarray(sorted_sample)
    y = np.ascontiguousarray(y, np.float64)
    loss = ctypes.c_double(0.0)
    grad = np.zeros(y.size, np.float64)
    absg = np.zeros(y.size, np.float64)
    lib().oracle_pl2_loss_grad(_code(s), _ptr(s), s.size, ctypes.byref(m), _ptr(y),
                               ctypes.byref(loss), _ptr(grad), _ptr(absg))
    if with_abs:
        return loss.value, grad, absg
    return loss.value, grad


def pl2_fit_f64(sorted_sample: np.ndarray, M: int = 64, K: int = 256):
    """The PL2 training of pl2_fit carried out in binary64: (model, knots as
    float64, loss after each step), or None when the range cannot be used."""
    s = np.ascontiguousarray(sorted_sample)
    m = Model()
    losses = np.zeros(PL2_STEPS + 1, np.float64)
    knots = np.zeros(M + 1, np.float64)
    if lib().oracle_pl2_fit_f64(_code(s), _ptr(s), s.size, M, K, ctypes.byref(m), _ptr(losses),
                                _ptr(knots)) != 0:
        return None
    return m, knots, losses


def std_sort(keys: np.ndarray) -> np.ndarray:
    """std::sort under IEEE totalOrder (the plain definition of the result)."""
    out = np.array(keys, copy=True)
    lib().oracle_std_sort(_code(out), _ptr(out), out.size)
    return out


def multiset_hash(keys: np.ndarray):
    keys = np.ascontiguousarray(keys)
    s, x = ctypes.c_uint64(), ctypes.c_uint64()
    lib().oracle_multiset_hash(_code(keys), _ptr(keys), keys.size, ctypes.byref(s),
                               ctypes.byref(x))
    return int(s.value), int(x.value)
