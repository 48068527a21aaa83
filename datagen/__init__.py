"""Seeded synthetic inputs for the sorting workloads (no sorting arithmetic).

The paper benchmarks on synthetic distributions (Ch.5, "Synthetic Datasets":
Uniform, Normal, Log-Normal, Mix Gauss, Exponential, Zipf, Root Dups, Two
Dups) plus real-world sets that are not available here.  These generators
produce the synthetic ones at any size, with the shapes the workloads name:

  uniform      U[0,1): (r >> 11) * 2^-53
  normal       N(0,1) by Box-Muller
  lognormal    exp(0.5 * N(0,1))
  exponential  rate 2: -log(1-U)/2
  mixgauss     5 equal-weight Gaussians, means U[-100,100], sd U[1,10]
  zipf         Zipf(s) over 1..N by inverse CDF (s=0.75, N=1e6 by default)
  rootdups     A[i] = i mod floor(sqrt(n))
  twodups      A[i] = (i^2 + n/2) mod n
  eightdups    A[i] = i mod 8
  raw64        raw 64-bit SplitMix64 draws (integer keys)

Both the CUDA path and the oracle receive the same bytes from here.  Float
draws map to u64/u32 keys by their order-preserving totalOrder bits; the
integer-valued generators give their integers directly.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libdatagen.so")
_lock = threading.Lock()
_lib = None

DISTS = {"uniform": 0, "normal": 1, "lognormal": 2, "exponential": 3, "mixgauss": 4,
         "zipf": 5, "rootdups": 6, "twodups": 7, "eightdups": 8, "raw64": 9}
# The nine-member set used when a workload draws "a config-1 style distribution"
# per segment or request: Uniform plus the eight 2^28 single-array distributions.
NINE = ["uniform", "normal", "lognormal", "exponential", "mixgauss", "zipf",
        "rootdups", "twodups", "eightdups"]
CONFIG2 = NINE[1:]
_T = {np.dtype(np.float64): 0, np.dtype(np.float32): 1, np.dtype(np.uint64): 2,
      np.dtype(np.uint32): 3}


def build(force: bool = False) -> str:
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                        "-ffp-contract=off", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        c = ctypes
        L.datagen_fill.argtypes = [c.c_int, c.c_int, c.c_int64, c.c_uint64, c.c_double,
                                   c.c_int64, c.c_int64, c.c_int64, c.c_void_p, c.c_int]
        L.datagen_fill_segments.argtypes = [c.c_void_p, c.c_int64, c.c_void_p, c.c_uint64, c.c_int,
                                            c.c_void_p, c.c_int]
        _lib = L
    return _lib


def _threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


def generate(dist: str, n: int, dtype=np.float64, seed: int = 0, *, zipf_s: float = 0.75,
             zipf_n: int = 1_000_000, out: np.ndarray | None = None,
             lo: int = 0, hi: int | None = None) -> np.ndarray:
    """Keys [lo, hi) of the seeded stream `dist` of size n, as `dtype`."""
    dtype = np.dtype(dtype)
    hi = n if hi is None else hi
    if out is None:
        out = np.empty(hi - lo, dtype)
    assert out.dtype == dtype and out.size == hi - lo and out.flags.c_contiguous
    rc = _load().datagen_fill(DISTS[dist], _T[dtype], n, seed & (2**64 - 1), zipf_s, zipf_n,
                              lo, hi, out.ctypes.data_as(ctypes.c_void_p), _threads())
    if rc != 0:
        raise ValueError(f"datagen: bad arguments for {dist}")
    return out


def config1(n: int = 1 << 20, seed: int = 0) -> np.ndarray:
    """Single f64 array, i.i.d. U[0,1)."""
    return generate("uniform", n, np.float64, seed)


def config2(dist: str, n: int = 1 << 28, seed: int | None = None) -> np.ndarray:
    """Single f64 array of one of the eight distributions (seeds 1..8)."""
    s = CONFIG2.index(dist) + 1 if seed is None else seed
    return generate(dist, n, np.float64, s)


def config3(kind: str, n: int | None = None, seed: int = 11) -> np.ndarray:
    """Integer/f32 arrays: u64 uniform over 2^64, u32 Zipf(1.0) over 1..2^24,
    f32 N(0,1)."""
    if kind == "u64":
        return generate("raw64", n or (1 << 30), np.uint64, seed)
    if kind == "u32":
        return generate("zipf", n or (1 << 30), np.uint32, seed, zipf_s=1.0, zipf_n=1 << 24)
    if kind == "f32":
        return generate("normal", n or (1 << 29), np.float32, seed)
    raise ValueError(kind)


def segment_sizes(count: int = 200_000, median: float = 2048.0, sigma: float = 1.5,
                  lo: int = 16, hi: int = 4_194_304, seed: int = 4) -> np.ndarray:
    """Segment sizes LogNormal(ln median, sigma) clamped to [lo, hi]."""
    z = generate("normal", count, np.float64, seed)
    s = np.rint(np.exp(np.log(median) + sigma * z))
    return np.clip(s, lo, hi).astype(np.int64)


def segmented(sizes: np.ndarray, seed: int = 4, dtype=np.float64):
    """Concatenated segments, each from one of the nine distributions chosen
    uniformly per segment; index formulas use segment-local i and size."""
    sizes = np.asarray(sizes, np.int64)
    offsets = np.zeros(sizes.size + 1, np.int64)
    np.cumsum(sizes, out=offsets[1:])
    keys = np.empty(int(offsets[-1]), np.dtype(dtype))
    pick = generate("raw64", sizes.size, np.uint64, seed ^ 0xabcdef)
    dist_ix = (pick % np.uint64(len(NINE))).astype(np.int64)
    codes = np.array([DISTS[NINE[i]] for i in dist_ix], np.int32)
    rc = _load().datagen_fill_segments(offsets.ctypes.data_as(ctypes.c_void_p), sizes.size,
                                       codes.ctypes.data_as(ctypes.c_void_p), seed & (2**64 - 1),
                                       _T[np.dtype(dtype)], keys.ctypes.data_as(ctypes.c_void_p),
                                       _threads())
    if rc != 0:
        raise ValueError("datagen: bad segment arguments")
    return keys, offsets, dist_ix
