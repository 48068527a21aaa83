"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a value the
paper prints, a closed form, a textbook/library routine, brute force on tiny
inputs, or an invariant.  These run without a GPU.
"""
import itertools
import math
import struct

import numpy as np
import pytest

import oracle
from conftest import load_golden

DTYPES = [np.float64, np.float32, np.uint64, np.uint32]


def _ord_py(x, dtype):
    """IEEE totalOrder key written from the standard's definition."""
    if dtype == np.float64:
        (b,) = struct.unpack("<Q", struct.pack("<d", float(x)))
        return (2**64 - 1 - b) if b >> 63 else b | (1 << 63)
    if dtype == np.float32:
        (b,) = struct.unpack("<I", struct.pack("<f", float(x)))
        return (2**32 - 1 - b) if b >> 31 else b | (1 << 31)
    return int(x)


# --------------------------------------------------------------------------
# Ch.4 worked example (golden file transcribed from the paper's tables)
# --------------------------------------------------------------------------
def test_worked_example_model_and_buckets():
    g = load_golden("worked_example.txt")
    k = int(g["k"][0])
    a, b = float(g["a"][0]), float(g["b"][0])
    x = np.array([float(v) for v in g["input"]])
    # the paper's model floor(a*x + b) is the centred form with x_lo = 0
    m = oracle.linear_model(a, b, k)
    assert oracle.classify(np.array([float(g["probe_key"][0])]), m)[0] == int(g["probe_bucket"][0])
    dst, counts = oracle.partition_with_model(x, m)
    assert counts.tolist() == [int(v) for v in g["bucket_sizes"]]
    # the contiguous-bucket table of the paper equals a stable scatter
    assert dst.tolist() == [float(v) for v in g["contiguous"]]


def test_worked_example_base_case():
    g = load_golden("worked_example.txt")
    k = int(g["k"][0])
    m = oracle.linear_model(float(g["a"][0]), float(g["b"][0]), k)
    x = np.array([float(v) for v in g["input"]])
    dst, counts = oracle.partition_with_model(x, m)
    below = int(g["base_case_below"][0])
    out, pos = [], 0
    for c in counts:
        assert c < below  # every bucket goes to the base case, as in the paper
        s, _, levels = oracle.sort(dst[pos:pos + c], cutoff=below - 1)
        assert levels <= 1
        out += s.tolist()
        pos += c
    assert out == [float(v) for v in g["sorted"]]


# --------------------------------------------------------------------------
# Sampling (SplitMix64) and the sample-size reading
# --------------------------------------------------------------------------
def test_splitmix64_published_outputs():
    # SplitMix64 seeded with 0: the first four outputs of the published
    # reference generator (Steele, Lea and Flood 2014; Vigna's splitmix64.c).
    g = 0x9E3779B97F4A7C15
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    assert [oracle.mix64((g * (i + 1)) % 2**64) for i in range(4)] == want


def test_sample_size_reading():
    # alpha = 0.2*floor(log2 n), S = alpha*k - 1 with k = 256 (Ch.4)
    assert oracle.sample_size(1 << 28, 1) == 1432
    assert oracle.sample_size(1 << 20, 1) == 1023
    assert oracle.sample_size(4096, 3) == 613
    assert oracle.sample_size(1 << 20, 0, root_sample=1 << 14) == 1 << 14
    assert oracle.sample_size(1 << 20, 1, root_sample=1 << 14) == 1023
    assert oracle.sample_size(5, 2, k=4) == 3  # never below 3
    for n in [33, 100, 4097, 10**6, 2**40]:
        L = int(math.floor(math.log2(n)))
        assert oracle.sample_size(n, 1) == max(3, (L * 256) // 5 - 1)


def test_sample_indices_range_and_spread():
    off, n = 12345, 1000
    idx = oracle.sample_indices(7, off, n, 2, 200_000)
    assert idx.min() >= off and idx.max() < off + n
    hist = np.bincount(idx - off, minlength=n)
    # with-replacement uniform draws: chi-square with n-1 dof, very loose bound
    chi2 = ((hist - 200.0) ** 2 / 200.0).sum()
    assert 800 < chi2 < 1200
    a = oracle.sample_indices(7, off, n, 2, 50)
    assert np.array_equal(a, idx[:50])  # counter-based: a prefix of the stream
    assert not np.array_equal(a, oracle.sample_indices(7, off, n, 3, 50))
    assert not np.array_equal(a, oracle.sample_indices(8, off, n, 2, 50))
    assert not np.array_equal(a - off, oracle.sample_indices(7, off + 1, n, 2, 50) - off - 1)


# --------------------------------------------------------------------------
# The whole sort: equal to the plain definition of the result
# --------------------------------------------------------------------------
def _special(dtype):
    if dtype == np.float64:
        return np.array([0.0, -0.0, np.inf, -np.inf, 5e-324, -5e-324, 1.7976931348623157e308,
                         -1.7976931348623157e308, 1.0, -1.0], np.float64)
    if dtype == np.float32:
        return np.array([0.0, -0.0, np.inf, -np.inf, 1e-45, -1e-45, 3.4e38, -3.4e38, 1.0],
                        np.float32)
    if dtype == np.uint64:
        return np.array([0, 1, 2**64 - 1, 2**63, 2**63 - 1], np.uint64)
    return np.array([0, 1, 2**32 - 1, 2**31], np.uint32)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("dist", ["uniform", "normal", "lognormal", "exponential",
                                  "mixgauss", "zipf", "rootdups", "twodups", "eightdups"])
def test_sort_equals_totalorder_definition(dtype, dist):
    import datagen
    n = 20_000
    x = datagen.generate(dist, n, dtype, seed=5)
    x[:: 997] = np.resize(_special(dtype), x[:: 997].size)
    out, recs, levels = oracle.sort(x, trace_cap=4096)
    # (1) the textbook routine under totalOrder
    assert np.array_equal(out.view(np.uint8), oracle.std_sort(x).view(np.uint8))
    # (2) an independent Python key written from IEEE 754 totalOrder
    want = sorted(x.tolist(), key=lambda v: _ord_py(v, dtype))
    got_ord = [_ord_py(v, dtype) for v in out.tolist()]
    assert got_ord == [_ord_py(v, dtype) for v in want]
    # (3) permutation by multiset hash
    assert oracle.multiset_hash(out) == oracle.multiset_hash(x)
    assert levels >= 2 and len(recs) >= 1


def test_sort_matches_numpy_without_signed_zero():
    rng = np.random.default_rng(1)
    x = rng.standard_normal(50_000) * 1e3
    out, _, _ = oracle.sort(x)
    assert np.array_equal(out, np.sort(x))
    u = rng.integers(0, 2**64, 50_000, dtype=np.uint64)
    out, _, _ = oracle.sort(u)
    assert np.array_equal(out, np.sort(u))


def test_nan_ordering():
    x = np.array([1.0, float("nan"), -2.0, -0.0, 0.0, -float("nan"), np.inf] * 20)
    out, _, _ = oracle.sort(x, cutoff=4)
    bits = out.view(np.uint64)
    assert np.isnan(out[:20]).all() and (bits[:20] >> np.uint64(63)).all()  # -NaN first
    assert np.isnan(out[-20:]).all() and not (bits[-20:] >> np.uint64(63)).any()
    assert np.array_equal(out.view(np.uint8), oracle.std_sort(x).view(np.uint8))
    zeros = out[(out == 0)]
    assert np.signbit(zeros[:20]).all() and not np.signbit(zeros[20:]).any()


@pytest.mark.parametrize("k,cutoff", [(3, 1), (4, 1), (4, 2), (256, 1)])
def test_bruteforce_all_permutations(k, cutoff):
    base_sets = [[3.0, 1.0, 2.0, 5.0, 4.0, 0.0, 6.0], [1.0, 1.0, 2.0, 2.0, 0.0, 7.0],
                 [0.0, -0.0, 1.0, -1.0, 0.0, -0.0], [5.0] * 5 + [4.0]]
    for s in base_sets:
        for p in set(itertools.permutations(s)):
            x = np.array(p, np.float64)
            out, _, _ = oracle.sort(x, k=k, cutoff=cutoff)
            want = sorted(p, key=lambda v: _ord_py(v, np.float64))
            assert [_ord_py(v, np.float64) for v in out] == [_ord_py(v, np.float64) for v in want]


# --------------------------------------------------------------------------
# FMCD (Ch.3 "Linear Models")
# --------------------------------------------------------------------------
def _same_model(a, b):
    return (a.D == b.D and a.capped == b.capped
            and struct.pack("<d", a.ud) == struct.pack("<d", b.ud)
            and struct.pack("<d", a.A) == struct.pack("<d", b.A)
            and struct.pack("<d", a.Bc) == struct.pack("<d", b.Bc)
            and a.xlo_bits == b.xlo_bits)


@pytest.mark.parametrize("dtype", DTYPES)
def test_fmcd_definition_equals_the_one_walk_search(dtype):
    rng = np.random.default_rng(2)
    ncapped = 0
    for trial in range(1500):
        N = int(rng.integers(3, 300))
        K = int(rng.choice([3, 4, 5, 8, 16, 256]))
        kind = trial % 4
        if kind == 0:
            v = rng.integers(0, 50, N)            # many duplicates
        elif kind == 1:
            v = rng.integers(0, 10**6, N)
        elif kind == 2:                           # two clusters (capped cases)
            v = np.concatenate([rng.integers(0, 100, N // 2), 10**6 + rng.integers(0, 100, N - N // 2)])
        else:
            v = np.round(rng.exponential(1000, N))
        x = np.sort(np.asarray(v).astype(dtype))
        a, b = oracle.fmcd(x, K), oracle.fmcd_incremental(x, K)
        assert _same_model(a, b), (trial, N, K)
        ncapped += a.capped
        if trial % 10 == 0 and dtype is not np.float32:
            # minimality, checked in numpy: every D' < D has a window of D'+1
            # points narrower than u_d(D') (for float32 keys the width is a
            # binary64 difference of promoted values; numpy agrees for the
            # 64-bit types)
            xd = x.astype(np.float64) if dtype is np.float64 else None
            for Dp in range(1, int(a.D) if not a.capped else int(a.D) - 1):
                if dtype is np.float64:
                    ud = (xd[N - 1 - Dp] - xd[Dp]) / (K - 2)
                    gaps = xd[Dp:] - xd[:-Dp]
                else:
                    xi = x.astype(np.uint64)
                    ud = float(xi[N - 1 - Dp] - xi[Dp]) / (K - 2)
                    gaps = (xi[Dp:] - xi[:-Dp]).astype(np.float64)
                assert not (gaps >= ud).all(), (trial, Dp, int(a.D))
    assert ncapped > 0  # the stale-u_d branch was exercised


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("N,K", [(1024, 256), (1000, 256), (300, 16), (2000, 256),
                                 (5000, 256), (1025, 256), (1026, 256), (257, 4), (100, 3)])
def test_fmcd_closed_form_on_arithmetic_progression(dtype, N, K):
    # x_i = c + i*s, distinct: gap(i,D) = D*s and span(D) = (N-1-2D)*s, so the
    # smallest D with D*s >= span(D)/(K-2) is ceil((N-1)/K).
    for c, s in [(0, 1), (7, 3), (1000, 5)]:
        x = (c + s * np.arange(N)).astype(dtype)
        m = oracle.fmcd(x, K)
        D = -(-(N - 1) // K)
        assert m.D == D and not m.capped
        ud = (N - 1 - 2 * D) * s / (K - 2)
        assert m.ud == ud and m.A == 1.0 / ud
        assert m.xlo == c + s * D
        # centred form equals the listing's A*x + B (exact here)
        for i in [0, D, N // 2, N - 1 - D, N - 1]:
            xi = float(c + s * i)
            assert math.isclose(m.A * xi + m.B, m.A * (xi - m.xlo) + m.Bc, abs_tol=1e-9)
        if ((N - 1 - 2 * D) * s) % (K - 2) == 0:
            # exact fit: x[D] opens bucket 1 and x[N-1-D] opens bucket K-1
            b = oracle.classify(x, m)
            assert b[D] == 1 and b[D - 1] == 0 and b[N - 1 - D] == K - 1


def test_fmcd_conflict_degree_bound():
    # Without duplicates and without the 3D > N cap, every D+1 consecutive
    # sample points span at least one bucket width, so no bucket holds more
    # than D+1 sample points; and D <= N/3 gives the paper's S/3 scale.
    rng = np.random.default_rng(3)
    seen = 0
    for trial in range(400):
        N = int(rng.integers(10, 3000))
        x = np.unique(rng.standard_normal(N * 2) * rng.uniform(0.1, 1e6))[:N]
        rng.shuffle(x)
        x = np.sort(x)
        m = oracle.fmcd(x, 256)
        if m.capped:
            continue
        seen += 1
        b = oracle.classify(x, m)
        assert np.bincount(b, minlength=256).max() <= m.D + 1
        assert 3 * m.D <= N
    assert seen > 300


def test_fmcd_degenerate_takes_splitter_fallback():
    # a sample constant on [D, N-1-D] gives u_d = 0: never A = inf
    x = np.array([0.0] * 3000 + [1.0] * 10 + [-1.0] * 10)
    dst, counts, m = oracle.partition_pass(x, root_sample=200)
    assert m.kind == oracle.KIND_SPLITTER
    assert counts.max() < x.size or np.unique(x).size == 1
    assert counts.sum() == x.size
    # homogeneous input: one equality bucket holds everything
    y = np.full(500, 3.25)
    dst, counts, m = oracle.partition_pass(y)
    assert m.kind == oracle.KIND_SPLITTER and m.nsplit == 1
    assert counts.tolist() == [0, 500, 0]


# --------------------------------------------------------------------------
# Model equation (Ch.3 "Linear Models") and the pass invariants
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", DTYPES)
def test_model_is_monotone_in_total_order(dtype):
    rng = np.random.default_rng(4)
    if dtype in (np.float64, np.float32):
        x = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.integers(-30, 30, 5000),
                            _special(dtype), [np.nan, -np.nan]]).astype(dtype)
    else:
        info = np.iinfo(dtype)
        x = np.concatenate([rng.integers(0, info.max, 5000, dtype=dtype, endpoint=True),
                            _special(dtype)]).astype(dtype)
    u = oracle.total_order(x)
    xs = x[np.argsort(u, kind="stable")]
    for trial in range(20):
        samp = np.sort(rng.choice(xs[np.isfinite(xs.astype(np.float64))], 300)
                       .astype(dtype), kind="stable")
        m = oracle.fmcd(np.sort(samp), 256)
        if not (np.isfinite(m.A) and m.A > 0 and np.isfinite(m.Bc)):
            continue
        b = oracle.classify(xs, m)
        assert (np.diff(b) >= 0).all()
        assert b.min() >= 0 and b.max() <= 255


def test_nan_inf_signed_zero_buckets():
    m = oracle.linear_model(2.0, 3.0, 256)
    x = np.array([-np.nan, np.nan, -np.inf, np.inf, -0.0, 0.0, 1e308, -1e308])
    x[0] = -abs(x[0]) if not np.signbit(x[0]) else x[0]
    x[0] = np.copysign(np.nan, -1.0)
    b = oracle.classify(x, m)
    assert b.tolist() == [0, 255, 0, 255, 3, 3, 255, 0]


@pytest.mark.parametrize("dtype", DTYPES)
def test_partition_pass_invariants(dtype):
    import datagen
    for dist in ["normal", "zipf", "rootdups"]:
        x = datagen.generate(dist, 30_000, dtype, seed=9)
        dst, counts, m = oracle.partition_pass(x, off=0, level=0)
        assert counts.sum() == x.size
        assert oracle.multiset_hash(dst) == oracle.multiset_hash(x)
        u_src, u_dst = oracle.total_order(x), oracle.total_order(dst)
        b = oracle.classify(x, m)
        pos = 0
        prev_max = None
        for j, c in enumerate(counts):
            if c == 0:
                continue
            seg = u_dst[pos:pos + c]
            # stable: the bucket keeps the input order of its keys
            assert np.array_equal(seg, u_src[b == j])
            if prev_max is not None:
                assert prev_max < seg.min()  # equal keys never straddle buckets
            prev_max = seg.max()
            pos += c


def test_trace_children_cover_parent():
    import datagen
    x = datagen.config1(1 << 16)
    out, recs, levels = oracle.sort(x, root_sample=1 << 14, trace_cap=100_000)
    assert np.array_equal(out, np.sort(x))
    root = recs[0]
    assert root.level == 0 and root.model.S == 1 << 14 and root.model.kind == 0
    by_level = {}
    for r in recs:
        by_level.setdefault(r.level, []).append(r)
    # every level-1 record is one non-empty root bucket above the cutoff
    kids = sorted((r.off, r.n) for r in by_level.get(1, []))
    pos, want = 0, []
    for c in root.counts[: root.model.nbuckets]:
        if c > 32:
            want.append((pos, c))
        pos += c
    assert kids == want
