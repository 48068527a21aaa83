"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Final outputs are compared bit for bit (the sorted permutation under
totalOrder is unique); pass-level parity compares, for every partition pass,
the fitted model (kind, D, A, Bc, x_lo bit for bit) and the bucket histogram.
"""
import numpy as np
import pytest

import datagen
import oracle
from gpu_util import compare_traces, from_dev, gpu_sort, gpu_sort_segmented, to_dev

pytestmark = pytest.mark.gpu

DTYPES = [np.float64, np.float32, np.uint64, np.uint32]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2208_06902_gb300 as p
    p.load()


def _same(a, b):
    return a.dtype == b.dtype and a.shape == b.shape and np.array_equal(a.view(np.uint8), b.view(np.uint8))


def test_config1_uniform_2p20_bit_exact_and_pass_parity():
    # 2^20 f64 U[0,1) seed 0, root sample 2^14, k = 256, cutoff 32
    x = datagen.config1(1 << 20, seed=0)
    want, recs, _ = oracle.sort(x, root_sample=1 << 14, cutoff=32, trace_cap=200_000)
    got, ctx = gpu_sort(x, root_sample=1 << 14, cutoff=32, trace_cap=200_000)
    assert _same(got, want)
    compare_traces(ctx.trace(), recs)
    st = ctx.stats()
    assert st.grid_levels >= 1 and st.resident_groups >= 1


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("dist", datagen.NINE)
def test_distributions_bit_exact_with_trace(dtype, dist):
    n = 300_017  # several tiles and a ragged tail
    x = datagen.generate(dist, n, dtype, seed=3)
    want, recs, _ = oracle.sort(x, trace_cap=100_000)
    got, ctx = gpu_sort(x, trace_cap=100_000)
    assert _same(got, want), dist
    compare_traces(ctx.trace(), recs)
    # every splitter-tree pass is counted once, wherever it ran
    assert ctx.stats().fallback_passes == sum(1 for r in recs if r.model.kind == 1)


@pytest.mark.parametrize("dtype", DTYPES)
def test_fast_path_equals_exact_binary64(dtype):
    x = datagen.generate("lognormal", 200_000, dtype, seed=4)
    a, ca = gpu_sort(x, trace_cap=50_000)
    b, cb = gpu_sort(x, trace_cap=50_000, exact_only=True)
    assert _same(a, b)
    ta = sorted((r.off, r.n, r.level, tuple(r.counts)) for r in ca.trace())
    tb = sorted((r.off, r.n, r.level, tuple(r.counts)) for r in cb.trace())
    assert ta == tb


def _boundary_keys(m, lo, hi, k=256):
    """Exact bucket thresholds of model m in totalOrder space, by bisection
    with the oracle's binary64 classification."""
    def ord_to_f64(u):
        u = np.asarray(u, np.uint64)
        b = np.where(u >> np.uint64(63), u & ~np.uint64(1 << 63), ~u)
        return b.view(np.float64)
    def f64_to_ord(x):
        b = np.asarray(x, np.float64).view(np.uint64)
        return np.where(b >> np.uint64(63), ~b, b | np.uint64(1 << 63))
    L = np.full(k - 1, f64_to_ord(lo), np.uint64)
    H = np.full(k - 1, f64_to_ord(hi), np.uint64)
    js = np.arange(1, k)
    for _ in range(70):
        mid = L + (H - L) // np.uint64(2)
        b = oracle.classify(ord_to_f64(mid), m)
        ge = b >= js
        H = np.where(ge, mid, H)
        L = np.where(ge, L, mid + np.uint64(1))
    t = ord_to_f64(L)
    below = ord_to_f64(L - np.uint64(1))
    return t, below


def test_keys_on_exact_bucket_boundaries():
    # Keys placed exactly on the model's bucket thresholds (and one ulp
    # below) at positions the root sample does not read: the root model is
    # unchanged and every one of those keys sits where the FP32 estimate is
    # least certain.
    n = 400_000
    x = datagen.generate("normal", n, np.float64, seed=8)
    S = oracle.sample_size(n, 0)
    idx = set(oracle.sample_indices(0, 0, n, 0, S).tolist())
    _, _, m = oracle.partition_pass(x)
    assert m.kind == 0
    t, below = _boundary_keys(m, x.min(), x.max())
    free = [i for i in range(0, n, 7) if i not in idx][: 2 * t.size * 3]
    vals = np.concatenate([t, below, t, below, t, below])
    x2 = x.copy()
    x2[np.array(free[: vals.size])] = vals
    want, recs, _ = oracle.sort(x2, trace_cap=100_000)
    assert recs[0].model.A == m.A  # same root model
    got, ctx = gpu_sort(x2, trace_cap=100_000)
    assert _same(got, want)
    compare_traces(ctx.trace(), recs)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 5, 31, 32, 33, 100, 8191, 8192, 8193, 40_977])
@pytest.mark.parametrize("dtype", [np.float64, np.uint32])
def test_sizes_and_ragged_tails(n, dtype):
    x = datagen.generate("uniform" if dtype == np.float64 else "zipf", max(n, 1), dtype, seed=n)[:n]
    got, _ = gpu_sort(x)
    assert _same(got, oracle.std_sort(x))


def test_special_values_and_duplicates():
    rng = np.random.default_rng(0)
    base = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, -np.nan, 5e-324, -5e-324,
                     1.7976931348623157e308, -1.7976931348623157e308, 1.0, -1.0])
    base[5] = np.copysign(np.nan, -1.0)
    for n in [50, 5000, 70_000]:
        x = rng.choice(base, n)
        got, _ = gpu_sort(x)
        assert _same(got, oracle.std_sort(x))
    for x in [np.full(100_000, 2.5), np.array([1.0, 2.0] * 50_000), np.arange(100_000.0)[::-1].copy(),
              np.arange(100_000.0), np.where(np.arange(200_000) % 2 == 0, 0.0, -0.0)]:
        got, _ = gpu_sort(x)
        assert _same(got, oracle.std_sort(x))


def test_extreme_integers():
    rng = np.random.default_rng(1)
    u = np.concatenate([rng.integers(0, 2**64, 100_000, dtype=np.uint64),
                        np.array([0, 1, 2**64 - 1, 2**63, 2**63 - 1] * 1000, np.uint64)])
    got, _ = gpu_sort(u)
    assert _same(got, oracle.std_sort(u))
    v = np.concatenate([rng.integers(2**64 - 5000, 2**64, 50_000, dtype=np.uint64, endpoint=False)])
    got, _ = gpu_sort(v)
    assert _same(got, oracle.std_sort(v))


@pytest.mark.parametrize("cutoff,k", [(1, 256), (3, 4), (16, 64), (200, 256), (4096, 256)])
def test_other_parameters(cutoff, k):
    x = datagen.generate("mixgauss", 120_000, np.float64, seed=cutoff)
    want, recs, _ = oracle.sort(x, k=k, cutoff=cutoff, trace_cap=200_000)
    got, ctx = gpu_sort(x, k=k, cutoff=cutoff, trace_cap=200_000)
    assert _same(got, want)
    compare_traces(ctx.trace(), recs)


@pytest.mark.parametrize("dist,dtype", [("uniform", np.float64), ("twodups", np.uint32),
                                        ("zipf", np.float32)])
def test_second_tail_sweep_matches_the_oracle(dist, dtype):
    # k = 64 and cutoff 16 on 2^22 keys: 4096 block-resident tasks of about
    # 1024 keys, whose buckets of about 16 keys are often above the cutoff
    # (some 50k children) -- those children take the second sweep, and what
    # they leave above the cutoff takes k_slow
    x = datagen.generate(dist, 1 << 22, dtype, seed=8)
    want, recs, _ = oracle.sort(x, k=64, cutoff=16, trace_cap=200_000)
    got, ctx = gpu_sort(x, k=64, cutoff=16, trace_cap=200_000)
    assert _same(got, want)
    compare_traces(ctx.trace(), recs)
    st = ctx.stats()
    assert st.sweep_tasks >= 1024
    assert st.fallback_passes == sum(1 for r in recs if r.model.kind == 1)


def test_segmented_equals_each_segment_alone():
    rng = np.random.default_rng(2)
    sizes = np.concatenate([rng.integers(0, 40, 300), rng.integers(1000, 9000, 30),
                            [0, 1, 8192, 8193, 50_000, 120_001]])
    rng.shuffle(sizes)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    x = datagen.generate("exponential", int(off[-1]), np.float64, seed=5)
    got, ctx = gpu_sort_segmented(x, off, trace_cap=100_000)
    for i in range(sizes.size):
        a, b = off[i], off[i + 1]
        assert _same(got[a:b], oracle.std_sort(x[a:b])), i
    # each segment is a level-0 subproblem keyed by its own offset
    want, recs, _ = oracle.sort_segments(x, off, trace_cap=100_000)
    assert _same(got, want)
    compare_traces(ctx.trace(), recs)


def test_repeated_calls_reuse_context():
    from paper_2208_06902_gb300 import Context
    ctx = Context()
    for seed in range(3):
        for n in [100, 300_000, 20_000]:
            x = datagen.generate("normal", n, np.float64, seed=seed)
            got, _ = gpu_sort(x, ctx=ctx)
            assert _same(got, oracle.std_sort(x))


def test_lookback_timeout_leaves_a_permutation():
    # spin_limit = 1: a chunk whose predecessor has not published yet gives
    # up at once, the level moves nothing, and its keys are restored; the
    # output must hold the input's keys, and be sorted when the call succeeds
    from paper_2208_06902_gb300 import Context, IPLSError
    x = datagen.generate("normal", 1 << 24, np.float64, seed=12)
    want = oracle.std_sort(x)
    timeouts = 0
    for trial in range(3):
        ctx = Context(spin_limit=1)
        d = to_dev(x)
        try:
            ctx.sort_ptr(d.data_ptr(), x.size, 0)
            got = from_dev(d, np.float64)
            assert _same(got, want)
        except IPLSError as e:
            assert e.status == -4
            timeouts += 1
            got = from_dev(d, np.float64)
            assert _same(oracle.std_sort(got), want)  # same multiset
        ctx.close()
    print(f"look-back timeouts in 3 trials: {timeouts}")
    # the context type still sorts correctly with a normal limit afterwards
    got, _ = gpu_sort(x)
    assert _same(got, want)

