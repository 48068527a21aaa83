"""Segments of the block-resident base case that hold copies of one key keep
their places instead of being ranked by counting (any order of equal keys
gives the same bytes).  These arrays fill tail tasks of both kernel sizes
with buckets and eighths of 9 to 256 copies of one key next to mixed ones,
on packed and on full words, and compare the sorted bytes and every
partition pass with the oracle."""
import numpy as np
import pytest

import oracle
from gpu_util import compare_traces, gpu_sort

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2208_06902_gb300 as p
    p.load()


def _copies(values, rng, lo, hi):
    """Each value repeated between lo and hi times, shuffled."""
    reps = rng.integers(lo, hi + 1, values.size)
    out = np.repeat(values, reps)
    rng.shuffle(out)
    return out


def _array(name, dtype, n, seed):
    rng = np.random.default_rng(seed)
    if name == "zipf":
        # Zipf(0.75) over 20,000 integers: from about 20 to about 30,000
        # copies of each value
        v = np.arange(1, 20_001, dtype=np.float64)
        p = v ** -0.75
        x = rng.choice(v, size=n, p=p / p.sum())
    elif name == "runs":
        # runs of 1 to 300 copies of consecutive integers
        x = _copies(np.arange(n // 150, dtype=np.float64), rng, 1, 300)[:n]
    elif name == "mixed_runs":
        # two thirds runs of 9 to 256 copies, one third distinct values in between
        r = _copies(np.arange(0, 2 * n // 130, 2, dtype=np.float64), rng, 9, 256)[: 2 * n // 3]
        d = rng.integers(0, 2 * n // 130, n - r.size).astype(np.float64) * 2 + 1 + rng.random(n - r.size)
        x = np.concatenate([r, d])
        rng.shuffle(x)
    elif name == "wide_runs":
        # copies of values spread over the whole 64-bit range (full words)
        x = _copies(rng.integers(0, 2**63, n // 100, dtype=np.uint64) * np.uint64(2), rng, 9, 200)[:n]
    else:
        raise KeyError(name)
    if dtype in (np.uint64, np.uint32) and name != "wide_runs":
        x = x.astype(np.uint64)
    if name == "wide_runs" and dtype == np.uint32:
        x = x >> np.uint64(32)
    if name == "wide_runs" and dtype in (np.float64, np.float32):
        x = x.view(np.float64) if dtype == np.float64 else (x >> np.uint64(32)).astype(np.uint32).view(np.float32)
        x = np.where(np.isfinite(x), x, 0)
    return np.ascontiguousarray(x.astype(dtype))


# about 600,000 keys: level-0 buckets of about 2,300 keys (the 256-thread
# tail kernel); about 1,500,000: buckets of about 5,900 (the 512-thread one)
@pytest.mark.parametrize("n", [600_011, 1_500_007])
@pytest.mark.parametrize("dtype", [np.float64, np.float32, np.uint64, np.uint32])
@pytest.mark.parametrize("name", ["zipf", "runs", "mixed_runs", "wide_runs"])
def test_tail_copies_equal_the_oracle(name, dtype, n):
    x = _array(name, dtype, n, 23)
    want, recs, _ = oracle.sort(x, k=256, cutoff=256, trace_cap=400_000)
    got, ctx = gpu_sort(x, k=256, cutoff=256, trace_cap=400_000)
    assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), (name, dtype, n)
    compare_traces(ctx.trace(), recs)
