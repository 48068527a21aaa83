"""The tail fit sorts each task's sample by radix sort on the highest three
digits that vary first and checks that every key is at most its right
neighbour; keys that agree on those digits but differ below them send the
sample through the whole sort again.  These arrays put tight clusters far
apart, so that tail tasks span many digits while the keys of one cluster
agree on the top ones (the second sort runs), next to arrays without such
ties (the first sort suffices).  The fitted models enter every pass record,
so comparing the pass trace with the oracle checks each sorted sample."""
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


def _array(name, dtype, n, seed):
    rng = np.random.default_rng(seed)
    if name == "clusters":
        # 20,000 clusters of about 75 keys, centres spread over the type's
        # range, widths of 2^12 units (2^4 for 32-bit types)
        nc = 20_000
        if dtype in (np.uint64, np.float64):
            c = rng.integers(0, 2**62, nc, dtype=np.uint64)
            w = np.uint64(4096)
        else:
            c = rng.integers(0, 2**30, nc, dtype=np.uint64)
            w = np.uint64(16)
        x = c[rng.integers(0, nc, n)] + rng.integers(0, int(w), n).astype(np.uint64)
        if dtype == np.float64:
            return x.view(np.float64)  # positive, finite: the top two bits clear
        if dtype == np.float32:
            return (x.astype(np.uint32)).view(np.float32)
        return x.astype(dtype)
    if name == "spread":
        # keys spread evenly over the type's range: no ties on the top digits
        if dtype in (np.uint64, np.uint32):
            return rng.integers(0, np.iinfo(dtype).max, n, dtype=dtype, endpoint=True)
        return rng.normal(0.0, 1.0, n).astype(dtype)
    raise KeyError(name)


@pytest.mark.parametrize("n", [600_011, 1_500_007])
@pytest.mark.parametrize("dtype", [np.float64, np.float32, np.uint64, np.uint32])
@pytest.mark.parametrize("name", ["clusters", "spread"])
def test_tail_fit_samples_sorted_like_the_oracle(name, dtype, n):
    x = np.ascontiguousarray(_array(name, dtype, n, 31))
    want, recs, _ = oracle.sort(x, k=256, cutoff=256, trace_cap=400_000)
    got, ctx = gpu_sort(x, k=256, cutoff=256, trace_cap=400_000)
    assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), (name, dtype, n)
    compare_traces(ctx.trace(), recs)
    # block-resident tasks (fitted by the tail fit) were there
    assert any(r.level >= 1 and 256 < r.n <= 8192 for r in recs)
