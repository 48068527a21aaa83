"""PL2 on the GPU against the oracle: the same sorted bytes, and for every
pass the same model kind, leaves and bucket counts (the device trains the
knots with the oracle's arithmetic, so the models agree bit for bit)."""
import numpy as np
import pytest

import datagen
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


def _same(a, b):
    return a.dtype == b.dtype and np.array_equal(a.view(np.uint8), b.view(np.uint8))


@pytest.mark.parametrize("leaves", [64, 1024])
@pytest.mark.parametrize("dtype", [np.float64, np.float32, np.uint64, np.uint32])
@pytest.mark.parametrize("dist", ["uniform", "normal", "lognormal", "exponential", "mixgauss",
                                  "zipf", "rootdups", "twodups"])
def test_pl2_passes_match_the_oracle(dtype, dist, leaves):
    x = datagen.generate(dist, 300_017, dtype, seed=31)
    want, recs, _ = oracle.sort(x, cutoff=64, trace_cap=100_000, pl2_leaves=leaves)
    got, ctx = gpu_sort(x, cutoff=64, trace_cap=100_000, pl2_leaves=leaves)
    assert _same(got, want)
    compare_traces(ctx.trace(), recs)
    if dist in ("uniform", "normal", "lognormal") and dtype in (np.float64, np.float32):
        assert any(r.kind == 2 for r in ctx.trace())


@pytest.mark.parametrize("leaves", [2, 16, 64, 256, 1024])
def test_pl2_grid_levels_match_the_oracle(leaves):
    x = datagen.generate("lognormal", 1 << 22, np.float64, seed=32)
    want, recs, _ = oracle.sort(x, cutoff=256, trace_cap=300_000, pl2_leaves=leaves)
    got, ctx = gpu_sort(x, cutoff=256, trace_cap=300_000, pl2_leaves=leaves)
    assert _same(got, want)
    compare_traces(ctx.trace(), recs)
    assert ctx.stats().grid_levels >= 2


def test_dense_cluster_takes_the_splitter_tree_on_the_gpu():
    rng = np.random.default_rng(2)
    n = 400_000
    x = np.concatenate([rng.uniform(0, 1, n // 2), 0.5 + rng.uniform(0, 1e-9, n // 2)])
    x = x[rng.permutation(n)]
    want, recs, _ = oracle.sort(x, cutoff=64, trace_cap=100_000, pl2_leaves=64)
    got, ctx = gpu_sort(x, cutoff=64, trace_cap=100_000, pl2_leaves=64)
    assert _same(got, want)
    compare_traces(ctx.trace(), recs)
    root = [r for r in ctx.trace() if r.level == 0][0]
    assert root.kind == 1
