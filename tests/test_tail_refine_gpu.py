"""Block-resident tasks of more than 4096 keys cut each bucket into eighths
by a refinement of the model's estimate before the base case ranks the keys.
The refinement only has to keep the keys of a bucket in order; these arrays
put keys where the estimates do not reach -- outside x_lo's binade, zeros
and values below binary32's normal range, values beyond binary32's range,
negative binades, mixed signs -- into tasks of 4097 to 8192 keys, and
compare the sorted bytes and every partition pass with the oracle."""
import numpy as np
import pytest

import oracle
from gpu_util import compare_traces, gpu_sort

pytestmark = pytest.mark.gpu

N = 1_500_007  # level-0 buckets of about 5900 keys: tasks of the large tail kernel


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2208_06902_gb300 as p
    p.load()


def _arrays(dtype, seed):
    rng = np.random.default_rng(seed)
    tiny = 1e-310 if dtype == np.float64 else 1e-40
    big = 1e300 if dtype == np.float64 else 3e38
    out = {
        # clusters on binade boundaries: most of a task in one binade, a few keys across
        "binade_edges": np.concatenate([s * (1.0 + rng.normal(0.0, 2e-3, N // 3)) for s in (0.5, 1.0, 2.0)]),
        # zeros of both signs, values around and below binary32's smallest normal
        "zeros_tiny": np.concatenate([np.zeros(N // 20), -np.zeros(N // 20),
                                      rng.normal(0.0, 1e-37, N // 4), rng.normal(0.0, 1e-35, N // 2),
                                      rng.normal(0.0, tiny, N // 20)]),
        # negative binades
        "negative": np.concatenate([-(1.0 + rng.random(N // 2)), -(2.0 + 2.0 * rng.random(N // 2))]),
        # signs mixed near zero
        "mixed_signs": rng.normal(0.0, 1e-3, N),
        # values beyond binary32's range (f64) or near its top (f32)
        "huge": np.concatenate([rng.lognormal(np.log(big), 0.5, N // 2), rng.normal(0.0, 1.0, N // 2)]),
    }
    res = {}
    for name, v in out.items():
        with np.errstate(over="ignore"):
            v = v.astype(dtype)
        if dtype == np.float32:
            v = np.where(np.isfinite(v), v, np.float32(3e38)).astype(np.float32)
        rng.shuffle(v)
        res[name] = v
    return res


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("name", ["binade_edges", "zeros_tiny", "negative", "mixed_signs", "huge"])
def test_large_tail_tasks_equal_the_oracle(dtype, name):
    x = _arrays(dtype, 11)[name]
    want, recs, _ = oracle.sort(x, k=256, cutoff=256, trace_cap=400_000)
    got, ctx = gpu_sort(x, k=256, cutoff=256, trace_cap=400_000)
    assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), name
    compare_traces(ctx.trace(), recs)
    # tasks of the large tail kernel were there
    assert any(4096 < r.n <= 8192 for r in recs)
