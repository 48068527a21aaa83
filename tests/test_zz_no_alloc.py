"""iplsSortSmallNoAlloc: the entry point that sorts without allocating, for
callers that cannot allocate device memory while they sort (a framework
pool that holds the device's memory, a loop where cudaMalloc could stall
the device, a pipeline that must not run out of memory half-way).

It is called through the C ABI and compared with iplsSort, the existing
entry point, on the same keys, and with the oracle's definition of the
result (std::sort under totalOrder). Two calls are made back to back, since
the static status block must be cleared between them. The size limit is
checked on the host before any CUDA call.
"""
import numpy as np
import pytest

import datagen
import oracle
from gpu_util import CODE, from_dev, to_dev


def _lib():
    import paper_2208_06902_gb300 as p
    return p


def test_rejects_sizes_above_the_limit():
    p = _lib()
    p.load()
    with pytest.raises(p.IPLSError) as e:
        p.ipls.iplsSortSmallNoAlloc(0x1000, 8193, 0)
    assert e.value.status == -1 and "8192" in str(e.value)
    cfg = p.iplsDefaultConfig()
    cfg.cutoff = 2  # resident limit 1024 * (2 + 1) = 3072 keys
    with pytest.raises(p.IPLSError):
        p.ipls.iplsSortSmallNoAlloc(0x1000, 3073, 0, cfg)


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", [np.float64, np.float32, np.uint64, np.uint32])
def test_two_calls_in_a_row_equal_iplsSort(dtype):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p = _lib()
    p.load()
    stream = torch.cuda.current_stream().cuda_stream
    cases = [("normal", 8192, 11), ("zipf", 5000, 12), ("eightdups", 777, 13), ("uniform", 33, 14),
             ("twodups", 2, 15)]
    for dist, n, seed in cases:
        x = datagen.generate(dist, n, dtype, seed=seed)
        a = to_dev(x)
        b = to_dev(x)
        # first call, then a second one straight after on other keys
        p.ipls.iplsSortSmallNoAlloc(a.data_ptr(), n, CODE[np.dtype(dtype)], None, stream)
        y = datagen.generate(dist, n, dtype, seed=seed + 100)
        a2 = to_dev(y)
        b2 = to_dev(y)
        p.ipls.iplsSortSmallNoAlloc(a2.data_ptr(), n, CODE[np.dtype(dtype)], None, stream)
        p.iplsSort(None, b.data_ptr(), n, CODE[np.dtype(dtype)])
        p.iplsSort(None, b2.data_ptr(), n, CODE[np.dtype(dtype)])
        torch.cuda.synchronize()
        for got, want, src in [(a, b, x), (a2, b2, y)]:
            g = from_dev(got, dtype)
            w = from_dev(want, dtype)
            assert np.array_equal(g.view(np.uint8), w.view(np.uint8)), (dist, n)
            ref = oracle.std_sort(src)
            assert np.array_equal(g.view(np.uint8), ref.view(np.uint8)), (dist, n)


@pytest.mark.gpu
def test_other_cutoffs_and_k():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p = _lib()
    p.load()
    for cutoff, k, n in [(1, 256, 2048), (3, 4, 4096), (256, 64, 8192)]:
        cfg = p.iplsDefaultConfig()
        cfg.cutoff, cfg.k = cutoff, k
        x = datagen.generate("mixgauss", n, np.float64, seed=cutoff)
        a = to_dev(x)
        p.ipls.iplsSortSmallNoAlloc(a.data_ptr(), n, 0, cfg, 0)
        ctx = p.Context(cutoff=cutoff, k=k)
        b = to_dev(x)
        ctx.sort_ptr(b.data_ptr(), n, 0)
        torch.cuda.synchronize()
        assert np.array_equal(from_dev(a, np.float64).view(np.uint8),
                              from_dev(b, np.float64).view(np.uint8)), (cutoff, k)
        assert np.array_equal(from_dev(a, np.float64).view(np.uint8),
                              oracle.std_sort(x).view(np.uint8)), (cutoff, k)
