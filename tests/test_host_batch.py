"""iplsSortHostBatch: host arrays sorted one after another with the copies
of neighbouring arrays overlapped with the sorts; every array must equal the
oracle's sorted array, pinned or pageable, whatever the sizes."""
import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2208_06902_gb300 as p
    p.load()


CODE = {np.dtype(np.float64): 0, np.dtype(np.float32): 1, np.dtype(np.uint64): 2,
        np.dtype(np.uint32): 3}


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("dtype", [np.float64, np.uint32])
def test_host_batch_equals_the_oracle(pinned, dtype):
    import torch
    from paper_2208_06902_gb300 import Context
    sizes = [300_017, 0, 1, 2, 40_977, 1 << 20, 5, 250_000]
    dists = ["normal", "zipf", "lognormal", "rootdups", "uniform", "exponential", "mixgauss", "twodups"]
    xs = [datagen.generate(d, max(s, 1), dtype, seed=7 + i)[:s] for i, (d, s) in enumerate(zip(dists, sizes))]
    bufs = []
    for x in xs:
        if pinned:
            t = torch.empty(max(x.nbytes, 1), dtype=torch.uint8, pin_memory=True)
            a = t.numpy()[: x.nbytes].view(dtype)
            a[:] = x
            bufs.append((t, a))
        else:
            a = np.array(x, copy=True)
            bufs.append((None, a))
    ctx = Context(k=256, cutoff=256)
    ptrs = [a.ctypes.data if a.size else 0 for _, a in bufs]
    for rep in range(2):  # the second call reuses the pipeline buffers
        if rep:
            for (_, a), x in zip(bufs, xs):
                a[:] = x
        ctx.sort_host_batch_ptrs(ptrs, [a.size for _, a in bufs], CODE[np.dtype(dtype)])
        for (_, a), x in zip(bufs, xs):
            assert np.array_equal(a.view(np.uint8), oracle.std_sort(x).view(np.uint8))
    ctx.close()


def test_host_batch_rejects_bad_arguments():
    from paper_2208_06902_gb300 import Context, IPLSError
    ctx = Context()
    with pytest.raises(IPLSError):
        ctx.sort_host_batch_ptrs([0], [10], 0)  # NULL array of 10 keys
    with pytest.raises(IPLSError):
        ctx.sort_host_batch_ptrs([0], [1], 7)   # unknown dtype
    ctx.close()
