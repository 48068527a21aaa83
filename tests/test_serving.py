"""Request serving through iplsSubmit/iplsPoll/iplsWait: batched requests of
mixed sizes and dtypes give exactly the sorted arrays they give alone."""
import time

import numpy as np
import pytest

import datagen
import oracle
from gpu_util import CODE, from_dev, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2208_06902_gb300 as p
    p.load()


def _requests(count, seed):
    rng = np.random.default_rng(seed)
    sizes = [0, 1, 2, 17, 300, 5000, 40_000, 200_000, 1 << 20]
    dtypes = [np.float64, np.uint64, np.float32, np.uint32]
    out = []
    for i in range(count):
        n = int(rng.choice(sizes))
        dt = dtypes[int(rng.integers(len(dtypes)))]
        dist = datagen.NINE[int(rng.integers(len(datagen.NINE)))]
        out.append(datagen.generate(dist, max(n, 1), dt, seed=1000 + i)[:n].copy())
    return out


def _serve(requests, **kw):
    import torch
    from paper_2208_06902_gb300 import Context
    ctx = Context(**kw)
    bufs = [to_dev(x) if x.size else torch.empty(0, dtype=torch.uint8, device="cuda") for x in requests]
    torch.cuda.synchronize()
    tickets = [ctx.submit_ptr(b.data_ptr(), x.size, CODE[x.dtype]) for b, x in zip(bufs, requests)]
    for t in tickets:
        assert ctx.wait(t) == 0
        assert ctx.poll(t) == 0
    outs = [from_dev(b, x.dtype) for b, x in zip(bufs, requests)]
    return outs, ctx


def test_batched_requests_equal_their_sorted_arrays():
    reqs = _requests(48, seed=1)
    outs, ctx = _serve(reqs)
    for x, y in zip(reqs, outs):
        assert np.array_equal(y.view(np.uint8), oracle.std_sort(x).view(np.uint8))
    ctx.close()


def test_one_at_a_time_gives_the_same_bytes():
    reqs = _requests(24, seed=2)
    a, c1 = _serve(reqs)
    b, c2 = _serve(reqs, max_batch=1)
    for x, y in zip(a, b):
        assert np.array_equal(x.view(np.uint8), y.view(np.uint8))
    c1.close()
    c2.close()


def test_requests_arriving_while_batches_run():
    import torch
    from paper_2208_06902_gb300 import Context
    reqs = _requests(40, seed=3)
    ctx = Context()
    bufs = [to_dev(x) if x.size else torch.empty(0, dtype=torch.uint8, device="cuda") for x in reqs]
    torch.cuda.synchronize()
    tickets = []
    for b, x in zip(bufs, reqs):
        tickets.append(ctx.submit_ptr(b.data_ptr(), x.size, CODE[x.dtype]))
        time.sleep(0.0005)
    for t in tickets:
        assert ctx.wait(t) == 0
    for b, x in zip(bufs, reqs):
        assert np.array_equal(from_dev(b, x.dtype).view(np.uint8), oracle.std_sort(x).view(np.uint8))
    ctx.close()


def test_budget_rejects_a_request_that_cannot_fit_and_batches_the_rest():
    from paper_2208_06902_gb300 import Context, IPLSError
    reqs = [datagen.generate("normal", 20_000, np.float64, seed=s) for s in range(12)]
    # 2 * 8 * 20000 = 320 kB per request: a 1 MB budget allows three at a time
    outs, ctx = _serve(reqs, budget_bytes=1 << 20)
    for x, y in zip(reqs, outs):
        assert np.array_equal(y.view(np.uint8), oracle.std_sort(x).view(np.uint8))
    big = to_dev(datagen.generate("normal", 100_000, np.float64, seed=99))
    with pytest.raises(IPLSError) as e:
        ctx.submit_ptr(big.data_ptr(), 100_000, 0)
    assert e.value.status == -5
    ctx.close()


def test_unknown_ticket_and_close_with_pending_requests():
    import torch
    from paper_2208_06902_gb300 import Context, IPLSError
    ctx = Context()
    with pytest.raises(IPLSError):
        ctx.poll(12345)
    xs = [datagen.generate("uniform", 1 << 20, np.float64, seed=s) for s in range(6)]
    bufs = [to_dev(x) for x in xs]
    torch.cuda.synchronize()
    for b, x in zip(bufs, xs):
        ctx.submit_ptr(b.data_ptr(), x.size, 0)
    ctx.close()  # waits for the queued work before releasing the context
    torch.cuda.synchronize()
    for b, x in zip(bufs, xs):
        assert np.array_equal(from_dev(b, np.float64).view(np.uint8), oracle.std_sort(x).view(np.uint8))
