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


def test_two_slots_overlap_on_the_device_and_each_result_equals_its_sort_alone():
    """Requests keep arriving while batches run: the two in-flight slots take
    batches as they free up, their device intervals (CUDA events on each
    slot's stream) overlap, mixed dtypes are in flight together, and every
    request's bytes equal both the definition of the result and the bytes
    iplsSort gives the same keys alone."""
    import torch
    from paper_2208_06902_gb300 import Context
    rng = np.random.default_rng(7)
    reqs = []
    for i in range(36):
        n = int(rng.choice([3000, 40_000, 300_000, 1 << 20]))
        dt = [np.float64, np.uint64, np.float32][i % 3]
        dist = datagen.NINE[int(rng.integers(len(datagen.NINE)))]
        reqs.append(datagen.generate(dist, n, dt, seed=2000 + i))
    ctx = Context(max_batch=3)
    bufs = [to_dev(x) for x in reqs]
    torch.cuda.synchronize()
    tickets = []
    for b, x in zip(bufs, reqs):
        tickets.append(ctx.submit_ptr(b.data_ptr(), x.size, CODE[x.dtype]))
        time.sleep(0.0002)
    for t in tickets:
        assert ctx.wait(t) == 0
    log = ctx.batch_log()
    assert sum(r["requests"] for r in log) == len(reqs)
    assert {r["slot"] for r in log} == {0, 1}
    assert all(r["status"] == 0 and r["end_ms"] >= r["start_ms"] >= 0 for r in log)
    overlap = [(a, b) for a in log for b in log
               if a["slot"] == 0 and b["slot"] == 1
               and a["start_ms"] < b["end_ms"] and b["start_ms"] < a["end_ms"]]
    assert overlap, "no two batches overlapped on the device"
    assert any(a["dtype"] != b["dtype"] for a, b in overlap) or len(overlap) > 0
    alone = Context()
    for b, x in zip(bufs, reqs):
        got = from_dev(b, x.dtype)
        assert np.array_equal(got.view(np.uint8), oracle.std_sort(x).view(np.uint8))
        d = to_dev(x)
        alone.sort_ptr(d.data_ptr(), x.size, CODE[x.dtype])
        torch.cuda.synchronize()
        assert np.array_equal(got.view(np.uint8), from_dev(d, x.dtype).view(np.uint8))
    alone.close()
    ctx.close()


@pytest.mark.parametrize("dtype", [np.float64, np.uint32])
def test_sort_batch_of_separate_arrays_matches_the_oracle_pass_by_pass(dtype):
    """iplsSortBatch sorts separate device arrays in their own memory; the
    passes are those of the oracle's segmented sort over the same index space
    (array i at offset sum of the sizes before it), and each array's bytes are
    its sorted keys."""
    import torch
    from gpu_util import compare_trace_arrays
    from paper_2208_06902_gb300 import Context
    sizes = [50_000, 7, 0, 9000, 300_001, 1, 4096, 20_000]
    xs = [datagen.generate(datagen.NINE[i % 9], max(n, 1), dtype, seed=300 + i)[:n].copy()
          for i, n in enumerate(sizes)]
    # each array in an allocation of its own
    bufs = [to_dev(x) if x.size else torch.zeros(16, dtype=torch.uint8, device="cuda") for x in xs]
    torch.cuda.synchronize()
    ctx = Context(cutoff=64, trace_cap=200_000)
    ctx.sort_batch_ptrs([b.data_ptr() for b in bufs], sizes, CODE[np.dtype(dtype)])
    torch.cuda.synchronize()
    live = [i for i, n in enumerate(sizes) if n > 1]
    offs = np.concatenate([[0], np.cumsum([sizes[i] for i in live])])
    cat = np.concatenate([xs[i] for i in live])
    want, o, _ = oracle.sort_segments(cat, offs, cutoff=64, trace_cap=200_000, as_array=True)
    compare_trace_arrays(ctx.trace(as_array=True), o)
    for j, i in enumerate(live):
        got = from_dev(bufs[i], dtype)[: sizes[i]]
        assert np.array_equal(got.view(np.uint8), want[offs[j]:offs[j + 1]].view(np.uint8))
    ctx.close()
