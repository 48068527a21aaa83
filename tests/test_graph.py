"""Segmented sorts on device-driven levels captured into a CUDA graph
(cfg.flags & IPLS_FLAG_GRAPH): the same sorted bytes and the same passes as
the oracle, graph replays on new keys in the same buffers, recursion deeper
than the captured levels finishing from the host, and a device-side timeout
leaving a permutation of the input."""
import numpy as np
import pytest

import datagen
import oracle
from gpu_util import CODE, compare_trace_arrays, from_dev, to_dev

pytestmark = pytest.mark.gpu

FLAG_GRAPH = 2


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2208_06902_gb300 as p
    p.load()


def _same(a, b):
    return a.dtype == b.dtype and np.array_equal(a.view(np.uint8), b.view(np.uint8))


def _segments(count, seed, dtype, big=False):
    """Segment sizes from the segmented workload's law (median 2048, sigma
    1.5), a few large ones added when `big`, each from one of nine
    distributions."""
    sizes = datagen.segment_sizes(count, seed=seed)
    if big:
        sizes[:: max(1, count // 4)] = [150_000, 40_000, 9000, 700_000][: len(sizes[:: max(1, count // 4)])]
    keys, offsets, _ = datagen.segmented(sizes, seed=seed, dtype=dtype)
    return keys, offsets


def _graph_sort(ctx, x, offsets, dev=None, off=None):
    import torch
    from paper_2208_06902_gb300 import iplsSortSegmented
    d = to_dev(x) if dev is None else dev
    o = torch.from_numpy(np.asarray(offsets, np.int64)).cuda() if off is None else off
    iplsSortSegmented(ctx.ctx, d.data_ptr(), o.data_ptr(), len(offsets) - 1, CODE[x.dtype])
    torch.cuda.synchronize()
    return d, o


@pytest.mark.parametrize("dtype", [np.float64, np.float32, np.uint64, np.uint32])
@pytest.mark.parametrize("big", [False, True])
def test_graph_segmented_equals_the_oracle_pass_by_pass(dtype, big):
    from paper_2208_06902_gb300 import Context
    x, offsets = _segments(300, seed=40, dtype=dtype, big=big)
    want, o, _ = oracle.sort_segments(x, offsets, cutoff=64, trace_cap=400_000, as_array=True)
    ctx = Context(cutoff=64, trace_cap=400_000, flags=FLAG_GRAPH)
    d, _ = _graph_sort(ctx, x, offsets)
    assert _same(from_dev(d, dtype), want)
    compare_trace_arrays(ctx.trace(as_array=True), o)
    if big:
        assert ctx.stats().grid_levels >= 1
    ctx.close()


def test_graph_replays_on_new_keys_in_the_same_buffers():
    import torch
    from paper_2208_06902_gb300 import Context
    x, offsets = _segments(2000, seed=41, dtype=np.float64, big=True)
    ctx = Context(cutoff=256, flags=FLAG_GRAPH)
    dev = to_dev(x)
    off = torch.from_numpy(offsets).cuda()
    for rep in range(4):
        y = datagen.segmented(np.diff(offsets), seed=100 + rep)[0]
        dev.copy_(torch.from_numpy(y.view(np.uint8)).cuda())
        _graph_sort(ctx, y, offsets, dev, off)
        want = oracle.sort_segments(y, offsets, cutoff=256)[0]
        assert _same(from_dev(dev, np.float64), want), rep
    ctx.close()


def test_recursion_deeper_than_the_graph_continues_from_the_host():
    # k = 4 needs about log4(n / cutoff) levels, far more than the graph holds
    from paper_2208_06902_gb300 import Context
    x = datagen.generate("mixgauss", 1 << 18, np.float64, seed=42)
    offsets = np.array([0, 100_000, x.size], np.int64)
    want, o, levels = oracle.sort_segments(x, offsets, k=4, cutoff=16, trace_cap=300_000, as_array=True)
    ctx = Context(k=4, cutoff=16, trace_cap=300_000, flags=FLAG_GRAPH)
    d, _ = _graph_sort(ctx, x, offsets)
    assert _same(from_dev(d, np.float64), want)
    compare_trace_arrays(ctx.trace(as_array=True), o)
    assert ctx.stats().grid_levels > 3
    ctx.close()


def test_graph_timeout_leaves_a_permutation():
    from paper_2208_06902_gb300 import Context, IPLSError
    x, offsets = _segments(40, seed=43, dtype=np.float64, big=True)
    x = np.concatenate([x, datagen.generate("normal", 1 << 22, np.float64, seed=44)])
    offsets = np.concatenate([offsets, [x.size]])
    want = oracle.sort_segments(x, offsets)[0]
    for trial in range(2):
        ctx = Context(spin_limit=1, flags=FLAG_GRAPH)
        d = to_dev(x)
        try:
            _graph_sort(ctx, x, offsets, d)
            assert _same(from_dev(d, np.float64), want)
        except IPLSError as e:
            assert e.status == -4
            got = from_dev(d, np.float64)
            for i in range(len(offsets) - 1):
                a, b = offsets[i], offsets[i + 1]
                assert _same(oracle.std_sort(got[a:b]), oracle.std_sort(x[a:b]))
        ctx.close()
