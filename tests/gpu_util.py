"""Helpers shared by the GPU tests: move numpy keys through the C ABI."""
import numpy as np

CODE = {np.dtype(np.float64): 0, np.dtype(np.float32): 1, np.dtype(np.uint64): 2,
        np.dtype(np.uint32): 3}


def to_dev(arr):
    import torch
    return torch.from_numpy(np.ascontiguousarray(arr).view(np.uint8)).cuda()


def from_dev(t, dtype):
    return t.cpu().numpy().view(dtype)


def gpu_sort(arr, ctx=None, **kw):
    """Sorts a copy of `arr` on the GPU through iplsSort; returns (out, ctx)."""
    import torch
    from paper_2208_06902_gb300 import Context
    arr = np.ascontiguousarray(arr)
    if ctx is None:
        ctx = Context(**kw)
    d = to_dev(arr)
    ctx.sort_ptr(d.data_ptr(), arr.size, CODE[arr.dtype])
    torch.cuda.synchronize()
    return from_dev(d, arr.dtype), ctx


def gpu_sort_segmented(arr, offsets, ctx=None, **kw):
    import torch
    from paper_2208_06902_gb300 import Context, iplsSortSegmented
    arr = np.ascontiguousarray(arr)
    if ctx is None:
        ctx = Context(**kw)
    d = to_dev(arr)
    o = torch.from_numpy(np.asarray(offsets, np.int64)).cuda()
    iplsSortSegmented(ctx.ctx, d.data_ptr(), o.data_ptr(), len(offsets) - 1, CODE[arr.dtype])
    torch.cuda.synchronize()
    return from_dev(d, arr.dtype), ctx


def trace_key(r):
    return (int(r.off), int(r.n), int(r.level))


def compare_traces(gpu_recs, oracle_recs):
    """Every pass of the oracle has a GPU pass with the same model and counts."""
    import struct
    g = {trace_key(r): r for r in gpu_recs}
    assert len(g) == len(gpu_recs), "duplicate GPU pass records"
    o = {(int(r.off), int(r.n), int(r.level)): r for r in oracle_recs}
    assert set(g) == set(o), (len(set(g) - set(o)), len(set(o) - set(g)))
    for key, orr in o.items():
        gr = g[key]
        om = orr.model
        assert gr.kind == om.kind, key
        assert gr.nbuckets == om.nbuckets, key
        assert gr.S == om.S, key
        if om.kind == 0:
            assert gr.D == om.D and gr.capped == om.capped, key
            assert struct.pack("<d", gr.A) == struct.pack("<d", om.A), key
            assert struct.pack("<d", gr.Bc) == struct.pack("<d", om.Bc), key
            assert gr.xlo_bits == om.xlo_bits, key
        else:
            assert gr.nsplit == om.nsplit, key
        nb = om.nbuckets
        assert list(gr.counts[:nb]) == list(orr.counts[:nb]), key
