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


def compare_trace_arrays(g, o, knots_g=None, knots_o=None):
    """Vectorised compare_traces for large traces: g is the GPU trace as a
    numpy array (iplsTraceRec layout), o the oracle's (oracle.TRACE_DTYPE).
    Every pass has the same (off, n, level) on both sides, and for each: the
    same model kind, bucket count, sample size; for FMCD passes the same D,
    capped flag and bits of A, Bc and x_lo; for splitter passes the same
    splitter count; and the same count in every bucket.  With knots, the PL2
    knots of the GPU's grid records (the first len(knots_g) records of g)
    equal the oracle's bit for bit.  Returns the number of passes compared."""
    import numpy as np
    assert len(g) == len(o), (len(g), len(o))
    kg = np.lexsort((g["level"], g["n"], g["off"]))
    ko = np.lexsort((o["level"], o["n"], o["off"]))
    G, O = g[kg], o[ko]
    for f in ("off", "n", "level"):
        assert np.array_equal(G[f], O[f]), f
    key = np.stack([G["off"], G["n"], G["level"].astype(np.int64)], 1)
    assert not (np.diff(key, axis=0) == 0).all(1).any(), "duplicate GPU pass records"
    om = O["model"]
    assert np.array_equal(G["kind"], om["kind"]), "model kind"
    assert np.array_equal(G["nbuckets"], om["nbuckets"]), "bucket count"
    assert np.array_equal(G["S"], om["S"]), "sample size"
    lin = om["kind"] == 0
    assert np.array_equal(G["D"][lin], om["D"][lin]), "FMCD D"
    assert np.array_equal(G["capped"][lin], om["capped"][lin]), "FMCD capped"
    for f in ("A", "Bc"):
        assert np.array_equal(G[f][lin].view(np.uint64), om[f][lin].view(np.uint64)), f
    assert np.array_equal(G["xlo_bits"][lin], om["xlo_bits"][lin]), "x_lo"
    spl = om["kind"] == 1
    assert np.array_equal(G["nsplit"][spl], om["nsplit"][spl]), "splitters"
    nb = om["nbuckets"].astype(np.int64)
    cols = np.arange(256)[None, :]
    mask = cols < nb[:, None]
    assert np.array_equal(np.where(mask, G["counts"], 0), np.where(mask, O["counts"][:, :256], 0)), \
        "bucket counts"
    assert (O["counts"][:, 256:] == 0).all()
    if knots_g is not None:
        ng = len(knots_g)
        # grid records come first in the GPU trace; map each to the oracle's
        gi = np.arange(len(g))
        pos_o = np.empty(len(o), np.int64)
        pos_o[ko] = np.arange(len(o))
        pos_g = np.empty(len(g), np.int64)
        pos_g[kg] = np.arange(len(g))
        for r in gi[:ng]:
            j = ko[pos_g[r]]
            assert np.array_equal(knots_g[r].view(np.uint32), knots_o[j].view(np.uint32)), \
                ("knots", int(g["off"][r]), int(g["n"][r]), int(g["level"][r]))
    return len(g)
