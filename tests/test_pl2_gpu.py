"""PL2 on the GPU against the oracle: the same sorted bytes; for every pass
the same model kind, leaves and bucket counts; the trained knots of every
PL2 pass equal bit for bit (the device trains them with the oracle's binary32
arithmetic); and the device's forward/backward pass (loss and gradient for
given knots) within the rounding bound of binary32 of the oracle's binary64
loss and gradient."""
import math

import numpy as np
import pytest

import datagen
import oracle
from gpu_util import compare_trace_arrays, compare_traces, gpu_sort

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
    want, recs, _, kn = oracle.sort(x, cutoff=64, trace_cap=100_000, pl2_leaves=leaves,
                                    as_array=True, knots=True)
    got, ctx = gpu_sort(x, cutoff=64, trace_cap=100_000, pl2_leaves=leaves)
    assert _same(got, want)
    g = ctx.trace(as_array=True)
    compare_trace_arrays(g, recs, ctx.trace_knots(), kn)
    if dist in ("uniform", "normal", "lognormal") and dtype in (np.float64, np.float32):
        assert (g["kind"] == 2).any()


@pytest.mark.parametrize("leaves", [2, 16, 64, 256, 1024])
def test_pl2_grid_levels_match_the_oracle(leaves):
    # pl2_depth 0: PL2 at every level above 8192 keys, so that knots of
    # several passes are compared
    x = datagen.generate("lognormal", 1 << 22, np.float64, seed=32)
    want, recs, _, kn = oracle.sort(x, cutoff=256, trace_cap=300_000, pl2_leaves=leaves,
                                    as_array=True, knots=True, pl2_depth=0)
    got, ctx = gpu_sort(x, cutoff=256, trace_cap=300_000, pl2_leaves=leaves, pl2_depth=0)
    assert _same(got, want)
    kg = ctx.trace_knots()
    g = ctx.trace(as_array=True)
    compare_trace_arrays(g, recs, kg, kn)
    assert ctx.stats().grid_levels >= 2
    assert (g["kind"][: len(kg)] == 2).sum() >= 2  # knots of several PL2 passes compared


@pytest.mark.parametrize("dist", ["lognormal", "exponential", "normal", "mixgauss"])
def test_pl2_at_the_root_balances_better_than_fmcd_on_the_gpu(dist):
    """What the trained model gains: on skewed keys (2^22 f64) the PL2 root
    pass (64 leaves, the top level only) puts fewer keys into its largest
    bucket than FMCD's linear model does, and the recursion is no deeper;
    both give the same sorted bytes.  (More of PL2's evenly sized children
    can sit above the block-resident size and take a grid pass, so the count
    of grid passes is not the measure.)"""
    x = datagen.generate(dist, 1 << 22, np.float64, seed=33)
    a, ca = gpu_sort(x, cutoff=256, trace_cap=300_000)
    b, cb = gpu_sort(x, cutoff=256, trace_cap=300_000, pl2_leaves=64, pl2_depth=1)
    assert _same(a, b)
    ra = [r for r in ca.trace() if r.level == 0][0]
    rb = [r for r in cb.trace() if r.level == 0][0]
    assert rb.kind == 2 and ra.kind != 2
    assert max(rb.counts[: rb.nbuckets]) < max(ra.counts[: ra.nbuckets])
    assert cb.stats().grid_levels <= ca.stats().grid_levels


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


def _sorted_sample(dist, dtype, S, seed):
    x = datagen.generate(dist, 1 << 20, dtype, seed=seed)[:S]
    return np.ascontiguousarray(x[np.argsort(oracle.total_order(x), kind="stable")])


def _features(x, m):
    """Leaf and in-leaf position of every sample under model m (float64),
    from the fixed-point image X = trunc(x / 2^rho) written out here."""
    rho, sh, x0, M = int(m.pl2_rho), int(m.pl2_sh), int(m.pl2_x0), int(m.nsplit)
    if x.dtype.kind == "f":
        X = np.trunc(np.ldexp(x.astype(np.float64), -rho)).astype(np.int64)
    else:
        u = x.astype(np.uint64)
        X = (u >> np.uint64(rho) if rho >= 0 else u << np.uint64(-rho)).astype(np.int64)
    U = X - x0
    leaf = np.minimum(U >> sh, M - 1)
    w = (U - (leaf << sh)).astype(np.float64) * 2.0 ** -sh
    return leaf, w


@pytest.mark.parametrize("M", [64, 1024])
@pytest.mark.parametrize("dtype", [np.float64, np.float32, np.uint64, np.uint32])
@pytest.mark.parametrize("dist", ["uniform", "normal", "lognormal", "mixgauss", "zipf"])
def test_device_loss_and_gradient_match_the_oracle(dist, dtype, M):
    """iplsPL2LossGrad runs the device's own forward and backward functions
    (the ones k_fit trains with) for given knots.  Its gradient 2 G_j / S must
    equal the oracle's binary64 gradient within the binary32 rounding bound:
    each residual carries at most ~7 roundings of values <= 1 (|dr| <= 2^-21),
    each term r t one more, and a sequential sum of m terms at most m - 1
    (Higham's gamma bound), so |d grad_j| <= (2/S) m_j 2^-21 + (m_j + 3)
    2^-24 sum_i |2 r_i t_i / S|, with m_j the samples in leaves j-1 and j.
    H_j = sum t_i^2 is checked the same way against float64 sums, and the
    loss to 1e-4 relative."""
    import torch
    import paper_2208_06902_gb300 as p
    S = 4000
    x = _sorted_sample(dist, dtype, S, seed=5)
    fit = oracle.pl2_fit(x, M)
    if fit is None:
        pytest.skip("sample range cannot carry PL2")
    m, _ = fit
    leaf, w = _features(x, m)
    cnt = np.bincount(leaf, minlength=M)
    mj = np.zeros(M + 1, np.int64)
    mj[:M] += cnt
    mj[1:] += cnt
    h_ref = np.zeros(M + 1)
    np.add.at(h_ref, leaf, (1 - w) ** 2)
    np.add.at(h_ref, leaf + 1, w ** 2)
    rng = np.random.default_rng(M)
    dev_x = torch.from_numpy(x.view(np.uint8)).cuda()
    for trial, y in enumerate([oracle.pl2_knots(m), np.sort(rng.uniform(0, 1, M + 1)).astype(np.float32)]):
        L, g, absg = oracle.pl2_loss_grad(x, m, y.astype(np.float64), with_abs=True)
        dev_y = torch.from_numpy(np.ascontiguousarray(y, np.float32)).cuda()
        out = torch.zeros(2 * (M + 1) + 2, dtype=torch.float32, device="cuda")
        p.iplsPL2LossGrad(dev_x.data_ptr(), S, {np.dtype(np.float64): 0, np.dtype(np.float32): 1,
                                                np.dtype(np.uint64): 2, np.dtype(np.uint32): 3}[x.dtype],
                          M, dev_y.data_ptr(), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        o = out.cpu().numpy().astype(np.float64)
        assert o[-1] == 1.0
        G, H, Ld = o[: M + 1], o[M + 1: 2 * (M + 1)], o[2 * (M + 1)]
        grad = 2.0 * G / S
        tol = (2.0 / S) * mj * 2.0 ** -21 + (mj + 3) * 2.0 ** -24 * absg
        bad = np.abs(grad - g) > tol
        assert not bad.any(), (np.flatnonzero(bad)[:5], grad[bad][:5], g[bad][:5], tol[bad][:5])
        assert (np.abs(H - h_ref) <= (mj + 4) * 2.0 ** -22 * np.maximum(h_ref, 1e-30)).all()
        assert math.isclose(Ld, L, rel_tol=1e-4, abs_tol=2.0 ** -40), (Ld, L)
        if trial == 1:  # random knots: the gradient is far above the bound
            assert np.abs(g).max() > 10 * tol.max()


def test_device_gradient_rejects_bad_arguments():
    import paper_2208_06902_gb300 as p
    with pytest.raises(p.IPLSError):
        p.iplsPL2LossGrad(0x1000, 1, 0, 64, 0x1000, 0x1000)
    with pytest.raises(p.IPLSError):
        p.iplsPL2LossGrad(0x1000, 100, 0, 48, 0x1000, 0x1000)
    with pytest.raises(p.IPLSError):
        p.iplsPL2LossGrad(0x1000, 5000, 0, 64, 0x1000, 0x1000)
