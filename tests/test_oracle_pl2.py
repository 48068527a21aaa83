"""Pins of the oracle's PL2 model (two-level piecewise-linear CDF) against
things other than its own code: finite differences for the gradient, the
empirical CDF written out again here for the initial knots, monotonicity,
the definition of the sorted result, closed-form balance on an arithmetic
progression, and the imbalance rule."""
import math

import numpy as np
import pytest

import datagen
import oracle


def _sample(dist, S=1432, dtype=np.float64, seed=3):
    return np.sort(datagen.generate(dist, S, dtype, seed))


@pytest.mark.parametrize("M", [64, 1024])
@pytest.mark.parametrize("dist", ["uniform", "normal", "lognormal", "exponential", "mixgauss"])
def test_gradient_matches_finite_differences(dist, M):
    x = _sample(dist, S=4000)
    m, _ = oracle.pl2_fit(x, M, 256)
    rng = np.random.default_rng(0)
    y = np.sort(rng.uniform(0, 1, m.nsplit + 1))
    L, g = oracle.pl2_loss_grad(x, m, y)
    h = 1e-6
    for j in rng.choice(m.nsplit + 1, 12, replace=False):
        e = np.zeros_like(y)
        e[j] = h
        Lp, _ = oracle.pl2_loss_grad(x, m, y + e)
        Lm, _ = oracle.pl2_loss_grad(x, m, y - e)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[j]) <= 1e-7 * max(1.0, abs(g[j])) + 1e-9, (j, fd, g[j])


def _fixed(v, rho):
    # X(v) = trunc(v / 2^rho), written out here from the definition
    return math.trunc(math.ldexp(float(v), -rho))


def test_first_loss_is_that_of_the_empirical_cdf_at_the_knots():
    x = _sample("normal")
    m, losses = oracle.pl2_fit(x, 32, 256)
    S, M, sh, rho = x.size, m.nsplit, m.pl2_sh, m.pl2_rho
    U = np.array([_fixed(v, rho) for v in x]) - m.pl2_x0
    y0 = np.array([np.count_nonzero(U < (j << sh)) / S for j in range(M + 1)])
    L0, _ = oracle.pl2_loss_grad(x, m, y0)
    assert L0 == pytest.approx(losses[0], rel=1e-4)   # training runs in binary32
    assert y0[0] == 0.0 and y0[-1] == 1.0


@pytest.mark.parametrize("M", [64, 1024])
@pytest.mark.parametrize("dist", ["uniform", "normal", "lognormal", "exponential", "mixgauss", "zipf"])
def test_training_does_not_raise_the_loss_and_knots_are_monotone(dist, M):
    x = _sample(dist, S=4000)
    r = oracle.pl2_fit(x, M, 256)
    if r is None:
        pytest.skip("degenerate sample")
    m, losses = r
    assert losses[-1] <= losses[0] * (1 + 1e-6)
    y = oracle.pl2_knots(m)
    assert np.all(np.diff(y) >= 0) and y[0] >= 0 and y[-1] <= 1


@pytest.mark.parametrize("M", [64, 1024])
@pytest.mark.parametrize("dtype", [np.float64, np.float32, np.uint64, np.uint32])
def test_bucket_map_is_monotone(dtype, M):
    x = np.sort(datagen.generate("lognormal", 1432, dtype, 5))
    m, _ = oracle.pl2_fit(x, M, 256)
    keys = oracle.std_sort(datagen.generate("lognormal", 200_000, dtype, 6))
    b = oracle.classify(keys, m)
    assert np.all(np.diff(b) >= 0)
    assert b.min() >= 0 and b.max() <= 255


@pytest.mark.parametrize("leaves", [64, 1024])
@pytest.mark.parametrize("dtype", [np.float64, np.float32, np.uint64, np.uint32])
@pytest.mark.parametrize("dist", ["uniform", "normal", "lognormal", "mixgauss", "zipf", "rootdups"])
def test_pl2_sort_equals_the_definition(dtype, dist, leaves):
    x = datagen.generate(dist, 120_000, dtype, seed=9)
    got, recs, _ = oracle.sort(x, cutoff=64, trace_cap=10_000, pl2_leaves=leaves)
    assert np.array_equal(got.view(np.uint8), oracle.std_sort(x).view(np.uint8))
    if dist in ("uniform", "normal", "lognormal") and dtype in (np.float64, np.float32):
        # PL2 ran on the large subproblems (the order-preserving integer
        # images of these draws are too concentrated for equal-width leaves:
        # there the imbalance rule takes the splitter tree, as it should)
        assert any(r.model.kind == 2 for r in recs)


@pytest.mark.parametrize("M,bound", [(64, 2), (1024, 4)])
def test_arithmetic_progression_splits_evenly(M, bound):
    # the empirical CDF of an arithmetic progression is linear, so the fitted
    # knots follow the knot fractions and every bucket gets about n/k keys;
    # with more leaves than samples the knots also follow the sample's noise,
    # and the bound is the 4n/k at which a pass would fall back
    n = 1 << 20
    x = np.arange(n, dtype=np.float64)
    s = np.sort(x[np.random.default_rng(1).choice(n, 1432)])
    m, _ = oracle.pl2_fit(s, M, 256)
    counts = np.bincount(oracle.classify(x, m), minlength=256)
    assert counts.max() <= bound * n // 256


def test_a_dense_cluster_falls_back_to_the_splitter_tree():
    # half the keys in a range a thousand times narrower than one leaf: the
    # PL2 pass would put them into one bucket (> 4n/k), so the pass takes
    # the splitter tree instead
    rng = np.random.default_rng(2)
    n = 40_000
    x = np.concatenate([rng.uniform(0, 1, n // 2), 0.5 + rng.uniform(0, 1e-9, n // 2)])
    x = x[rng.permutation(n)]
    got, recs, _ = oracle.sort(x, cutoff=64, trace_cap=10_000, pl2_leaves=64)
    assert np.array_equal(got, oracle.std_sort(x))
    root = [r for r in recs if r.level == 0][0]
    assert root.model.kind == 1


@pytest.mark.parametrize("dist", ["lognormal", "exponential"])
def test_pl2_balances_a_skewed_root_better_than_fmcd(dist):
    # what the learned CDF gains: on skewed keys the linear FMCD model leaves
    # some root buckets far above n/k; the trained PL2 stays close to n/k
    x = datagen.generate(dist, 1 << 20, np.float64, seed=7)
    _, rf, _ = oracle.sort(x, cutoff=256, trace_cap=50_000)
    _, rp, _ = oracle.sort(x, cutoff=256, trace_cap=50_000, pl2_leaves=64)
    root_f = [r for r in rf if r.level == 0][0]
    root_p = [r for r in rp if r.level == 0][0]
    assert root_p.model.kind == 2 and root_f.model.kind == 0
    max_f = max(root_f.counts[: root_f.model.nbuckets])
    max_p = max(root_p.counts[: root_p.model.nbuckets])
    assert max_p * 2 < max_f, (max_p, max_f)


@pytest.mark.parametrize("M", [64, 1024])
@pytest.mark.parametrize("dist", ["uniform", "normal", "lognormal", "exponential"])
def test_last_half_sweep_leaves_even_knots_at_their_coordinate_minimum(dist, M):
    # each step ends with the even knots, each moved to the exact minimiser of
    # the loss along its own coordinate within [y_{j-1}, y_{j+1}]; so moving
    # one of them by a quarter of its smaller gap, either way, cannot lower
    # the loss (evaluated independently, in binary64).  Gaps below 1e-5 are
    # skipped: there the move is close to the binary32 rounding of the knot.
    x = _sample(dist, S=4000)
    m, _ = oracle.pl2_fit(x, M, 256)
    y = oracle.pl2_knots(m).astype(np.float64)
    L0, _ = oracle.pl2_loss_grad(x, m, y)
    checked = 0
    for j in range(2, M - 1, 2):
        gap = min(y[j] - y[j - 1], y[j + 1] - y[j])
        if gap < 1e-5:
            continue
        for d in (0.25 * gap, -0.25 * gap):
            z = y.copy()
            z[j] += d
            L, _ = oracle.pl2_loss_grad(x, m, z)
            assert L >= L0 * (1 - 1e-12), (j, d, L, L0)
        checked += 1
    assert checked >= M // 8


@pytest.mark.parametrize("M", [16, 64, 1024])
@pytest.mark.parametrize("dtype", [np.float64, np.float32, np.uint64, np.uint32])
@pytest.mark.parametrize("dist", ["uniform", "normal", "lognormal", "exponential", "mixgauss", "zipf"])
def test_binary32_training_reaches_the_binary64_loss(dist, dtype, M):
    """The PL2 model is trained in binary32.  The same training carried out in
    binary64 is the reference: the binary32 knots, evaluated in binary64,
    give a loss within 1e-4 (relative) of the binary64 training's final loss,
    and every knot lies within 2^-12 of its binary64 counterpart -- far below
    one bucket (1/k = 2^-8 of the CDF), so the precision does not shape the
    partition."""
    x = np.sort(datagen.generate(dist, 1 << 20, dtype, seed=3)[:4095])
    f32 = oracle.pl2_fit(x, M)
    f64 = oracle.pl2_fit_f64(x, M)
    assert (f32 is None) == (f64 is None)
    if f32 is None:
        return
    m32, _ = f32
    m64, y64, losses64 = f64
    assert (m32.pl2_sh, m32.pl2_rho, m32.pl2_x0) == (m64.pl2_sh, m64.pl2_rho, m64.pl2_x0)
    y32 = oracle.pl2_knots(m32).astype(np.float64)
    L32, _ = oracle.pl2_loss_grad(x, m32, y32)
    L64, _ = oracle.pl2_loss_grad(x, m64, y64)
    assert math.isclose(L64, losses64[-1], rel_tol=1e-12)
    assert L32 <= L64 * (1 + 1e-4) + 1e-12, (L32, L64)
    assert np.abs(y32 - y64).max() <= 2.0 ** -12
