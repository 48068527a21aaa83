"""Autotuner table lookups (CPU) and a small tuning run on the GPU whose
chosen parameters still give the unique sorted output."""
import numpy as np
import pytest

import datagen
from paper_2208_06902_gb300 import autotune


def _table():
    return {"entries": {"f64": {"4096": {"k": 128, "cutoff": 64},
                                "1048576": {"k": 256, "cutoff": 256, "pl2_leaves": 64}}}}


def test_lookup_takes_the_largest_class_not_above_n():
    t = _table()
    assert autotune.tuned_config(4096, 0, t) == {"k": 128, "cutoff": 64, "pl2_leaves": 0}
    assert autotune.tuned_config(1 << 19, 0, t) == {"k": 128, "cutoff": 64, "pl2_leaves": 0}
    assert autotune.tuned_config(1 << 20, 0, t) == {"k": 256, "cutoff": 256, "pl2_leaves": 64}
    assert autotune.tuned_config(1 << 30, 0, t) == {"k": 256, "cutoff": 256, "pl2_leaves": 64}
    assert autotune.tuned_config(10, 0, t) == {"k": 128, "cutoff": 64, "pl2_leaves": 0}  # below every class
    with pytest.raises(KeyError):
        autotune.tuned_config(4096, 3, t)  # no u32 entry


def test_table_round_trips_through_json(tmp_path):
    p = tmp_path / "t.json"
    autotune.save(_table(), str(p))
    assert autotune.load(str(p)) == _table()


def test_segmented_generator_matches_per_segment_streams():
    sizes = datagen.segment_sizes(500)
    keys, off, dist = datagen.segmented(sizes)
    for s in range(0, sizes.size, 11):
        a, b = int(off[s]), int(off[s + 1])
        ref = datagen.generate(datagen.NINE[dist[s]], b - a, np.float64, 4 * 1_000_003 + s)
        assert np.array_equal(ref.view(np.uint64), keys[a:b].view(np.uint64)), s


@pytest.mark.gpu
def test_small_tuning_run_gives_exact_sorts():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from gpu_util import gpu_sort
    table = autotune.tune(sizes=[1 << 12, 1 << 16], dtypes=[0, 3], cutoffs=[32, 256], ks=[64, 256],
                          pl2=[0, 64], reps=1, log=lambda *a: None)
    for dtype, np_t in [(0, np.float64), (3, np.uint32)]:
        for n in [3000, 1 << 16, 100_000]:
            cfg = autotune.tuned_config(n, dtype, table)
            assert cfg["k"] in (64, 256) and cfg["cutoff"] in (32, 256) and cfg["pl2_leaves"] in (0, 64)
            x = datagen.generate("lognormal" if dtype == 0 else "zipf", n, np_t, seed=n)
            got, _ = gpu_sort(x, **cfg)
            assert np.array_equal(got.view(np.uint8), oracle.std_sort(x).view(np.uint8))


def test_workload_tuner_keeps_the_fastest_candidate():
    times = {64: 3.0, 128: 2.0, 256: 2.5}
    calls = []

    def run(cfg):
        calls.append(cfg["k"])
        return times[cfg["k"]]

    r = autotune.tune_workload(run, [{"k": 64}, {"k": 128}, {"k": 256}], reps=3, log=lambda *a: None)
    assert r["best"] == {"k": 128} and r["ms"] == 2.0
    assert len(calls) == 3 * 4  # a warm-up and three timed runs each
