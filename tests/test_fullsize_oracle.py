"""The CUDA path against the oracle at the workloads' full sizes, pass by
pass, in the launch configuration the bench times (k = 256, cutoff 256):

- 2^28 f64 keys: normal, Zipf(0.75), the five-Gaussian mixture, root-dups
  (the bench's arrays, seeds 1..8 by distribution);
- 2^29 f32 Normal(0,1) keys;
- 2^30 u32 Zipf(1.0) keys over 1..2^24 (a heavy-duplicate integer array).

Every partition pass the oracle makes (its model, sample size, and all
bucket counts) must appear in the GPU's trace, and the sorted bytes must be
equal.  The serial oracle takes tens of seconds per array, so the six runs
start together in a pool of spawned worker processes when the first test of
this file needs them; the GPU side sorts each array while they run."""
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle
import oracle_jobs
from gpu_util import CODE, compare_trace_arrays

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = [("normal", "config2", "normal"), ("zipf", "config2", "zipf"),
         ("mixgauss", "config2", "mixgauss"), ("rootdups", "config2", "rootdups"),
         ("f32", "config3", "f32"), ("u32", "config3", "u32")]


@pytest.fixture(scope="module")
def oracle_runs(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2208_06902_gb300 as p
    p.load()
    outdir = str(tmp_path_factory.mktemp("oracle_full"))
    pool = mp.get_context("spawn").Pool(min(len(CASES), max(1, (os.cpu_count() or 2) - 1)))
    runs = {c[0]: pool.apply_async(oracle_jobs.run, (c, outdir)) for c in CASES}
    yield runs
    pool.close()
    pool.join()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_full_size_passes_equal_the_oracle(case, oracle_runs):
    from paper_2208_06902_gb300 import Context
    x = oracle_jobs.inputs(case)
    code = CODE[x.dtype]
    dev = torch.from_numpy(x.view(np.uint8)).cuda()
    ctx = Context(k=256, cutoff=256, trace_cap=1_000_000)
    ctx.sort_ptr(dev.data_ptr(), x.size, code)
    torch.cuda.synchronize()
    got = dev.cpu().numpy().view(x.dtype)
    del dev
    g = ctx.trace(as_array=True)
    ctx.close()
    torch.cuda.empty_cache()
    res = oracle_runs[case[0]].get(timeout=3600)
    want = np.load(res["out"], mmap_mode="r")
    assert np.array_equal(got.view(np.uint8), np.asarray(want).view(np.uint8)), "sorted bytes differ"
    o = np.load(res["trace"])
    assert o.dtype == oracle.TRACE_DTYPE
    n = compare_trace_arrays(g, o)
    assert n == res["records"] and n > 0
    print(f"{case[0]}: {n} passes equal, oracle {res['seconds']} s, {res['levels']} levels")
