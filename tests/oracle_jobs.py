"""Oracle runs at the workloads' full sizes, for worker processes.

Each job regenerates its seeded input (the same bytes the GPU test sorts),
sorts it with the oracle with the trace on, and saves the sorted array and
the trace (numpy .npy files) for the test process to compare with the GPU.
Only numpy, the input generators and the oracle are imported here, so a
spawned worker starts quickly and never touches the GPU."""
import os
import time

import numpy as np

import datagen
import oracle


def inputs(case):
    """The seeded full-size input of a case (name, generator, args)."""
    name, gen, arg = case
    if gen == "config2":
        return datagen.config2(arg, 1 << 28)
    return datagen.config3(arg)


def run(case, outdir: str, k: int = 256, cutoff: int = 256, trace_cap: int = 1_000_000):
    t0 = time.perf_counter()
    x = inputs(case)
    out, trace, levels = oracle.sort(x, k=k, cutoff=cutoff, trace_cap=trace_cap, as_array=True)
    if len(trace) >= trace_cap:
        raise RuntimeError(f"{case[0]}: oracle trace capacity {trace_cap} reached")
    p_out = os.path.join(outdir, f"{case[0]}_out.npy")
    p_tr = os.path.join(outdir, f"{case[0]}_trace.npy")
    np.save(p_out, out)
    np.save(p_tr, trace)
    return {"out": p_out, "trace": p_tr, "levels": levels, "records": len(trace),
            "seconds": round(time.perf_counter() - t0, 1)}
