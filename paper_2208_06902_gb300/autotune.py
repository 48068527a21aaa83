"""Autotuner for the sort's run parameters, by measurement on this GPU.

The sorted output is unique (ascending totalOrder), so the base-case cutoff,
the buckets per pass k, the partition model (FMCD, or PL2 at the top level)
and the graph mode of segmented sorts change only the speed and the pass
trace, never the result.

- ``tune`` times a grid of (k, cutoff, PL2 leaves) on seeded synthetic arrays
  of each size class and dtype (normal, lognormal and Zipf keys) and keeps
  the fastest; ``tuned_config`` looks a size up in the resulting table,
  which ``save``/``load`` keep as JSON.
- ``tune_workload`` times candidate configurations on a whole workload (for
  example a segmented batch of uneven segments) through a caller-supplied
  runner and keeps the fastest.

    python -m paper_2208_06902_gb300.autotune --out table.json
"""
from __future__ import annotations

import argparse
import json
import os
import time

DTYPE_NAMES = {0: "f64", 1: "f32", 2: "u64", 3: "u32"}
DEFAULT_SIZES = [1 << 12, 1 << 16, 1 << 20, 1 << 24, 1 << 27]
DEFAULT_CUTOFFS = [32, 64, 128, 256, 512, 1024]
DEFAULT_KS = [64, 128, 256]
DEFAULT_PL2 = [0, 64]


def tuned_config(n: int, dtype: int, table: dict) -> dict:
    """The tuned {"k", "cutoff"} for n keys of dtype: the entry of the
    largest size class not above n (the smallest class when n is below all
    of them). Raises KeyError when the table has no entry for the dtype."""
    rows = table["entries"][DTYPE_NAMES[dtype]]
    classes = sorted(int(s) for s in rows)
    pick = classes[0]
    for s in classes:
        if s <= n:
            pick = s
    r = rows[str(pick)]
    return {"k": int(r["k"]), "cutoff": int(r["cutoff"]), "pl2_leaves": int(r.get("pl2_leaves", 0))}


def save(table: dict, path: str) -> None:
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
        f.write("\n")


def load(path: str) -> dict:
    with open(path) as f:
        return json.load(f)


def _inputs(n: int, dtype: int):
    """Three seeded arrays per size class: Normal(0,1), LogNormal(0,0.5) (or
    raw 64-bit draws for integers) and Zipf, as dtype."""
    import numpy as np

    import datagen
    np_t = {0: np.float64, 1: np.float32, 2: np.uint64, 3: np.uint32}[dtype]
    if dtype in (0, 1):
        return [datagen.generate("normal", n, np_t, 21), datagen.generate("lognormal", n, np_t, 23),
                datagen.generate("zipf", n, np_t, 22)]
    return [datagen.generate("raw64", n, np_t, 21), datagen.generate("lognormal", n, np_t, 23),
            datagen.generate("zipf", n, np_t, 22)]


def tune_workload(run, candidates, reps: int = 3, log=print) -> dict:
    """Times every candidate configuration (a dict of Context keywords) with
    ``run(cfg) -> ms`` (the caller's workload, one timed execution; the
    first call of each candidate is a warm-up) and returns {"best": cfg,
    "ms": best time, "all": [(cfg, ms), ...]}."""
    results = []
    for cfg in candidates:
        run(cfg)
        ms = sorted(run(cfg) for _ in range(reps))[reps // 2]
        results.append((cfg, round(ms, 4)))
        log(f"{cfg}: {ms:.3f} ms")
    best = min(results, key=lambda r: r[1])
    return {"best": best[0], "ms": best[1], "all": results}


def tune(sizes=DEFAULT_SIZES, dtypes=(0, 1, 2, 3), cutoffs=DEFAULT_CUTOFFS, ks=DEFAULT_KS,
         pl2=DEFAULT_PL2, reps: int = 3, log=print) -> dict:
    """Times every (k, cutoff, PL2 leaves) on each size class and dtype;
    returns the table."""
    import numpy as np
    import torch

    from . import ipls
    entries: dict = {}
    dev = torch.device("cuda", torch.cuda.current_device())
    for dtype in dtypes:
        rows = {}
        for n in sizes:
            arrays = [torch.from_numpy(np.ascontiguousarray(a).view(np.uint8)).to(dev)
                      for a in _inputs(n, dtype)]
            work = torch.empty_like(arrays[0])
            best = None
            for k, cutoff, leaves in [(k, c, p) for k in ks for c in cutoffs for p in pl2]:
                ctx = ipls.Context(k=k, cutoff=cutoff, pl2_leaves=leaves)
                total = 0.0
                for rep in range(reps + 1):
                    for a in arrays:
                        work.copy_(a)
                        s0 = torch.cuda.Event(enable_timing=True)
                        s1 = torch.cuda.Event(enable_timing=True)
                        s0.record()
                        ctx.sort_ptr(work.data_ptr(), n, dtype)
                        s1.record()
                        torch.cuda.synchronize()
                        if rep > 0:  # the first round allocates scratch
                            total += s0.elapsed_time(s1)
                ctx.close()
                ms = total / (reps * len(arrays))
                if best is None or ms < best["ms"]:
                    best = {"k": k, "cutoff": cutoff, "pl2_leaves": leaves, "ms": round(ms, 4),
                            "gkeys_s": round(n / (ms * 1e-3) / 1e9, 3)}
            rows[str(n)] = best
            log(f"{DTYPE_NAMES[dtype]} n={n}: {best}")
        entries[DTYPE_NAMES[dtype]] = rows
    return {"device": torch.cuda.get_device_name(dev), "reps": reps, "cutoffs": list(cutoffs),
            "ks": list(ks), "pl2": list(pl2), "created": time.strftime("%Y-%m-%d %H:%M:%S"),
            "entries": entries}


def main(argv=None) -> int:
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--out", required=True)
    p.add_argument("--sizes", default=",".join(str(s) for s in DEFAULT_SIZES))
    p.add_argument("--dtypes", default="0,1,2,3")
    p.add_argument("--reps", type=int, default=3)
    a = p.parse_args(argv)
    table = tune(sizes=[int(s) for s in a.sizes.split(",")],
                 dtypes=[int(d) for d in a.dtypes.split(",")], reps=a.reps)
    save(table, a.out)
    print(json.dumps({"written": os.path.abspath(a.out)}))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
