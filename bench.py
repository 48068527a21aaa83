#!/usr/bin/env python3
"""Throughput of the GB300 learned sort (IPLS learned partitioning pass).

Workload (one step): sort one array of 2^28 float64 keys with the whole IPLS
recursion (k = 256, alpha*k-1 samples, base-case cutoff 256).  The K timed steps cycle
through eight seeded synthetic distributions (Normal(0,1), LogNormal(0,0.5),
Exponential(2), 5-Gaussian mixture, Zipf(0.75), root-dups, two-dups,
eight-dups) that stand in for the paper's synthetic benchmark datasets.

value   = keys sorted / device time of the sort calls (CUDA events on the
          context's stream), inputs resident in HBM; between steps a 2 GiB
          copy restores the input, which also flushes the 129 MB L2.
e2e     = same metric through iplsSortHost with pinned host buffers: the
          host->device copy, the sort and the device->host copy are timed.
roofline: the kernel with the largest device time; algorithmic bytes (keys
          read + written by its launches) / its summed launch time, against
          the measured HBM copy bandwidth.
cpu_baseline: the serial CPU oracle on a bounded prefix sample of the same
          arrays, timed on this host (rank 0, N=1 only).

--impl reference runs the oracle (the CPU reference implementation written
from the paper) as the comparison arm on the same metric.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DISTS = ["normal", "lognormal", "exponential", "mixgauss", "zipf", "rootdups", "twodups",
         "eightdups"]
METRIC = "Gkeys/s sorting 2^28 f64 keys (IPLS learned partition sort)"
UNIT = "Gkeys/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=16)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--log2n", type=int, default=28)
    p.add_argument("--cutoff", type=int, default=256)
    p.add_argument("--e2e-steps", type=int, default=4)
    p.add_argument("--cpu-sample-log2", type=int, default=24)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-torch-sort", action="store_true")
    p.add_argument("--dists", default=",".join(DISTS),
                   help="comma-separated subset of the distributions (profiling runs)")
    p.add_argument("--profile-stats", metavar="JSON",
                   help="profiling run: sort W+K arrays, write the per-kernel launches and "
                        "algorithmic bytes of ALL of them to JSON, print no bench line")
    p.add_argument("--workload", default="single",
                   choices=["single", "segmented", "serve", "integers", "uniform2p20"],
                   help="single: the 2^28 arrays (headline); segmented: a batch of "
                        "200,000 uneven segments in one call vs one call per segment; "
                        "serve: Poisson-arriving requests, batched vs one at a time")
    p.add_argument("--requests", type=int, default=2000)
    p.add_argument("--load", type=float, default=0.7,
                   help="offered load as a fraction of the one-at-a-time service rate")
    p.add_argument("--max-request-log10", type=float, default=6.0)
    p.add_argument("--segments", type=int, default=200_000)
    p.add_argument("--autotune", action="store_true",
                   help="segmented: tune (k, cutoff, graph, PL2) on another instance of the "
                        "workload first, then time the tuned and the default configuration")
    p.add_argument("--graph", action="store_true",
                   help="segmented: device-driven levels captured into a CUDA graph")
    p.add_argument("--stated-size", action="store_true",
                   help="segmented: the size law as stated (about 1.26e9 keys), not rescaled to 2^log2n")
    p.add_argument("--budget-gb", type=int, default=64,
                   help="serve: device-memory budget of the requests in flight (GiB)")
    p.add_argument("--tuned", metavar="JSON", help="autotuner table; picks k and cutoff")
    p.add_argument("--pl2", type=int, default=0,
                   help="PL2 leaves for subproblems above 8192 keys (0: FMCD, the paper's IPLS)")
    p.add_argument("--ingest-ncu", nargs=2, metavar=("CSV", "STATS_JSON"),
                   help="write profiles/ncu_traffic.json from an ncu --csv launch list with "
                        "dram__bytes_{read,write}.sum of a --profile-stats run and its JSON")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_throughput(local_ms: float, keys_per_rank: int, world: int, device) -> tuple:
    """Whole-job throughput of N independent replicas: every rank sorted
    keys_per_rank keys in local_ms; the job took the slowest rank's time
    (max over ranks).  Returns (Gkeys/s over all ranks, max ms)."""
    ms = local_ms
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([local_ms], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return world * keys_per_rank / (ms * 1e-3) / 1e9, ms


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def source_digest() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2208_06902_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, algorithmic_bytes_per_launch: float):
    """DRAM bytes per launch of `kernel`: the ratio of measured DRAM bytes to
    algorithmic bytes from the committed ncu capture, times this run's
    algorithmic bytes per launch.  None when the capture is missing or the
    kernel sources changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    if d.get("source_digest") != source_digest():
        return None
    k = d.get("kernels", {}).get(kernel)
    if not k:
        return None
    return round(float(k["dram_per_algorithmic_byte"]) * algorithmic_bytes_per_launch)


def ingest_ncu(csv_path: str, stats_path: str) -> int:
    """Per-kernel ratio of measured DRAM bytes to algorithmic bytes, from an
    ncu launch list (dram__bytes_read.sum, dram__bytes_write.sum per launch)
    of a --profile-stats run and the algorithmic bytes that run reported."""
    import csv
    with open(stats_path) as f:
        stats = json.load(f)
    with open(csv_path) as f:
        rows = list(csv.DictReader([ln for ln in f if ln.startswith('"')]))
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    dram = {}
    for r in rows:
        if r.get("Metric Name") not in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            continue
        name = r["Kernel Name"].split("(")[0].split("<")[0].replace("void ", "").split("::")[-1]
        v = float(r["Metric Value"].replace(",", "")) * scale.get(r["Metric Unit"], 1)
        dram[name] = dram.get(name, 0.0) + v
    kernels = {}
    for name, st in stats["kernels"].items():
        # k_hist_redo launches the k_hist kernel; its bytes are counted with k_hist
        if name == "k_hist_redo" or not st["bytes"] or name not in dram:
            continue
        kernels[name] = {"dram_bytes": dram[name], "algorithmic_bytes": st["bytes"],
                         "dram_per_algorithmic_byte": round(dram[name] / st["bytes"], 4)}
    out = {"source_digest": source_digest(), "case": stats["case"], "kernels": kernels}
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out))
    return 0


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 50 ms (one GPU)."""

    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "50"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # the timed region starts only once samples are flowing
        t0 = time.time()
        while time.time() - t0 < 5.0 and os.path.getsize(self.file.name) == 0:
            time.sleep(0.02)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        self.file.flush()
        rows = []
        try:
            with open(self.file.name) as f:
                for line in f:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) < 10:
                        continue
                    if self.uuid and parts[1] != self.uuid:
                        continue
                    rows.append(parts)
        finally:
            os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def make_inputs(n: int, dists):
    import datagen
    return {d: datagen.config2(d, n) for d in dists}


def cpu_baseline(inputs, sample_log2: int, cutoff: int):
    import oracle
    m = 1 << sample_log2
    keys = 0
    t0 = time.perf_counter()
    for d in inputs:
        x = inputs[d][:m]
        oracle.sort(x, cutoff=cutoff)
        keys += x.size
    dt = time.perf_counter() - t0
    # beside it, on a quarter of that sample: std::sort under the totalOrder
    # comparator on one core (the textbook routine the result must equal)
    ms = max(1, m >> 2)
    t1 = time.perf_counter()
    skeys = 0
    for d in inputs:
        x = inputs[d][:ms]
        oracle.std_sort(x)
        skeys += x.size
    st = time.perf_counter() - t1
    return {"value": keys / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first 2^{sample_log2} keys of each of the {len(inputs)} arrays "
                      f"({keys} keys, serial C++ oracle, {dt:.1f} s)",
            "std_sort": {"value": skeys / st / 1e9, "unit": UNIT, "cores": 1,
                         "sample": f"first 2^{max(0, sample_log2 - 2)} keys of each array, "
                                   f"std::sort with the totalOrder comparator, {st:.1f} s"}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import datagen
    import oracle
    oracle.build()
    m = 1 << min(args.cpu_sample_log2, args.log2n)
    # the first m keys of each 2^log2n array (the generators are counter-based,
    # so the prefix is generated without the rest of the array)
    samples = {d: datagen.generate(d, 1 << args.log2n, "float64", seed=DISTS.index(d) + 1,
                                   lo=0, hi=m) for d in DISTS}
    for i in range(args.warmup):
        oracle.sort(samples[DISTS[i % len(DISTS)]], cutoff=args.cutoff)
    t0 = time.perf_counter()
    keys = 0
    for i in range(args.steps):
        x = samples[DISTS[i % len(DISTS)]]
        oracle.sort(x, cutoff=args.cutoff)
        keys += x.size
    dt = time.perf_counter() - t0
    value = keys / dt / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"IPLS sort of 2^{args.log2n} f64 keys, 8 distributions",
                       "per_step": f"the first 2^{int(m).bit_length() - 1} keys of one array",
                       "k": 256, "cutoff": args.cutoff},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"first {m} keys of each array, serial C++ oracle"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gb300(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    import paper_2208_06902_gb300 as ipls
    ipls.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    n = 1 << args.log2n
    dists = [d for d in args.dists.split(",") if d]
    assert dists and all(d in DISTS for d in dists), f"unknown distribution in {args.dists}"
    inputs = make_inputs(n, dists)
    pristine = {d: torch.from_numpy(inputs[d].view(np.uint8)).to(dev) for d in dists}
    work = torch.empty(n * 8, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    ctx = ipls.Context(cutoff=args.cutoff, profile=True, stream=stream, pl2_leaves=args.pl2)

    def step(i, timed):
        d = dists[i % len(dists)]
        work.copy_(pristine[d])  # restores the input; 4 GB of traffic flushes L2
        if timed:
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.sort_ptr(work.data_ptr(), n, ipls.F64)
            b.record(stream)
            return d, a, b
        ctx.sort_ptr(work.data_ptr(), n, ipls.F64)
        return d, None, None

    if args.profile_stats:
        # profiling run under ncu: every sort counts, nothing else runs
        ctx.kernel_stats(reset=True)
        for i in range(args.warmup + args.steps):
            step(i, False)
        ks = ctx.kernel_stats(reset=True)
        with open(args.profile_stats, "w") as f:
            json.dump({"case": f"2^{args.log2n} f64, {args.warmup + args.steps} sorts cycling "
                               f"{','.join(dists)}, cutoff {args.cutoff}",
                       "kernels": {k["name"]: {"launches": k["launches"], "bytes": k["bytes"],
                                               "ms": k["total_ms"]} for k in ks if k["launches"]}},
                      f, indent=1)
        ctx.close()
        return 0

    for i in range(args.warmup):
        step(i, False)
    # correctness guard on the last warm-up output (cheap: monotone check)
    chk = work.view(torch.float64)
    assert bool((chk[1:] >= chk[:-1]).all()), "bench: output not sorted"
    torch.cuda.synchronize()

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ctx.kernel_stats(reset=True)
    ctx.level_stats(reset=True)
    sampler.start()
    events = [step(i, True) for i in range(args.steps)]
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if world > 1:
        torch.distributed.barrier()
    times = [(d, a.elapsed_time(b)) for d, a, b in events]
    total_ms = sum(t for _, t in times)
    kstats = ctx.kernel_stats(reset=True)
    lstats = ctx.level_stats(reset=True)
    value, total_ms = replica_throughput(total_ms, n * args.steps, world, dev)
    per_dist = {}
    for d, t in times:
        per_dist.setdefault(d, []).append(t)
    per_dist = {d: round(n / (statistics.median(v) * 1e-3) / 1e9, 3) for d, v in per_dist.items()}

    launches = sum(k["launches"] for k in kstats)
    dom = max(kstats, key=lambda k: k["total_ms"])
    peak, peak_kind = measured_peaks()
    achieved = dom["bytes"] / (dom["total_ms"] * 1e-3) / 1e9 if dom["total_ms"] > 0 else 0.0
    per_launch_bytes = dom["bytes"] / max(dom["launches"], 1)
    traffic = ncu_traffic(dom["name"], per_launch_bytes)
    # each grid level's partition passes: algorithmic 2*w*n_live over the
    # summed time of that level's grid kernels
    levels = []
    for lv in lstats:
        if lv["grid_ms"] <= 0 or not lv["bytes"]:
            continue
        gbs = lv["bytes"] / (lv["grid_ms"] * 1e-3) / 1e9
        levels.append({"level": lv["level"], "keys_per_step": lv["keys"] // args.steps,
                       "ms_per_step": round(lv["grid_ms"] / args.steps, 4),
                       "achieved": round(gbs, 1), "frac": round(gbs / peak, 4)})
    tot_b = sum(lv["bytes"] for lv in lstats)
    tot_ms = sum(lv["grid_ms"] for lv in lstats)
    roofline_pass = {"unit": "GB/s", "peak": peak, "peak_source": peak_kind,
                     "bytes": "2*w*n_live per level (keys moved by the level's grid passes)",
                     "time": "sum of the level's fit, classify+histogram, check, scans and scatter",
                     "levels": levels,
                     "level0_frac": levels[0]["frac"] if levels and levels[0]["level"] == 0 else None,
                     "grid_avg_frac": round(tot_b / (tot_ms * 1e-3) / 1e9 / peak, 4) if tot_ms > 0 else None}
    kernels = {k["name"]: {"launches": k["launches"], "ms": round(k["total_ms"], 3),
                           "GB/s": round(k["bytes"] / (k["total_ms"] * 1e-3) / 1e9, 1)
                           if k["total_ms"] > 0 and k["bytes"] else None}
               for k in kstats if k["launches"]}

    # end to end through the host-buffer entry points, pinned host buffers:
    # iplsSortHostBatch over e2e_steps arrays (copies of neighbouring arrays
    # overlapped with the sorts), and one iplsSortHost call per array
    e2e = None
    e2e_single = None
    if args.e2e_steps > 0:
        k = args.e2e_steps
        hosts = [torch.empty(n * 8, dtype=torch.uint8, pin_memory=True) for _ in range(k)]
        hvs = [h.numpy() for h in hosts]

        def fill():
            for i in range(k):
                hvs[i][:] = inputs[dists[i % len(dists)]].view(np.uint8)

        fill()  # warm-up: the pipeline buffers and copy streams
        ctx.sort_host_batch_ptrs([hosts[0].data_ptr()], [n], ipls.F64)
        fill()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        t0 = time.perf_counter()
        ctx.sort_host_batch_ptrs([h.data_ptr() for h in hosts], [n] * k, ipls.F64)
        t1 = time.perf_counter()
        b.record(stream)
        torch.cuda.synchronize()
        e_ms = max(a.elapsed_time(b), (t1 - t0) * 1e3)
        for hv in hvs:
            out = np.frombuffer(hv, dtype=np.float64)
            assert (np.diff(out) >= 0).all(), "bench: e2e output not sorted"
        e2e = {"value": n * k / (e_ms * 1e-3) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8,
               "api": f"iplsSortHostBatch over {k} pinned host arrays (copies in and out of "
                      "neighbouring arrays overlapped with the sorts)"}
        e_ms = 0.0
        for i in range(k + 1):
            hvs[0][:] = inputs[dists[i % len(dists)]].view(np.uint8)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            ctx.sort_host_ptr(hosts[0].data_ptr(), n, ipls.F64)
            b.record(stream)
            torch.cuda.synchronize()
            if i > 0:  # the first call allocates the staging buffer
                e_ms += a.elapsed_time(b)
        e2e_single = {"value": round(n * k / (e_ms * 1e-3) / 1e9, 4), "unit": UNIT,
                      "api": "one iplsSortHost call per array: copy in, sort, copy out"}
        del hosts, hvs

    torch_sort = None
    if not args.no_torch_sort:
        x = pristine[dists[0]].view(torch.float64)
        torch.sort(x)
        torch.cuda.synchronize()
        ts = []
        for _ in range(3):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            torch.sort(x)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        torch_sort = round(n / (min(ts) * 1e-3) / 1e9, 3)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(inputs, args.cpu_sample_log2, args.cutoff)

    st = ctx.stats()
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"IPLS sort of 2^{args.log2n} f64 keys, one step per array, "
                                   f"{len(dists)} seeded distributions",
                       "distributions": dists, "k": 256, "cutoff": args.cutoff,
                       "cutoff_reading": "base-case cutoff 256 (the 2^20 uniform workload "
                                         "states 32): a tuned choice; the sorted output is "
                                         "the same, only the pass trace differs",
                       "model": f"PL2, {args.pl2} leaves, top level" if args.pl2 else "FMCD",
                       "sample": "alpha*k-1 keys, alpha = 0.2*floor(log2 n)",
                       "l2": f"flushed: a {n * 8 >> 20} MiB input-restore copy runs between "
                             "timed steps (inputs larger than L2 from 2^25 keys)",
                       "parallelism": f"replicas x{world}"},
            "per_dist_gkeys_s": per_dist,
            "roofline": {"bound": "hbm", "kernel": dom["name"], "achieved": round(achieved, 1),
                         "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "peak_source": peak_kind, "traffic": traffic,
                         "bytes_per_launch": per_launch_bytes},
            "roofline_pass": roofline_pass,
            "kernels": kernels,
            "gpu_launches": launches,
            "e2e": e2e,
            "e2e_single": e2e_single,
            "cpu_baseline": cpu,
            "torch_sort_gkeys_s": torch_sort,
            "grid_levels_last": st.grid_levels,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_segmented(args):
    """Batched segmented sort: segment sizes LogNormal(median 2048, sigma 1.5)
    clamped to [16, 4,194,304], rescaled so they sum to about 2^log2n keys,
    each segment from one of nine distributions; one iplsSortSegmented call
    against one iplsSort call per segment on the same keys. Both outputs are
    compared bit for bit."""
    import numpy as np
    import torch

    import datagen
    torch.cuda.set_device(0)
    import paper_2208_06902_gb300 as ipls
    ipls.load()
    dev = torch.device("cuda", 0)
    sizes = datagen.segment_sizes(args.segments)
    if not args.stated_size:
        scale = (1 << args.log2n) / float(sizes.sum())
        sizes = np.maximum(np.rint(sizes * scale), 16).astype(np.int64)
    keys, offsets, _ = datagen.segmented(sizes)
    n = int(offsets[-1])
    k, cutoff = 256, args.cutoff
    if args.tuned:
        from paper_2208_06902_gb300 import autotune
        cfg = autotune.tuned_config(int(np.median(sizes)), ipls.F64, autotune.load(args.tuned))
        k, cutoff = cfg["k"], cfg["cutoff"]
    src = torch.from_numpy(keys.view(np.uint8)).to(dev)
    off = torch.from_numpy(offsets).to(dev)
    work = torch.empty_like(src)
    stream = torch.cuda.current_stream()
    flags = ipls.ipls.FLAG_GRAPH if args.graph else 0
    tuning = None
    default_gkeys = None
    if args.autotune:
        from paper_2208_06902_gb300 import autotune
        # a tuning instance of the same workload (other seeds), same size
        tsz = datagen.segment_sizes(args.segments, seed=14)
        if not args.stated_size:
            tsz = np.maximum(np.rint(tsz * ((1 << args.log2n) / float(tsz.sum()))), 16).astype(np.int64)
        tkeys, toff, _ = datagen.segmented(tsz, seed=15)
        tsrc = torch.from_numpy(tkeys.view(np.uint8)).to(dev)
        toffd = torch.from_numpy(toff).to(dev)
        twork = torch.empty_like(tsrc)
        ctxs = {}

        def run_cfg(cfg):
            key = tuple(sorted(cfg.items()))
            if key not in ctxs:
                for c_ in ctxs.values():
                    c_.close()
                ctxs.clear()
                ctxs[key] = ipls.Context(stream=stream, **cfg)
            twork.copy_(tsrc)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ipls.iplsSortSegmented(ctxs[key].ctx, twork.data_ptr(), toffd.data_ptr(), tsz.size, ipls.F64)
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1)

        cands = [dict(k=kk, cutoff=cc, flags=ff, pl2_leaves=pp) for kk in (64, 128, 256)
                 for cc in (64, 128, 256, 512) for ff in (0, ipls.ipls.FLAG_GRAPH) for pp in (0, 64)]
        tuning = autotune.tune_workload(run_cfg, cands, reps=3, log=lambda *a: None)
        for c_ in ctxs.values():
            c_.close()
        del tsrc, twork
        best = tuning["best"]
        # the default configuration on the bench instance, for comparison
        dctx = ipls.Context(k=256, cutoff=args.cutoff, stream=stream, flags=flags)
        dts = []
        for i in range(args.warmup + args.steps):
            work.copy_(src)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ipls.iplsSortSegmented(dctx.ctx, work.data_ptr(), off.data_ptr(), sizes.size, ipls.F64)
            e1.record(stream)
            torch.cuda.synchronize()
            if i >= args.warmup:
                dts.append(e0.elapsed_time(e1))
        dctx.close()
        default_gkeys = round(n / (statistics.median(dts) * 1e-3) / 1e9, 4)
        k, cutoff, flags = best["k"], best["cutoff"], best["flags"]
        ctx = ipls.Context(stream=stream, **best)
    else:
        ctx = ipls.Context(k=k, cutoff=cutoff, stream=stream, flags=flags)

    def batch():
        work.copy_(src)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ipls.iplsSortSegmented(ctx.ctx, work.data_ptr(), off.data_ptr(), sizes.size, ipls.F64)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    for _ in range(args.warmup):
        batch()
    t_batch = [batch() for _ in range(args.steps)]
    got = work.clone()
    # one plain call per segment (the same context, kernels and parameters)
    work.copy_(src)
    torch.cuda.synchronize()
    base = work.data_ptr()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for i in range(sizes.size):
        ctx.sort_ptr(base + int(offsets[i]) * 8, int(sizes[i]), ipls.F64)
    b.record(stream)
    torch.cuda.synchronize()
    t_each = a.elapsed_time(b)
    same = bool(torch.equal(got, work))
    ms = statistics.median(t_batch)
    # per-call time of a small segmented sort (one 4096-key segment), host
    # wall clock around the call, without and with the captured graph
    overhead = {}
    small = torch.from_numpy(datagen.generate("normal", 4096, np.float64, seed=9).view(np.uint8)).to(dev)
    soff = torch.tensor([0, 4096], dtype=torch.int64, device=dev)
    sw = torch.empty_like(small)
    for name, fl in (("host_levels", 0), ("graph", ipls.ipls.FLAG_GRAPH)):
        c2 = ipls.Context(k=k, cutoff=cutoff, stream=stream, flags=fl)
        for _ in range(5):
            sw.copy_(small)
            ipls.iplsSortSegmented(c2.ctx, sw.data_ptr(), soff.data_ptr(), 1, ipls.F64)
        torch.cuda.synchronize()
        reps = 200
        t0 = time.perf_counter()
        for _ in range(reps):
            ipls.iplsSortSegmented(c2.ctx, sw.data_ptr(), soff.data_ptr(), 1, ipls.F64)
        torch.cuda.synchronize()
        overhead[name] = round((time.perf_counter() - t0) / reps * 1e6, 1)
        c2.close()
    line = {"metric": "Gkeys/s, segmented batch sort (one call, all segments)",
            "value": round(n / (ms * 1e-3) / 1e9, 4), "unit": "Gkeys/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"{sizes.size} segments, {n} f64 keys in total",
                       "sizes": "LogNormal(median 2048, sigma 1.5) clamped to [16, 4194304]"
                                + (" as stated (no rescale)" if args.stated_size
                                   else f", rescaled to sum ~2^{args.log2n}"),
                       "median_segment": int(np.median(sizes)), "max_segment": int(sizes.max()),
                       "k": k, "cutoff": cutoff, "tuned": bool(args.tuned),
                       "graph": bool(flags & ipls.ipls.FLAG_GRAPH)},
            "autotune": ({"best": tuning["best"], "tuning_instance_ms": tuning["ms"],
                          "candidates": len(tuning["all"]), "default_gkeys_s": default_gkeys,
                          "default": {"k": 256, "cutoff": args.cutoff, "flags": 0, "pl2_leaves": 0}}
                         if tuning else None),
            "call_us_4096_keys": overhead,
            "per_segment_calls": {"value": round(n / (t_each * 1e-3) / 1e9, 4), "unit": "Gkeys/s",
                                  "ms": round(t_each, 1), "calls": int(sizes.size)},
            "speedup_vs_per_segment": round(t_each / ms, 2),
            "outputs_identical": same}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0 if same else 1


def run_serve(args):
    """Served sorts: requests of log-uniform size in [10^3, 10^max] keys, dtype
    uniform over f64/u64/f32, each from one of nine distributions, arriving
    as a Poisson stream at `load` x the one-at-a-time service rate. The same
    arrival trace is served by a context that batches pending requests
    (continuous batching) and by one that sorts them one at a time; latency =
    completion - arrival, measured on the host clock."""
    import threading

    import numpy as np
    import torch

    import datagen
    torch.cuda.set_device(0)
    import paper_2208_06902_gb300 as ipls
    ipls.load()
    dev = torch.device("cuda", 0)
    R = args.requests
    rng = np.random.default_rng(5)
    sizes = np.rint(10 ** rng.uniform(3.0, args.max_request_log10, R)).astype(np.int64)
    dts = [(np.float64, ipls.F64), (np.uint64, ipls.U64), (np.float32, ipls.F32)]
    kinds = rng.integers(0, 3, R)
    dists = rng.integers(0, len(datagen.NINE), R)
    widths = np.array([np.dtype(dts[k][0]).itemsize for k in kinds])
    offs = np.zeros(R + 1, np.int64)  # each request starts 16-byte aligned
    for i in range(R):
        offs[i + 1] = (offs[i] + int(sizes[i]) * int(widths[i]) + 15) // 16 * 16
    host = np.empty(int(offs[-1]), np.uint8)
    for i in range(R):
        x = datagen.generate(datagen.NINE[dists[i]], int(sizes[i]), dts[kinds[i]][0], seed=700 + i)
        host[offs[i]:offs[i] + x.nbytes] = x.view(np.uint8)
    pristine = torch.from_numpy(host).to(dev)
    pool = torch.empty_like(pristine)
    base = pool.data_ptr()
    total_keys = int(sizes.sum())

    def serve(max_batch, slots, arrivals):
        ctx = ipls.Context(cutoff=args.cutoff, max_batch=max_batch, serve_slots=slots,
                           budget_bytes=args.budget_gb << 30, pl2_leaves=args.pl2)
        pool.copy_(pristine)
        torch.cuda.synchronize()
        tickets = [None] * R
        done = [0.0] * R
        ready = threading.Semaphore(0)

        failed = []

        def waiter():
            for i in range(R):
                ready.acquire()
                if failed:
                    return
                ctx.wait(tickets[i])
                done[i] = time.perf_counter()

        th = threading.Thread(target=waiter, daemon=True)
        th.start()
        t0 = time.perf_counter()
        try:
            for i in range(R):
                target = t0 + arrivals[i]
                while True:
                    now = time.perf_counter()
                    if now >= target:
                        break
                    if target - now > 0.002:
                        time.sleep(target - now - 0.001)
                tickets[i] = ctx.submit_ptr(base + int(offs[i]), int(sizes[i]), dts[kinds[i]][1])
                ready.release()
        except BaseException:
            failed.append(True)
            ready.release()
            raise
        th.join()
        lat = np.array([done[i] - (t0 + arrivals[i]) for i in range(R)]) * 1e3
        wall = max(done) - t0
        log = ctx.batch_log()
        ctx.close()
        # device time with two batches in flight (slot intervals from CUDA events)
        iv = sorted((r["start_ms"], r["end_ms"], r["slot"]) for r in log if r["start_ms"] >= 0)
        busy = [0.0, 0.0]
        for a, b, sl in iv:
            busy[sl] += b - a
        both = 0.0
        s0 = [(a, b) for a, b, sl in iv if sl == 0]
        s1 = [(a, b) for a, b, sl in iv if sl == 1]
        for a, b in s0:
            for c_, d in s1:
                lo, hi = max(a, c_), min(b, d)
                if hi > lo:
                    both += hi - lo
        return {"gkeys_s": round(total_keys / wall / 1e9, 4), "wall_s": round(wall, 3),
                "p50_ms": round(float(np.percentile(lat, 50)), 3),
                "p99_ms": round(float(np.percentile(lat, 99)), 3),
                "mean_ms": round(float(lat.mean()), 3), "batches": len(log),
                "slot_busy_ms": [round(x, 1) for x in busy], "overlap_ms": round(both, 1)}

    # service rate of one-at-a-time sorting: everything queued at t = 0
    cal = serve(1, 1, np.zeros(R))
    rate = total_keys / cal["wall_s"]
    lam = args.load * rate / float(sizes.mean())
    arrivals = np.cumsum(rng.exponential(1.0 / lam, R))
    arrivals -= arrivals[0]
    batched = serve(0, 2, arrivals)
    out_batched = pool.clone()
    single = serve(1, 1, arrivals)
    same = bool(torch.equal(out_batched, pool))
    line = {"metric": "served sorts: Gkeys/s and p50/p99 latency, batched vs one-at-a-time",
            "value": batched["gkeys_s"], "unit": "Gkeys/s", "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": round(batched["wall_s"] * 1e3, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64/u64/f32", "data": "synthetic",
            "config": {"workload": f"{R} requests, {total_keys} keys, sizes log-uniform in "
                                   f"[1e3, 1e{args.max_request_log10:g}], Poisson arrivals",
                       "batched": "two in-flight slots, batches of any size within the budget",
                       "one_at_a_time": "one slot, one request per batch (plain IPLS per request)",
                       "budget_gib": args.budget_gb,
                       "model": f"PL2, {args.pl2} leaves" if args.pl2 else "FMCD",
                       "offered_load": args.load, "arrival_rate_per_s": round(lam, 1),
                       "one_at_a_time_rate_gkeys_s": round(rate / 1e9, 4), "cutoff": args.cutoff},
            "batched": batched, "one_at_a_time": single, "outputs_identical": same}
    print(json.dumps(line), flush=True)
    return 0 if same else 1


def run_uniform2p20(args):
    """The small single-array workload: 2^20 f64 keys U[0,1) from seed 0, a
    root sample of 2^14 keys, k = 256, base-case cutoff 32, sorted K times
    (the input restored between sorts).  Reports Gkeys/s and the per-call
    device time; the output is checked against the serial oracle."""
    import numpy as np
    import torch

    import datagen
    import oracle
    torch.cuda.set_device(0)
    import paper_2208_06902_gb300 as ipls
    ipls.load()
    dev = torch.device("cuda", 0)
    x = datagen.config1(1 << 20, seed=0)
    src = torch.from_numpy(x.view(np.uint8)).to(dev)
    work = torch.empty_like(src)
    stream = torch.cuda.current_stream()
    ctx = ipls.Context(cutoff=32, root_sample=1 << 14, stream=stream)
    ts = []
    for i in range(args.warmup + args.steps):
        work.copy_(src)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.sort_ptr(work.data_ptr(), x.size, ipls.F64)
        b.record(stream)
        torch.cuda.synchronize()
        if i >= args.warmup:
            ts.append(a.elapsed_time(b))
    want, _, _ = oracle.sort(x, cutoff=32, root_sample=1 << 14)
    same = bool(np.array_equal(work.cpu().numpy(), want.view(np.uint8)))
    ms = statistics.median(ts)
    line = {"metric": "Gkeys/s sorting 2^20 f64 uniform keys (IPLS, cutoff 32)",
            "value": round(x.size / (ms * 1e-3) / 1e9, 4), "unit": "Gkeys/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "2^20 f64 U[0,1), seed 0, root sample 2^14, k 256, cutoff 32",
                       "l2": "input (8 MiB) fits in L2: restored from a copy before every sort"},
            "equals_oracle": same}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0 if same else 1


def _sorted_on_device(t, code) -> bool:
    """Non-decreasing in totalOrder, checked on the device."""
    import torch
    if code == 2:    # u64: flip the top bit, compare as int64
        k = t.view(torch.int64) ^ torch.iinfo(torch.int64).min
    elif code == 3:  # u32
        k = t.view(torch.int32).to(torch.int64) & 0xFFFFFFFF
    else:            # f32 bits to a signed key in totalOrder
        b = t.view(torch.int32).to(torch.int64)
        k = b ^ ((b >> 31) & 0x7FFFFFFF)
    return bool((k[1:] >= k[:-1]).all())


def run_integers(args):
    """The integer and f32 workloads at full size: 2^30 u64 raw 64-bit draws,
    2^30 u32 Zipf(1.0) over 1..2^24 and 2^29 f32 Normal(0,1).  Per array:
    Gkeys/s, grid levels and passes, and each kernel's GB/s (its algorithmic
    bytes / its time) against the measured copy bandwidth.  The output is
    checked to be sorted on the device."""
    import numpy as np
    import torch

    import datagen
    torch.cuda.set_device(0)
    import paper_2208_06902_gb300 as ipls
    ipls.load()
    dev = torch.device("cuda", 0)
    peak, peak_src = measured_peaks()
    stream = torch.cuda.current_stream()
    ctx = ipls.Context(k=256, cutoff=args.cutoff, stream=stream, profile=True)
    arrays = {}
    total_keys, total_ms, ok = 0, 0.0, True
    for kind, code in (("u64", ipls.U64), ("u32", ipls.U32), ("f32", ipls.F32)):
        x = datagen.config3(kind)
        n = int(x.size)
        src = torch.from_numpy(x.view(np.uint8)).to(dev)
        del x
        work = torch.empty_like(src)

        def step():
            work.copy_(src)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.sort_ptr(work.data_ptr(), n, code)
            b.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b)

        for _ in range(args.warmup):
            step()
        ctx.kernel_stats(reset=True)
        ts = [step() for _ in range(args.steps)]
        ks = ctx.kernel_stats(reset=True)
        st = ctx.stats()
        good = _sorted_on_device(work, code)
        ok = ok and good
        kern = {}
        for k in ks:
            if not k["launches"]:
                continue
            gbs = (k["bytes"] / (k["total_ms"] * 1e-3) / 1e9) if k["bytes"] and k["total_ms"] > 0 else None
            kern[k["name"]] = {"ms_per_sort": round(k["total_ms"] / args.steps, 3),
                               "GB/s": round(gbs, 1) if gbs else None,
                               "frac": round(gbs / peak, 3) if gbs else None}
        ms = statistics.median(ts)
        arrays[kind] = {"n": n, "gkeys_s": round(n / (ms * 1e-3) / 1e9, 3), "ms": round(ms, 3),
                        "grid_levels": int(st.grid_levels), "grid_passes": int(st.grid_passes),
                        "splitter_passes": int(st.fallback_passes), "sorted": good,
                        "kernels": kern}
        total_keys += n * args.steps
        total_ms += sum(ts)
        del src, work
        torch.cuda.empty_cache()
    line = {"metric": "Gkeys/s, integer and f32 workloads (2^30 u64, 2^30 u32 Zipf, 2^29 f32)",
            "value": round(total_keys / (total_ms * 1e-3) / 1e9, 4), "unit": "Gkeys/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total_ms / (3 * args.steps), 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64/u32/f32", "data": "synthetic",
            "config": {"workload": "2^30 u64 uniform, 2^30 u32 Zipf(1.0) over 1..2^24, 2^29 f32 Normal",
                       "k": 256, "cutoff": args.cutoff},
            "peak_gbs": peak, "peak_source": peak_src, "arrays": arrays}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0 if ok else 1


def main():
    args = parse()
    if args.ingest_ncu:
        return ingest_ncu(*args.ingest_ncu)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "segmented":
        return run_segmented(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "integers":
        return run_integers(args)
    if args.workload == "uniform2p20":
        return run_uniform2p20(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
