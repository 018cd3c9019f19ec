"""Benchmark of the GB300 dual-tree Gauss transform.

One step = one full dual-tree sum of the workload: build the kd-tree and
raw moments of the points (Q = R), then dfgt_sum over every bandwidth of
the workload at eps.  For a bichromatic workload (a reference set and
uneven query batches) a step builds the reference tree and one query tree
over all batches and sums them in log form (dfgt_sum_log: every query
within eps, including sums below the float range) at the first eps.  The metric is effective query-reference pairs per
second, |Q| |R| n_h / time, next to the GPU brute force on the same data.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl dfgt|reference]

Under torchrun every rank runs an independent replica on its own GPU
(its own seeded draw of the same workload; weak scaling, no collective on
the data path); rank 0 prints one JSON line with the max time over ranks.
``--impl reference`` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1102_2878_gb300 import datagen  # noqa: E402

METRIC = "effective query-ref pairs/s (|Q|·|R|/time) at ε=1e-2, DFGT vs GPU brute force"
UNIT = "pairs/s"
# the largest single-GPU configuration: D = 16, 1e6 points, 8 bandwidths
DEFAULT_WORKLOAD = "kde16d_n1e6_sweep8"
# GB300: 152 SMs.  A loop of eight independent ex2.approx chains per thread
# on every SM retired 31.4 ex2 per clock per SM at the sampled 1987 MHz, and
# the profiler puts the exact-sum kernel's XU pipe at 43% while it runs 12.8
# ex2 per clock per SM: the unit takes 32 ex2 per clock per SM (8 per
# sub-partition)
SM_COUNT, SFU_EX2_PER_CLK_PER_SM = 152, 32
# queries per query tree of a bichromatic workload's batch groups (the
# frontier of a larger group could pass 2^28 node pairs at the large
# bandwidths of D = 32, where nothing prunes)
GROUP_QUERIES = 200_000


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def replica_points(x, rank):
    """Points of rank `rank`: the workload itself on rank 0, an independent
    draw of the same recipe (permuted, jittered by 1e-4) on other ranks."""
    if rank == 0:
        return x
    rng = np.random.default_rng(1000 + rank)
    y = x[rng.permutation(len(x))] + rng.normal(0, 1e-4, size=x.shape).astype(np.float32)
    return np.ascontiguousarray(np.clip(y, 0, 1).astype(np.float32))


def max_over_ranks(value, world):
    """Largest per-step time over all ranks (host-side gloo all-reduce)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# DRAM bytes read + written by one exact-sum launch of a workload, from an
# ncu capture of `bench.py --steps 1 --warmup 1 --only-dfgt`, with the
# SHA-256 prefix of the kernel's source file at the time of the capture: a
# figure whose source has changed since is stale and reported as null.
K_BASE_TRAFFIC = {"kde3d_n2e5_sweep10": ("actions.cu", "", 40073728),
                  # k_base_tc: 15 launches of two full-size steps, 1.372e10 bytes
                  "kde16d_n1e6_sweep8": ("base_tc.cu", "283102800236594e", 914780000)}
FMA_PER_CLK_PER_SM = 128  # FP32 FMA lanes per SM


def source_sha(name):
    import hashlib

    path = os.path.join(ROOT, "paper_1102_2878_gb300", "csrc", name)
    try:
        with open(path, "rb") as f:
            return hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        return None


def base_traffic(workload):
    rec = K_BASE_TRAFFIC.get(workload)
    if not rec:
        return None
    name, sha, value = rec
    return value if sha and source_sha(name) == sha else None


def roofline_by_kernel(stats, tinfo, N, D, nh, sm_clk, hbm_gbs):
    """Achieved fraction of each kernel's bound, from the work counters of
    the sums and the kernels' live CUDA-event times (means over the timed
    steps).  Units: exact sums one ex2 per pair interaction; far field,
    local moments and far-to-local one FMA per series term (|Q| p^D, |R| p^D
    and p^{2D} per pair); traversal, post pass, level build and moment pass
    their algorithmic bytes (node boxes and pair records read, sums and
    coefficients read and written, point rows moved) against HBM."""
    mean = lambda k: statistics.mean(s[k] for s in stats)  # noqa: E731
    ex2_peak = SM_COUNT * SFU_EX2_PER_CLK_PER_SM * sm_clk * 1e6
    fma_peak = SM_COUNT * FMA_PER_CLK_PER_SM * sm_clk * 1e6
    hbm = hbm_gbs * 1e9
    dp = D if D <= 2 else (D + 3) // 4 * 4
    nn = statistics.mean(t["n_nodes"] for t in tinfo)
    depth = statistics.mean(t["depth"] for t in tinfo)
    P = tinfo[0]["n_coeff"]
    out = {}

    def put(kernel, units, unit, ms, bound, peak, peak_unit):
        if ms is None or ms <= 0 or units <= 0:
            return
        rate = units / (ms / 1e3)
        out[kernel] = {"units_per_step": units, "unit": unit, "ms_per_step": ms, "bound": bound,
                       "achieved": rate, "peak": peak, "peak_unit": peak_unit, "frac": rate / peak}

    if D <= 5:
        put("k_base", mean("base_interactions"), "pair interactions", mean("ms_base"), "alu", ex2_peak,
            "ex2/s (SFU)")
    else:
        # tensor form: one ex2 per interaction on the SFU (the binding unit);
        # direct form (SIMT): 2D + 2 FMA-pipe operations per interaction
        put("k_base_tc", mean("base_expanded"), "pair interactions", mean("ms_base_tc"), "alu", ex2_peak,
            "ex2/s (SFU)")
        direct = mean("base_interactions") - mean("base_expanded")
        put("k_base_hd", direct * (2 * D + 2), "FMA-pipe operations (2D + 2 per interaction)",
            mean("ms_base") - mean("ms_base_tc"), "alu", fma_peak, "FMA/s")
    put("k_farfield", mean("farfield_terms"), "series terms |Q| p^D", mean("ms_farfield"), "alu",
        fma_peak, "FMA/s")
    put("k_local", mean("local_terms"), "series terms |R| p^D", mean("ms_local"), "alu", fma_peak, "FMA/s")
    put("k_f2l", mean("f2l_terms"), "coefficient products p^2D", mean("ms_f2l"), "alu", fma_peak, "FMA/s")
    # traversal: two boxes (2 D floats each) and a 16-byte pair record read per pair
    put("k_traverse", mean("pairs_visited") * (16 * D + 16), "bytes", mean("ms_classify"), "hbm", hbm,
        "B/s (measured copy)")
    # post: per-query accumulators read and sums written, local coefficients read
    put("k_post", nh * N * 16 + nh * nn * P * 8, "bytes", mean("ms_post"), "hbm", hbm, "B/s (measured copy)")
    # level build: every level reads and writes each point row and its index
    put("k_build_levels", depth * N * (2 * dp * 4 + 8), "bytes",
        statistics.mean(t["ms_levels"] for t in tinfo), "hbm", hbm, "B/s (measured copy)")
    # moment pass: points read once; float64 moments and float32 copies written per node
    put("k_moments", N * dp * 4 + nn * P * 12, "bytes", statistics.mean(t["ms_moments"] for t in tinfo),
        "hbm", hbm, "B/s (measured copy)")
    return out


def load_problem(name, n):
    """(queries, references or None for Q = R, bandwidths, eps, query batch
    sizes or None) of a named workload; ``n`` gives a smaller case (points,
    or references of a bichromatic workload)."""
    if name in datagen.BICHROMATIC:
        refs, batches, hs, eps_list = datagen.bichromatic(name, nr=n)
        return (np.ascontiguousarray(np.concatenate(batches)), refs, hs, eps_list[0],
                [len(b) for b in batches])
    x, hs, eps = datagen.workload(name, n)
    return x, None, hs, eps, None


def query_groups(sizes, limit):
    """Query index spans [a, b) of consecutive batches holding at most
    ``limit`` queries each (a larger batch is a span of its own)."""
    spans, a, b = [], 0, 0
    for m in sizes:
        if b > a and b - a + m > limit:
            spans.append((a, b))
            a = b
        b += m
    if b > a:
        spans.append((a, b))
    return spans


def cpu_oracle_rate(x, hs, target_s, seed=0, r=None):
    """Time the FP64 oracle's exact sums on a bounded query sample (all
    references, all bandwidths), in batches grown until about target_s of
    work is done; returns (pairs/s, sample description, cores, seconds)."""
    import oracle

    oracle.build()
    x64 = x.astype(np.float64)
    r64 = x64 if r is None else r.astype(np.float64)
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(x))
    oracle.naive_kde(x64[order[:16]], r64, hs[0])  # thread pool and pages warm
    done, spent, batch = 0, 0.0, 16
    while done < len(x) and spent < target_s:
        sel = x64[order[done:done + batch]]
        t0 = time.perf_counter()
        for h in hs:
            oracle.naive_kde(sel, r64, h)
        dt = time.perf_counter() - t0
        spent += dt
        done += len(sel)
        per_query = dt / len(sel)
        batch = int(max(16, min(len(x) - done, (target_s - spent) / max(per_query, 1e-9))))
    pairs = done * len(r64) * len(hs)
    cores = oracle.num_threads()
    desc = f"{done} of {len(x)} queries x all {len(r64)} references x {len(hs)} bandwidths, {spent:.1f} s"
    return pairs / spent, desc, cores, spent


def run_reference(args, rank, world):
    if rank != 0:
        return
    x, r, hs, eps, _ = load_problem(args.workload, args.n)
    vals, secs = [], []
    desc, cores = "", 0
    per_step = max(2.0, min(12.0, 150.0 / max(1, args.steps + args.warmup)))
    for i in range(args.warmup + args.steps):
        v, desc, cores, sec = cpu_oracle_rate(x, hs, per_step, seed=i, r=r)
        if i >= args.warmup:
            vals.append(v)
            secs.append(sec)
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "D": x.shape[1], "N": len(x), "nh": len(hs),
                       "eps": eps, "q_eq_r": r is None,
                       **({} if r is None else {"n_ref": len(r)})},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": desc + " per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_dfgt(args, rank, world, local):
    import torch

    import paper_1102_2878_gb300 as dfgt

    torch.cuda.set_device(local)
    dfgt.build()
    x, r, hs, eps, sizes = load_problem(args.workload, args.n)
    x = replica_points(x, rank)  # independent replica per rank (weak scaling)
    N, D, nh = x.shape[0], x.shape[1], len(hs)
    NR = N if r is None else r.shape[0]
    ctx = dfgt.Context(local)
    pts = torch.from_numpy(x).to(f"cuda:{local}")
    rpts = pts if r is None else torch.from_numpy(r).to(f"cuda:{local}")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{local}")
    torch.cuda.synchronize()

    ev_build = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    tinfo = []

    def step():
        ev_build[0].record(ctx.stream)
        if r is not None:
            # the reference tree, then the batches in groups of query trees
            rtree = dfgt.Tree(ctx, rpts)
            ev_build[1].record(ctx.stream)
            outs, st = dfgt.kde_sum_batches(ctx, list(torch.split(pts, sizes)), rtree, hs, eps,
                                            max_queries=GROUP_QUERIES, log=True)
            tinfo.append(rtree.info())
            rtree.close()
            st["ms_build"] = ev_build[0].elapsed_time(ev_build[1])
            return torch.cat([g for g, _ in outs], dim=1), st
        tree = dfgt.Tree(ctx, pts)
        ev_build[1].record(ctx.stream)
        G, st = dfgt.kde_sum(ctx, tree, tree, hs, eps)
        tinfo.append(tree.info())
        tree.close()
        st["ms_build"] = ev_build[0].elapsed_time(ev_build[1])
        return G, st

    for _ in range(args.warmup):
        G, st = step()
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    launches0 = ctx.launch_count()
    times, stats = [], []
    for _ in range(args.steps):
        with torch.cuda.stream(ctx.stream):
            flush.fill_(1.0)  # evict L2 (129 MB) between timed steps
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        G, st = step()
        e1.record(ctx.stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        stats.append(st)
    launches = ctx.launch_count() - launches0
    tinfo = tinfo[-args.steps:]
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = max_over_ranks(statistics.mean(times), world)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    pairs_step = N * NR * nh
    value = world * pairs_step / (ms / 1e3)

    if args.only_dfgt:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": world * pairs_step / (ms / 1e3), "unit": UNIT,
                              "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup,
                              "config": {"workload": args.workload, "N": N}, "note": "dual-tree steps only"}))
        ctx.close()
        return
    # GPU brute force on the same data (the comparison named by the metric)
    Gb = dfgt.kde_sum_bruteforce(ctx, pts, rpts, hs)
    bf_ms = []
    for _ in range(max(2, min(args.steps, 3))):
        with torch.cuda.stream(ctx.stream):
            flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        dfgt.kde_sum_bruteforce(ctx, pts, rpts, hs, out=Gb)
        e1.record(ctx.stream)
        e1.synchronize()
        bf_ms.append(e0.elapsed_time(e1))
    bf = statistics.mean(bf_ms)
    ok = Gb > 1e-30
    rel = ((G - Gb).abs()[ok] / Gb[ok]).max().item()

    # end to end through the host-buffer C-ABI call (copies inside the timed region)
    xh = torch.from_numpy(x).pin_memory().numpy()
    Gh = torch.empty((nh, N), dtype=torch.float64).pin_memory().numpy()
    rh = None if r is None else torch.from_numpy(r).pin_memory().numpy()
    # a bichromatic workload goes through the host call once per batch group
    spans = [(0, N)] if r is None else query_groups(sizes, GROUP_QUERIES)
    Gparts = [Gh] if r is None else [torch.empty((nh, b - a), dtype=torch.float64).pin_memory().numpy()
                                     for a, b in spans]

    def host_step():
        for (a, b), out in zip(spans, Gparts):
            dfgt.kde_host(ctx, xh[a:b], rh, hs, eps, out=out)

    host_step()
    e2e_t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        host_step()
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = statistics.mean(e2e_t)

    if rank != 0:
        return
    # roofline of the dominant kernel: the exact sums (DFGTBase), one ex2 per
    # pair interaction, bounded by the SFU ex2 issue rate; for D >= 6 the
    # tensor-core kernel if it takes the larger share of their time
    peaks = measured_peaks()
    sm_clk = (clocks or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    peak = SM_COUNT * SFU_EX2_PER_CLK_PER_SM * sm_clk * 1e6
    inter = statistics.mean(s["base_interactions"] for s in stats)
    roof_units = inter
    roof_ms = statistics.mean(s["ms_base"] for s in stats)
    kernel = "k_base (DFGTBase exact sums)"
    if D >= 6:
        tc_ms = statistics.mean(s["ms_base_tc"] for s in stats)
        expanded = statistics.mean(s["base_expanded"] for s in stats)
        if tc_ms >= roof_ms - tc_ms:
            roof_units, roof_ms = expanded, tc_ms
            kernel = "k_base_tc (DFGTBase exact sums, tcgen05 tensor form)"
        else:
            roof_units, roof_ms = inter - expanded, roof_ms - tc_ms
            kernel = "k_base_hd (DFGTBase exact sums, direct form)"
    unit, source = "pair-interactions/s", (f"one ex2 per interaction: 152 SMs x 32 ex2/clk x {sm_clk:.0f} MHz "
                                           "(measured: independent ex2.approx chains retired 31.4 ex2/clk/SM)")
    if kernel.startswith("k_base_hd"):
        # the direct form is bound by the FMA pipe: 2D + 2 operations per interaction
        roof_units *= 2 * D + 2
        peak = SM_COUNT * FMA_PER_CLK_PER_SM * sm_clk * 1e6
        unit, source = "FMA-pipe operations/s", (f"2D + 2 FMA-pipe operations per interaction: 152 SMs x 128 "
                                                  f"FP32 lanes x {sm_clk:.0f} MHz")
    achieved = roof_units / (roof_ms / 1e3) if roof_ms > 0 else 0.0
    roof = {"bound": "alu", "kernel": kernel, "achieved": achieved,
            "peak": peak, "unit": unit, "frac": achieved / peak,
            "traffic": base_traffic(args.workload), "peak_source": source}
    cpu_rate, cpu_desc, cores = (None, None, None)
    if not args.no_cpu_baseline:
        cpu_rate, cpu_desc, cores, _ = cpu_oracle_rate(x, hs, args.cpu_seconds, r=r)
    mean = lambda k: statistics.mean(s[k] for s in stats)  # noqa: E731
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "D": D, "N": N, "nh": nh,
                   "h": [float(v) for v in hs], "eps": eps, "q_eq_r": r is None,
                   **({} if r is None else {"n_ref": NR, "query_batches": f"grouped into query trees of at most "
                                                                          f"{GROUP_QUERIES} queries",
                                            "sum": "dfgt_sum_log (e2e: dfgt_kde_host, plain G)"}),
                   "step": "kd-tree build + moments + dual-tree sum over all bandwidths",
                   "l2": "flushed between timed steps (512 MB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "bruteforce": {"value": world * pairs_step / (bf / 1e3), "unit": UNIT, "ms_per_step": bf},
        "speedup_vs_bruteforce": bf / ms,
        "max_rel_err_vs_bruteforce": rel,
        "breakdown_ms": {"build": mean("ms_build"), "classify": mean("ms_classify"),
                         "traverse": mean("ms_traverse"), "base": mean("ms_base"),
                         "base_tensor_form": mean("ms_base_tc"),
                         "farfield": mean("ms_farfield"), "local": mean("ms_local"),
                         "f2l": mean("ms_f2l"), "post": mean("ms_post")},
        "work": {"pairs_visited": mean("pairs_visited"), "prune": mean("n_prune"),
                 "farfield": mean("n_farfield"), "local": mean("n_local"), "f2l": mean("n_f2l"),
                 "base_pairs": mean("n_base"), "base_interactions": inter,
                 "base_expanded": mean("base_expanded"), "rounds": mean("rounds")},
        "roofline": roof,
        "roofline_by_kernel": roofline_by_kernel(stats, tinfo, N, D, nh, sm_clk, peaks.get("hbm_gbs", 6800.0)),
        "cpu_baseline": None if cpu_rate is None else
        {"value": cpu_rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": cpu_desc},
        "e2e": {"value": pairs_step / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": int(x.nbytes) + (0 if r is None else int(r.nbytes)),
                "d2h_bytes_per_step": int(Gh.nbytes)},
        "clocks": clocks,
        "gpu_launches": int(launches),
    }
    print(json.dumps(line), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["dfgt", "reference"], default="dfgt")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=sorted(datagen.WORKLOADS) + sorted(datagen.BICHROMATIC))
    ap.add_argument("--n", type=int, default=None,
                    help="points drawn from the workload's recipe (default: its own count); for small profiling cases")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only-dfgt", action="store_true",
                    help="time the dual-tree steps only (no brute force, e2e or CPU legs); for profiling")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    args = ap.parse_args()
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        else:
            run_dfgt(args, rank, world, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
