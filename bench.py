"""Benchmark: right-hand sides solved per second to relative residual 1e-8.

One step is one pass of the whole hot path on R-MAT scale 24 (a, b, c =
.57, .19, .19, 8 * 2^24 samples, unit weights, largest connected component:
n = 7,368,759 nodes, 131.7M edges, seed 5), the largest single-GPU
configuration and the one where HBM bandwidth binds: ingest of the edge list
and construction of the hierarchy (lap_build_hierarchy), generation of the
k = 64 Johnson-Lindenstrauss right-hand sides, the block solve to
||b - Lx|| <= 1e-8 ||b|| per column in FP32 PCG inside FP64 refinement, and
the farness reduction for node 0 (cfc_farness_jl).  value = 64 * N / step
time.

The line also carries: the same step through the C ABI with host buffers
(e2e), the dominant solver family against the measured HBM bandwidth
(roofline, with ncu DRAM traffic from profiles/traffic.json) and every
family's achieved bandwidth, the solve's HBM-roofline ideal, the 100k-node
Barabasi-Albert configuration's rate with the batched mixed-precision solve
against FP64 batched and FP64 one right-hand side at a time, a small serving
mix (p50/p99 latency), the oracle on the host cores (cpu_baseline: on R-MAT
24 capped iterations, extrapolated) and this run's error against it
(parity: right-hand sides at sampled nodes and the oracle's FP64 residual of
the device's solutions), and the SM clocks sampled during the timed steps.

Other workloads: --workload ba100k_jl64, rmat20_jl16/64/128, grid1024_jl64,
grid4096_jl64 (the same step), serve_mix (16 resident graphs, Poisson
arrivals) and accuracy (both estimators against the exact farness).

--impl reference times the CPU FP64 oracle on the same workload and metric.
Run with torchrun for N > 1 GPUs: the step becomes one JL query of 64 * N
rows split over the GPUs (each rank builds the graph's hierarchy and solves
its own 64 rows, cfc_farness_jl_rows), and one NCCL all-reduce adds the q
partial farness sums, the split's only exchange (weak scaling; the line's
split_check compares the result with the same query on one GPU).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "RHS solved/s to rel. residual 1e-8"
# the largest single-GPU configuration, where the HBM roofline binds: R-MAT
# scale 24 (LCC), JL farness of one node with k = 64
DEFAULT_WORKLOAD = "rmat24_jl64"
WORKLOADS = {
    "ba100k_jl64": dict(kind="ba", n=100000, m_per=5, seed=2, k=64, jl_seed=1, nodes=[0]),
    "grid48_jl32": dict(kind="grid", a=48, k=32, jl_seed=1, nodes=[0]),
    "rmat20_jl16": dict(kind="rmat", scale=20, seed=3, k=16, jl_seed=1, nodes=[0]),
    "rmat20_jl64": dict(kind="rmat", scale=20, seed=3, k=64, jl_seed=1, nodes=[0]),
    "rmat20_jl128": dict(kind="rmat", scale=20, seed=3, k=128, jl_seed=1, nodes=[0]),
    # between L2 and the headline size: profiling cases whose FP32 blocks exceed L2
    "rmat21_jl64": dict(kind="rmat", scale=21, seed=5, k=64, jl_seed=1, nodes=[0]),
    "rmat22_jl64": dict(kind="rmat", scale=22, seed=5, k=64, jl_seed=1, nodes=[0]),
    "grid1024_jl64": dict(kind="grid", a=1024, k=64, jl_seed=1, nodes=[0]),
    "grid4096_jl64": dict(kind="grid", a=4096, k=64, jl_seed=1, nodes=[0]),
    "rmat24_jl64": dict(kind="rmat", scale=24, seed=5, k=64, jl_seed=1, nodes=[0]),
}


# precision mode of lap_solve_opts_t, dtype of the JSON line, description
PRECISIONS = {
    "fp32": (1, "f32+f64", "fp32 V-cycle/PCG in fp64 refinement"),
    "bf16coarse": (2, "f32+bf16+f64", "fp32 V-cycle/PCG with bf16 weights below the finest level, fp64 refinement"),
    "fp64": (0, "f64", "fp64 PCG + V-cycle"),
}


def make_graph(wl):
    if wl["kind"] == "ba":
        n, s, d, _ = synth.barabasi_albert(wl["n"], wl["m_per"], seed=wl["seed"])
        w = synth.uniform_weights(s.size, seed=wl["seed"])
    elif wl["kind"] == "grid":
        n, s, d, w = synth.grid2d(wl["a"])
    else:
        n, s, d, w = synth.rmat(wl["scale"], seed=wl["seed"])
    return n, s, d, w


# resident graphs of the serving mix: grids 256^2 .. 1024^2, BA n = 10k .. 500k,
# R-MAT scales 14 .. 21 (LCC); unit weights on grids and R-MAT, U[1, 2) on BA
SERVE_GRAPHS = ([dict(kind="grid", a=a) for a in (256, 384, 512, 768, 1024)] +
                [dict(kind="ba", n=n, m_per=5, seed=4) for n in (10000, 30000, 100000, 200000, 500000)] +
                [dict(kind="rmat", scale=sc, seed=4) for sc in (14, 16, 18, 19, 20, 21)])
# the small mix reported beside every default line
SERVE_SMALL = [dict(kind="grid", a=256), dict(kind="ba", n=100000, m_per=5, seed=2), dict(kind="rmat", scale=16, seed=4)]


def run_serving(P, specs, n_queries, loads, seed=4, n_pivots=200, slots=4, resident=False):
    """Continuous-batching request loop on resident graphs (cfc_server_*):
    a burst of requests measures the saturation rate, then for each load
    factor Poisson arrivals at that fraction of it; latencies (submit ->
    result) come from the server.  Query: 1..32 nodes of a uniformly chosen
    graph, the sampling estimator with n_pivots pivots: drawn per request, or
    (resident=True) one pivot set per graph whose solutions stay on the
    device, so a request solves only its nodes' columns."""
    rng = np.random.default_rng(seed)
    sv = P.cfc_server_create(P.cfc_server_default_opts(slots=slots, resident_pivots=n_pivots if resident else 0,
                                                       pivot_seed=seed))
    req_pivots = 0 if resident else n_pivots
    t0 = time.time()
    sizes = []
    for spec in specs:
        n, s, d, w = make_graph(spec)
        P.cfc_server_add_graph(sv, n, s, d, w)
        sizes.append(n)
    add_s = time.time() - t0

    def queries(count):
        out = []
        for _ in range(count):
            g = int(rng.integers(len(sizes)))
            q = int(rng.integers(1, 33))
            nodes = rng.choice(sizes[g], size=q, replace=False).astype(np.int32)
            out.append((g, nodes, int(rng.integers(1 << 40))))
        return out

    def burst(qs):
        P.cfc_server_reset_stats(sv)
        ids = [P.cfc_server_submit(sv, g, nodes, req_pivots, sd) for g, nodes, sd in qs]
        for r in ids:
            P.cfc_server_poll(sv, r, -1, q=32)
        return P.cfc_server_stats(sv)

    burst(queries(2 * slots))  # warm-up
    sat = burst(queries(n_queries))
    result = {"graphs": len(specs), "nodes_max": max(sizes), "slots": slots, "n_pivots": n_pivots,
              "pivots": "one resident set per graph" if resident else "drawn per request",
              "queries_per_load": n_queries, "add_graphs_s": add_s,
              "saturation": {"queries_per_s": sat["queries_per_s"], "rhs_per_s": sat["rhs_per_s"],
                             "p50_ms": sat["p50_ms"], "p99_ms": sat["p99_ms"],
                             "max_in_flight": sat["max_in_flight"]},
              "loads": []}
    for f in loads:
        rate = f * sat["queries_per_s"]
        qs = queries(n_queries)
        gaps = rng.exponential(1.0 / rate, size=len(qs))
        P.cfc_server_reset_stats(sv)
        ids = []
        t_next = time.perf_counter()
        for (g, nodes, sd), gap in zip(qs, gaps):
            t_next += gap
            dt = t_next - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            ids.append(P.cfc_server_submit(sv, g, nodes, req_pivots, sd))
        for r in ids:
            P.cfc_server_poll(sv, r, -1, q=32)
        st = P.cfc_server_stats(sv)
        result["loads"].append({"load": f, "offered_qps": rate, "queries_per_s": st["queries_per_s"],
                                "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
                                "max_in_flight": st["max_in_flight"]})
    sv.destroy()
    return result


def kernel_source_digest():
    """Digest of the solver kernels' sources: the row-kernel templates, the
    solver and the shared header with their constants (comments and blank
    lines left out, so that documentation edits keep stored counters valid)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in ("rowops.cuh", "solve.cu", "internal.h"):
        with open(os.path.join(ROOT, "paper_1607_02955_gb300", "csrc", f)) as fh:
            text = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        for line in text.splitlines():
            line = re.sub(r"//.*$", "", line).strip()
            if line:
                h.update(line.encode() + b"\n")
    return h.hexdigest()[:16]


def read_traffic(workload, family):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, or None when it was taken on other kernel sources."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None, None, None
    with open(p) as fh:
        j = json.load(fh)
    e = j.get(workload, {}).get(family)
    if not e or e.get("source_digest") != kernel_source_digest():
        return None, None, None
    return e["dram_bytes_per_launch"], e["kernel"], e.get("note")


def write_traffic(csv_path, log_path):
    """Pairs the library's launches in an ncu per-launch CSV (metrics
    dram__bytes_read.sum, dram__bytes_write.sum, gpu__time_duration.sum) of
    the timed steps with the launch log of the same command, then stores the
    DRAM bytes per launch of every kernel family in profiles/traffic.json and
    prints a per-family and per-kernel summary."""
    import csv
    import collections
    with open(log_path) as fh:
        log = json.load(fh)
    launches = collections.OrderedDict()
    hdr = None
    with open(csv_path) as fh:
        for r in csv.reader(fh):
            if r and r[0] == "ID":
                hdr = r
                continue
            if not hdr or len(r) != len(hdr):
                continue
            d = dict(zip(hdr, r))
            if "cfc::" not in d["Kernel Name"]:
                continue  # the L2 flush between steps is torch's
            e = launches.setdefault(d["ID"], {"kernel": d["Kernel Name"]})
            e[d["Metric Name"]] = float(d["Metric Value"].replace(",", ""))
    L = list(launches.values())
    fams = log["families"]
    if len(L) != len(fams):
        raise SystemExit(f"ncu lists {len(L)} library launches, the log {len(fams)}")
    if log["source_digest"] != kernel_source_digest():
        raise SystemExit("the launch log was taken on other kernel sources")
    per_fam = collections.OrderedDict()
    per_kernel = collections.OrderedDict()
    for f, e in zip(fams, L):
        b = e.get("dram__bytes_read.sum", 0.0) + e.get("dram__bytes_write.sum", 0.0)
        t = e.get("gpu__time_duration.sum", 0.0)
        a = per_fam.setdefault(f, {"launches": 0, "dram_bytes": 0.0, "ns": 0.0, "kernels": collections.Counter()})
        a["launches"] += 1
        a["dram_bytes"] += b
        a["ns"] += t
        name = e["kernel"].replace("cfc::", "").replace("<unnamed>::", "").replace("void ", "")
        name = name[:name.index(">(") + 1] if ">(" in name else name.split("(")[0]
        a["kernels"][name] += t  # device time per kernel within the family
        k = per_kernel.setdefault((f, name), [0, 0.0, 0.0])
        k[0] += 1
        k[1] += b
        k[2] += t
    path = os.path.join(ROOT, "profiles", "traffic.json")
    j = json.load(open(path)) if os.path.exists(path) else {}
    wl = j.setdefault(log["workload"], {})
    tot_ns = sum(a["ns"] for a in per_fam.values())
    print(f"workload {log['workload']}, {log['steps']} timed step(s), {len(L)} library launches, "
          f"source digest {log['source_digest']}")
    print(f"{'family':14s} {'launches':>8s} {'MB/launch':>10s} {'us/launch':>10s} {'share':>7s}  kernel with most time")
    for f, a in sorted(per_fam.items(), key=lambda x: -x[1]["ns"]):
        top = a["kernels"].most_common(1)[0][0]
        wl[f] = {"source_digest": log["source_digest"], "launches": a["launches"],
                 "dram_bytes_per_launch": a["dram_bytes"] / a["launches"], "kernel": top}
        print(f"{f:14s} {a['launches']:8d} {a['dram_bytes'] / a['launches'] / 1e6:10.3f} "
              f"{a['ns'] / a['launches'] / 1e3:10.2f} {100 * a['ns'] / tot_ns:6.2f}%  {top}")
    print()
    print(f"{'kernel':72s} {'launches':>8s} {'MB/launch':>10s} {'us/launch':>10s} {'share':>7s}")
    for (f, name), (c, b, t) in sorted(per_kernel.items(), key=lambda x: -x[1][2]):
        print(f"{name[:72]:72s} {c:8d} {b / c / 1e6:10.3f} {t / c / 1e3:10.2f} {100 * t / tot_ns:6.2f}%")
    with open(path, "w") as fh:
        json.dump(j, fh, indent=1, sort_keys=True)


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            j = json.load(fh)
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples (every 100 ms).  Started before the
    warm-up so that nvidia-smi's own start-up does not fall in the timed
    region; mark() / stop() bound the window whose samples are kept."""

    def __init__(self, gpu_index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.t0 = self.t1 = None
        q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def mark(self):
        self.t0 = time.time()

    def stop(self):
        self.t1 = time.time()
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)  # let the sample that covers the end of the window arrive
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        text = self.f.read()
        os.unlink(self.f.name)
        return summarize_clocks(text, self.t0, self.t1)


def summarize_clocks(text, t0, t1):
    """Median SM clock, the maximum clock and the active throttle reasons of
    the nvidia-smi samples (timestamp first) taken in [t0, t1] (host time,
    seconds; 100 ms of slack each side); a window shorter than the sampling
    period takes the sample nearest its middle."""
    import datetime
    rows = []
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in text.splitlines():
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 10:
            continue
        try:
            ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            rows.append((ts, float(parts[2]), float(parts[3]),
                         {nm for nm, v in zip(names, parts[6:10]) if v.lower() == "active"}))
        except ValueError:
            continue
    t0 = t0 if t0 is not None else -1e30
    inside = [r for r in rows if t0 - 0.1 <= r[0] <= t1 + 0.1]
    if not inside and rows:  # a window shorter than the sampling period
        inside = [min(rows, key=lambda r: abs(r[0] - 0.5 * (t0 + t1)))]
    sm = [r[1] for r in inside]
    reasons = set().union(*[r[3] for r in inside]) if inside else set()
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(r[2] for r in inside) if inside else None,
            "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch
        import torch.distributed as dist
        dist.barrier(device_ids=[torch.cuda.current_device()])


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, wl, rank, world):
    """The reference arm: the CPU FP64 oracle on the same workload and metric,
    on all host cores (the oracle's columns solved in threads).  Small
    graphs: each step is the whole oracle pipeline (canonical graph,
    Laplacian, the k JL right-hand sides, CG to 1e-8, farness of the query
    node).  Large graphs: the oracle graph is built once; each step is the
    oracle's CG capped at one iteration on one column per thread, and the
    rate is extrapolated to the estimated iteration count (a capped run
    costs about three iteration-equivalents: projection and first residual,
    the iteration, the final residual check; a full solve about iters + 2)."""
    if rank != 0:
        return
    from oracle import jl
    threads = oracle_threads()
    n, s, d, w = make_graph(wl)
    k = wl["k"]
    times = []
    extra = {}
    if wl_nodes(wl) <= LARGE_N:
        for it in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            g, L, _ = oracle_graph(wl)
            Y = jl.jl_rhs(g, k, wl["jl_seed"])
            Z, _, used = cg_threaded(L, Y.T, 1e-8, 100000, threads)
            jl.farness_from_Z(Z.T, wl["nodes"])
            dt = time.perf_counter() - t0
            if it >= args.warmup:
                times.append(dt)
        sec = sum(times) / len(times)
        value = k / sec
        sample = (f"full {args.workload} step per step (canonical graph + Laplacian, {k} JL RHS, FP64 Jacobi-CG "
                  f"to 1e-8 on {used} threads, farness of node {wl['nodes'][0]})")
    else:
        g, L, setup_s = oracle_graph(wl)
        iters, spec = oracle_iterations_estimate(wl, threads)
        B = np.random.default_rng(0).standard_normal((g.n, threads))
        for it in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            _, _, used = cg_threaded(L, B, 1e-8, 1, threads)
            dt = time.perf_counter() - t0
            if it >= args.warmup:
                times.append(dt * (iters + 2) / 3.0)
        sec = sum(times) / len(times)
        value = threads / sec
        sample = (f"extrapolated: per step the oracle's FP64 Jacobi-CG capped at 1 iteration on {threads} columns "
                  f"of this graph (one per thread), scaled by (iters + 2) / 3 to the {iters} iterations estimated "
                  f"from the same oracle on {spec}; oracle setup ({setup_s:.1f} s) excluded")
        extra = {"extrapolated": True, "iterations": iters}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "RHS/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "k": k, "n": n, "m": int(s.size)},
            "cpu_baseline": {"value": value, "unit": "RHS/s", "cores": threads, "kind": "oracle", "sample": sample,
                             **extra},
            "e2e": {"value": value, "unit": "RHS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


CPU_SAMPLE_ROWS = 8
# workloads with more nodes take the extrapolated CPU baseline (capped oracle
# iterations): a converged oracle solve of them takes far longer than the bench
LARGE_N = 2_000_000


def oracle_threads():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def cg_threaded(L, B, tol, maxiter, threads):
    """The oracle's CG (oracle.cg.cg_solve, unchanged) on column chunks of B
    in host threads: its columns are independent systems, and SciPy's sparse
    products release the GIL, so the chunks run on separate cores.  Returns
    (X, max iterations over the chunks)."""
    from concurrent.futures import ThreadPoolExecutor
    from oracle.cg import cg_solve
    chunks = [c for c in np.array_split(np.arange(B.shape[1]), min(threads, B.shape[1])) if c.size]
    with ThreadPoolExecutor(len(chunks)) as ex:
        res = list(ex.map(lambda c: cg_solve(L, np.ascontiguousarray(B[:, c]), tol=tol, maxiter=maxiter), chunks))
    X = np.empty(B.shape)
    for c, (x, _, _) in zip(chunks, res):
        X[:, c] = x
    return X, max(r[1] for r in res), len(chunks)


def oracle_graph(wl):
    """The oracle's graph and Laplacian of a workload, and the seconds it took."""
    from oracle.graph import canonical_graph, laplacian
    n, s, d, w = make_graph(wl)
    t0 = time.perf_counter()
    g = canonical_graph(n, s, d, w)
    L = laplacian(g)
    return g, L, time.perf_counter() - t0


def oracle_iterations_estimate(wl, threads):
    """Iterations of the oracle's CG to 1e-8 (8 JL right-hand sides) on a
    smaller instance of the workload's family, standing in for the large
    instance, whose converged solve does not fit the bench.  R-MAT: scale 20,
    same generator and seed (the count barely grows with the scale: 24, 27,
    28 iterations at scales 16, 18, 20).  Grid: the 256 x 256 grid, the count
    multiplied by side / 256 (Jacobi-CG iterations grow with the square root
    of the condition number, which grows with the square of the side)."""
    from oracle import jl
    if wl["kind"] == "rmat":
        spec, factor = dict(kind="rmat", scale=20, seed=wl.get("seed", 3)), 1.0
    else:
        spec, factor = dict(kind="grid", a=256), wl["a"] / 256.0
    g, L, _ = oracle_graph(spec)
    Y = jl.jl_rhs(g, 8, wl["jl_seed"])
    _, it, _ = cg_threaded(L, Y.T, 1e-8, 100000, threads)
    return int(round(it * factor)), spec


def cpu_baseline(wl, threads, gL=None):
    """The oracle on a bounded sample of the workload, on `threads` host
    cores.  Small graphs: the first 8 of the k JL rows solved to 1e-8
    (returns their solutions for the parity check).  Large graphs: the
    oracle's CG on `threads` columns capped at 1 and 3 iterations gives the
    time per iteration, extrapolated to the iteration count of the same
    oracle on R-MAT 20 (oracle_iterations_estimate); setup excluded."""
    from oracle import jl
    if wl_nodes(wl) <= LARGE_N:
        ks = CPU_SAMPLE_ROWS
        t0 = time.perf_counter()
        g, L, _ = oracle_graph(wl)
        Y = jl.jl_rhs(g, wl["k"], wl["jl_seed"])[:ks]
        Z, _, used = cg_threaded(L, Y.T, 1e-8, 100000, threads)
        sec = time.perf_counter() - t0
        info = {"value": ks / sec, "unit": "RHS/s", "cores": used, "kind": "oracle",
                "sample": f"{ks} of the {wl['k']} JL right-hand sides (canonical graph + Laplacian + RHS + FP64 "
                          f"Jacobi-CG to 1e-8, one column per thread)"}
        return info, Z.T
    g, L, setup_s = gL if gL is not None else oracle_graph(wl)
    cols = threads
    B = np.random.default_rng(0).standard_normal((g.n, cols))
    t0 = time.perf_counter()
    cg_threaded(L, B, 1e-8, 1, threads)
    t1 = time.perf_counter()
    _, _, used = cg_threaded(L, B, 1e-8, 3, threads)
    t3 = time.perf_counter()
    per_it = (t3 - t1 - (t1 - t0)) / 2.0
    fixed = max(t1 - t0 - per_it, 0.0)  # projection, first residual and final residual check
    iters, spec = oracle_iterations_estimate(wl, threads)
    sec = fixed + iters * per_it
    info = {"value": cols / sec, "unit": "RHS/s", "cores": used, "kind": "oracle", "extrapolated": True,
            "sample": f"the oracle's FP64 Jacobi-CG on {cols} columns of this graph, one per thread, capped at 1 and "
                      f"3 iterations ({per_it:.2f} s per iteration, {fixed:.2f} s fixed); extrapolated to the "
                      f"{iters} iterations estimated from the same oracle on {spec} (oracle_iterations_estimate); "
                      f"oracle setup (canonical graph + Laplacian, {setup_s:.1f} s) excluded",
            "per_iteration_s": per_it, "iterations": iters}
    return info, None


def wl_nodes(wl):
    if wl["kind"] == "rmat":
        return 1 << wl["scale"]
    if wl["kind"] == "grid":
        return wl["a"] * wl["a"]
    return wl["n"]


def _ranks(x):
    r = np.empty(len(x))
    r[np.argsort(x, kind="stable")] = np.arange(len(x))
    return r


def accuracy_rows(P, torch, spec, eps_list, piv_list, rng):
    """The farness of every node of one graph by the projection estimator
    (k = ceil(ln n / eps^2), Sec. 6.4) and the sampling estimator (|S| pivots),
    against the exact farness (dense, on the device): per setting the device
    time, the largest relative error, the Spearman correlation of the
    closeness ranking with the exact one and the fraction of node pairs whose
    order flips."""
    n, s, d, w = make_graph(spec)
    f_exact, _ = P.cfc_exact_small(n, s, d, w)
    h = P.lap_build_hierarchy(n, s, d, w)
    nodes = np.arange(n, dtype=np.int32)
    pairs = rng.integers(0, n, size=(200000, 2))
    ex_order = np.sign(f_exact[pairs[:, 0]] - f_exact[pairs[:, 1]])
    rows = []

    def record(kind, param, fn):
        fn()  # first call: autotuning for this column count
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f = fn()
        ms = (time.perf_counter() - t0) * 1e3
        rel = float(np.max(np.abs(f - f_exact) / f_exact))
        rho = float(np.corrcoef(_ranks(f), _ranks(f_exact))[0, 1])
        flips = float(np.mean(np.sign(f[pairs[:, 0]] - f[pairs[:, 1]]) != ex_order))
        rows.append({"estimator": kind, **param, "ms": ms, "max_rel_err": rel, "spearman": rho,
                     "pair_flips": flips})

    for eps in eps_list:
        k = int(np.ceil(np.log(n) / eps ** 2))
        record("projection", {"eps": eps, "k": k}, lambda k=k: P.cfc_farness_jl(h, k, 1, nodes))
    for piv in piv_list:
        # the sampling estimate scales a sum over |S| pivots by n/|S| (Proposition 1)
        record("sampling", {"pivots": piv}, lambda piv=piv: P.cfc_farness_sampled(h, piv, 1, nodes))
    h.destroy()
    return {"n": n, "m": int(s.size), "rows": rows}


ACCURACY_GRAPHS = {"ba3000": dict(kind="ba", n=3000, m_per=5, seed=2), "grid48": dict(kind="grid", a=48)}


def accuracy_main(args):
    """Accuracy against time of the two estimators on synthetic graphs (the
    shape of Sec. 6.4): eps = 0.5 .. 0.05 and |S| = 10 .. 1000, every node
    queried (accuracy_rows)."""
    import torch
    torch.cuda.init()
    import paper_1607_02955_gb300 as P
    from paper_1607_02955_gb300 import build_ext
    build_ext.build()
    rng = np.random.default_rng(4)
    out = {name: accuracy_rows(P, torch, spec, (0.5, 0.4, 0.3, 0.2, 0.1, 0.05), (10, 30, 100, 300, 1000), rng)
           for name, spec in ACCURACY_GRAPHS.items()}
    print(json.dumps({"metric": "estimator accuracy vs device time", "data": "synthetic", "n_gpus": 1,
                      "config": {"workload": "accuracy", "queried": "every node"}, "accuracy": out}), flush=True)


def serve_main(args):
    """The serving mix: 16 resident graphs, Poisson arrivals at 0.25, 0.5 and
    0.8 of the measured saturation rate, p50/p99 latency."""
    import torch
    torch.cuda.init()
    import paper_1607_02955_gb300 as P
    from paper_1607_02955_gb300 import build_ext
    build_ext.build()
    resident = getattr(args, "resident_pivots", False)
    r = run_serving(P, SERVE_GRAPHS, n_queries=max(64, 16 * args.steps), loads=(0.25, 0.5, 0.8),
                    resident=resident)
    mid = r["loads"][1]
    print(json.dumps({"metric": "query p99 latency at 0.5x saturation", "value": mid["p99_ms"], "unit": "ms",
                      "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
                      "scaling": "none", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                      "config": {"workload": "serve_mix",
                                 "estimator": ("sampling, one resident set of 200 pivots per graph" if resident
                                               else "sampling, 200 pivots per query"),
                                 "query_nodes": "1..32 uniform", "arrivals": "Poisson"},
                      "serving": r}), flush=True)


def hier_opts(P, args):
    """Hierarchy options from the command line (library defaults otherwise)."""
    kw = {}
    if getattr(args, "coarse_max", None) is not None:
        kw["coarse_max"] = args.coarse_max
    if getattr(args, "aggregation", None) is not None:
        kw["aggregation"] = {"strength": 0, "affinity": 1}[args.aggregation]
    if getattr(args, "hub_factor", None) is not None:
        kw["hub_factor"] = args.hub_factor
    if getattr(args, "chunking", None) is not None:
        kw["chunking"] = args.chunking
    if getattr(args, "reorder", None) is not None:
        kw["reorder"] = args.reorder
    return P.lap_default_hier_opts(**kw)


def gpu_workload(P, torch, name, args, steps, warmup, local, world, clk=None, full=True):
    """Times `steps` steps of a workload on this rank's GPU (after `warmup`
    untimed ones), device-resident inputs, L2 flushed between steps.  With
    `full`: also the same steps through the C ABI with host buffers (e2e),
    the launch count, and an instrumented pass (per-family device time by
    CUDA events on the launching stream)."""
    wl = WORKLOADS[name]
    n, s, d, w = make_graph(wl)
    k = wl["k"]
    nodes = np.array(wl["nodes"], np.int32)
    dev = torch.device("cuda", local)
    src_d = torch.tensor(s, dtype=torch.int32, device=dev)
    dst_d = torch.tensor(d, dtype=torch.int32, device=dev)
    w_d = torch.tensor(w, dtype=torch.float64, device=dev) if w is not None else None
    nodes_d = torch.tensor(nodes, device=dev)
    far_d = torch.empty(len(nodes), dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(device=dev)
    sp = stream.cuda_stream
    prec_mode, dtype, prec_text = PRECISIONS[args.precision]
    sopts = P.lap_default_solve_opts(precision=prec_mode)
    if args.levels is not None:
        sopts.levels_used = args.levels
    hopts = hier_opts(P, args)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2

    rank = int(os.environ.get("RANK", "0"))

    def farness(h, nodes_arg, out):
        """One GPU: the whole query.  N GPUs: one query of k * N rows, this
        rank's k rows (cfc_farness_jl_rows), then one all-reduce of the q
        partial sums on the device (the split's only exchange)."""
        if world == 1:
            P.cfc_farness_jl(h, k, wl["jl_seed"], nodes_arg, opts=sopts, out=out, stream=sp)
            return
        import torch.distributed as dist
        P.cfc_farness_jl_rows(h, k * world, k * rank, k, wl["jl_seed"], nodes_arg, opts=sopts, out=out, stream=sp)
        t = out if out.is_cuda else out.to(dev)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        if t is not out:
            out.copy_(t.cpu())

    def step_device():
        h = P.lap_build_hierarchy(n, src_d, dst_d, w_d, hopts, stream=sp)
        farness(h, nodes_d, far_d)
        h.destroy()

    # host-buffer variant: pinned host inputs, result read back to the host
    src_h = torch.tensor(s, dtype=torch.int32).pin_memory()
    dst_h = torch.tensor(d, dtype=torch.int32).pin_memory()
    w_h = torch.tensor(w, dtype=torch.float64).pin_memory() if w is not None else None
    far_h = torch.empty(len(nodes), dtype=torch.float64).pin_memory()

    def step_host():
        h = P.lap_build_hierarchy(n, src_h, dst_h, w_h, hopts, stream=sp)
        farness(h, nodes, far_h)
        h.destroy()

    def timed(step, K):
        total = 0.0
        with torch.cuda.stream(stream):
            for _ in range(K):
                flush.fill_(1.0)
                torch.cuda.synchronize()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                step()
                b.record(stream)
                b.synchronize()
                total += a.elapsed_time(b)
        return total

    for _ in range(warmup):
        step_device()
        if full:
            step_host()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    P.lap_stats_reset()
    P.lap_stats_set_log(full and args.launch_log is not None)
    if clk is not None:
        clk.mark()
    torch.cuda.profiler.start()  # ncu --profile-from-start off captures exactly the timed steps
    ms_total = timed(step_device, steps)
    torch.cuda.profiler.stop()
    P.lap_stats_set_log(False)
    stats = P.lap_stats_read()
    if world > 1:
        # the distributed result against the same query of k * N rows on this GPU alone
        with torch.cuda.stream(stream):
            step_device()
            h = P.lap_build_hierarchy(n, src_d, dst_d, w_d, hopts, stream=sp)
            one = P.cfc_farness_jl(h, k * world, wl["jl_seed"], nodes, opts=sopts, stream=sp)
            h.destroy()
        split_err = float(np.max(np.abs(far_d.cpu().numpy() - one) / np.abs(one)))
    out = {"wl": wl, "wl_name": name, "n": n, "m": int(s.size), "k": k, "dtype": dtype, "prec_text": prec_text, "sopts": sopts,
           "graph": (n, src_d, dst_d, w_d), "stream": stream, "dev": dev, "launches": stats["launches_total"],
           "split_check": ({"quantity": f"farness of node(s) {wl['nodes']} from {world} row shards + all-reduce "
                                        f"against the same {k * world}-row query on one GPU",
                            "max_rel_err": split_err, "bound": 1e-6} if world > 1 else None)}
    if full and args.launch_log and int(os.environ.get("RANK", "0")) == 0:
        with open(args.launch_log, "w") as fh:
            json.dump({"workload": name, "steps": steps, "source_digest": kernel_source_digest(),
                       "families": P.lap_stats_read_log()}, fh)
    out["clocks"] = clk.stop() if clk is not None else None
    torch.cuda.synchronize()
    barrier(world)
    ms_total = max_over_ranks(ms_total, world)
    out["ms_step"] = ms_total / steps
    out["value"] = k * world / (out["ms_step"] / 1e3)
    if not full:
        return out
    # end to end through the C ABI with host buffers
    barrier(world)
    ms_e2e = max_over_ranks(timed(step_host, steps) / steps, world)
    out["e2e"] = {"value": k * world / (ms_e2e / 1e3), "unit": "RHS/s",
                  "h2d_bytes_per_step": int(s.size) * (4 + 4 + (8 if w is not None else 0)) + len(nodes) * 4,
                  "d2h_bytes_per_step": len(nodes) * 8}
    # instrumented pass: per-kernel-family device time by CUDA events on the launch stream
    P.lap_stats_reset()
    P.lap_stats_set_timing(True)
    timed(step_device, steps)
    out["families"] = P.lap_stats_read()["families"]
    P.lap_stats_set_timing(False)
    return out


def solve_rate(P, torch, res, precision, kk, reps):
    """Solve-only rate on a built hierarchy (setup excluded), the same 1e-8
    FP64 residual test; the first solve autotunes for its configuration."""
    n, src_d, dst_d, w_d = res["graph"]
    stream, dev, wl = res["stream"], res["dev"], res["wl"]
    sp = stream.cuda_stream
    h = P.lap_build_hierarchy(n, src_d, dst_d, w_d, stream=sp)
    Yk = torch.empty((n, kk), dtype=torch.float64, device=dev)
    Xk = torch.empty_like(Yk)
    P.cfc_jl_rhs(h, kk, wl["jl_seed"], Yk, stream=sp)
    o = P.lap_default_solve_opts(precision=precision)
    P.lap_solve_multi(h, Yk, Xk, o, stream=sp)
    with torch.cuda.stream(stream):
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            inf = P.lap_solve_multi(h, Yk, Xk, o, stream=sp)
        b.record(stream)
        b.synchronize()
    h.destroy()
    return {"rhs_per_s": kk * reps / (a.elapsed_time(b) / 1e3), "k": kk, "solves": reps,
            "inner_iters": inf["inner_iters"], "max_rel_residual": inf["max_rel_residual"]}


def precision_comparison(P, torch, res, args):
    """The batched mixed-precision solve against FP64 batched and FP64 one
    right-hand side at a time (solve only, same 1e-8 test)."""
    prec_mode = PRECISIONS[args.precision][0]
    k = res["k"]
    return {"solve_only": True, "workload": res["wl_name"],
            args.precision + "_batched": solve_rate(P, torch, res, prec_mode, k, 3),
            "fp64_batched": solve_rate(P, torch, res, 0, k, 1),
            "fp64_one_rhs": solve_rate(P, torch, res, 0, 1, 4)}


def parity_large(P, torch, res, g, L, threads):
    """This run's error against the oracle at a size the oracle cannot solve
    within the bench: the first 8 JL right-hand sides (k = 64 scaling) on the
    device against the oracle's at sampled nodes (jl_rhs_at), and the
    oracle's FP64 residual ||Y - L Z|| / ||Y|| of the device's solutions of
    those columns (a property every solution at 1e-8 has, at any size)."""
    from concurrent.futures import ThreadPoolExecutor
    from oracle import jl
    n, src_d, dst_d, w_d = res["graph"]
    wl, stream, dev = res["wl"], res["stream"], res["dev"]
    sp = stream.cuda_stream
    k, ks = wl["k"], CPU_SAMPLE_ROWS
    h = P.lap_build_hierarchy(n, src_d, dst_d, w_d, stream=sp)
    Y = torch.empty((n, k), dtype=torch.float64, device=dev)
    P.cfc_jl_rhs(h, k, wl["jl_seed"], Y, stream=sp)
    Y8 = Y[:, :ks].contiguous()
    del Y
    Z8 = torch.empty_like(Y8)
    info = P.lap_solve_multi(h, Y8, Z8, res["sopts"], stream=sp)
    h.destroy()
    torch.cuda.synchronize()
    Yh, Zh = Y8.cpu().numpy(), Z8.cpu().numpy()
    del Y8, Z8
    deg = np.diff(L.indptr)
    nodes = [0, int(np.argmax(deg)), n // 2, n - 1]
    Yo = jl.jl_rhs_at(g, k, wl["jl_seed"], nodes)[:ks]  # k x len(nodes) -> first ks rows
    rhs_err = float(np.abs(Yh[nodes, :].T - Yo).max() / np.abs(Yo).max())
    chunks = [c for c in np.array_split(np.arange(ks), min(threads, ks)) if c.size]
    with ThreadPoolExecutor(len(chunks)) as ex:
        LZ = list(ex.map(lambda c: L @ Zh[:, c], chunks))
    R = np.empty_like(Yh)
    for c, v in zip(chunks, LZ):
        R[:, c] = v
    Yp = Yh - Yh.mean(axis=0)
    rel = np.linalg.norm(Yp - R, axis=0) / np.linalg.norm(Yp, axis=0)
    return {"quantity": f"JL right-hand sides 0-{ks - 1} at nodes {nodes} against the oracle, and the oracle's "
                        f"FP64 residual of the device's solutions of those columns",
            "rhs_rel_err": rhs_err, "rhs_bound": 1e-13, "max_rel_residual": float(rel.max()), "bound": 1e-8,
            "device_reported_residual": info["max_rel_residual"]}


def roofline_of(res, steps, P):
    """The dominant solver kernel family's algorithmic bytes over its
    event-timed duration, against the measured copy bandwidth, and the
    HBM-roofline ideal of the whole solve."""
    fam = res["families"]
    solve_fams = {kf: v for kf, v in fam.items() if v["ms"] > 0 and kf not in ("setup", "cfc")}
    dom = max(solve_fams, key=lambda kf: solve_fams[kf]["ms"])
    peak, peak_src = read_peaks()
    dm = fam[dom]
    achieved = (dm["bytes"] / 1e9) / (dm["ms"] / 1e3) if dm["ms"] > 0 else 0.0
    traffic, traffic_kernel, traffic_note = read_traffic(res["wl_name"], dom)
    per_launch = dm["bytes"] / max(dm["launches"], 1)
    roof = {"bound": "hbm", "kernel_family": dom, "achieved": achieved, "peak": peak,
            "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else peak_src,
            "unit": "GB/s", "frac": achieved / peak, "traffic": traffic, "traffic_kernel": traffic_kernel,
            "traffic_note": traffic_note, "algorithmic_bytes_per_launch": per_launch,
            "traffic_over_algorithmic": traffic / per_launch if traffic else None,
            "launches": dm["launches"], "ms": dm["ms"]}
    k = res["k"]
    solve_bytes = sum(v["bytes"] for v in solve_fams.values()) / steps
    solve_ms = sum(v["ms"] for v in solve_fams.values()) / steps
    ideal = {"rhs_per_s": k / (solve_bytes / (peak * 1e9)) if solve_bytes > 0 else None,
             "solve_bytes_per_step": solve_bytes, "measured_solve_ms_per_step": solve_ms,
             "measured_rhs_per_s_solve_kernels": k / (solve_ms / 1e3) if solve_ms > 0 else None}
    achieved_by_family = {kf: (v["bytes"] / 1e9) / (v["ms"] / 1e3) for kf, v in fam.items()
                          if v["ms"] > 0 and v["bytes"] > 0}
    return roof, ideal, achieved_by_family


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS) + ["serve_mix", "accuracy"])
    ap.add_argument("--no-serving", action="store_true", help="skip the small serving mix of the default line")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the BA 100k block (its rate and the FP64 batched / one-RHS comparison)")
    ap.add_argument("--print-digest", action="store_true", help="print the kernel source digest and exit")
    ap.add_argument("--levels", type=int, default=None,
                    help="levels_used of the V-cycle (default: autotuned; -1: every level)")
    ap.add_argument("--coarse-max", type=int, default=None,
                    help="hierarchy option coarse_max (default 0: automatic, n / 4096 in [256, 1024])")
    ap.add_argument("--aggregation", default=None, choices=["strength", "affinity"],
                    help="hierarchy option aggregation (default: strength)")
    ap.add_argument("--hub-factor", type=int, default=None,
                    help="hierarchy option hub_factor (default 0: no hub rule)")
    ap.add_argument("--resident-pivots", action="store_true",
                    help="serve_mix: one resident pivot set per graph (requests solve only their nodes)")
    ap.add_argument("--reorder", type=int, default=None, choices=[0, 1, 2],
                    help="hierarchy option reorder (default 0: longest rows first where row lengths are uneven)")
    ap.add_argument("--chunking", type=int, default=None, choices=[0, 1, 2],
                    help="hierarchy option chunking (default 0: by level size)")
    ap.add_argument("--precision", default="fp32", choices=sorted(PRECISIONS),
                    help="arithmetic of the solve (fp32: FP32 PCG + V-cycle in FP64 refinement)")
    ap.add_argument("--launch-log", default=None,
                    help="write the kernel family of every launch in the timed steps to this JSON file")
    ap.add_argument("--write-traffic", nargs=2, metavar=("NCU_CSV", "LAUNCH_LOG"), default=None,
                    help="no GPU: attribute the DRAM bytes of an ncu launch list of the timed steps "
                         "to kernel families and record them in profiles/traffic.json")
    args = ap.parse_args()
    if args.print_digest:
        print(kernel_source_digest())
        return
    if args.write_traffic:
        write_traffic(*args.write_traffic)
        return
    if args.workload == "serve_mix":
        serve_main(args)
        return
    if args.workload == "accuracy":
        accuracy_main(args)
        return
    wl = WORKLOADS[args.workload]
    rank, world, local = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, wl, rank, world)
        return

    import torch
    torch.cuda.set_device(local)
    torch.cuda.init()
    import paper_1607_02955_gb300 as P
    from paper_1607_02955_gb300 import build_ext
    build_ext.build()

    clk = ClockSampler(local)
    res = gpu_workload(P, torch, args.workload, args, args.steps, args.warmup, local, world, clk=clk)
    n, k = res["n"], res["k"]
    roof, ideal, by_family = roofline_of(res, args.steps, P)
    fam = res["families"]

    # setup alone (ingest + hierarchy) and solver iteration counts, for context
    gn, src_d, dst_d, w_d = res["graph"]
    sp = res["stream"].cuda_stream
    hopts = hier_opts(P, args)
    h = P.lap_build_hierarchy(gn, src_d, dst_d, w_d, hopts, stream=sp)
    Y = torch.empty((n, k), dtype=torch.float64, device=res["dev"])
    X = torch.empty_like(Y)
    P.cfc_jl_rhs(h, k, wl["jl_seed"], Y, stream=sp)
    sinfo = P.lap_solve_multi(h, Y, X, res["sopts"], stream=sp)
    hinfo = P.lap_hierarchy_info(h)
    h.destroy()
    del Y, X

    large = wl_nodes(wl) > LARGE_N
    if rank == 0:
        line = {
            "metric": METRIC, "value": res["value"], "unit": "RHS/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["ms_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": res["dtype"], "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "m": res["m"], "k": k,
                       "query_nodes": wl["nodes"], "tol": 1e-8, "precision": res["prec_text"],
                       "setup_included": True,
                       "l2": "flushed between steps (256 MiB write, untimed)" +
                             ("; every FP32 block (n x 64 x 4 B) is larger than L2" if large else ""),
                       "levels_built": hinfo["levels"], "level_n": hinfo["level_n"], "setup_ms": hinfo["setup_ms"],
                       "level_row_order": hinfo["level_row_order"], "elim_levels": hinfo["elim_levels"],
                       "hier_opts": {"coarse_max": hopts.coarse_max, "aggregation": hopts.aggregation,
                                     "hub_factor": hopts.hub_factor, "eliminate": hopts.eliminate,
                                     "chunking": hopts.chunking, "reorder": hopts.reorder},
                       "solve": {key: sinfo[key] for key in ("outer_iters", "inner_iters", "max_rel_residual",
                                                              "k_tile", "levels_used", "nu_coarse", "cycle",
                                                              "coarse_scale", "w_levels")},
                       "parallelism": (f"one JL query of {k * world} rows split over {world} GPUs ({k} rows each, "
                                       f"replicated graph), one NCCL all-reduce of the q partial sums"
                                       if world > 1 else "one GPU")},
            "e2e": res["e2e"],
            "gpu_launches": res["launches"],
            "roofline": roof,
            "achieved_gbs_by_family": by_family,
            "family_ms_per_step": {kf: v["ms"] / args.steps for kf, v in fam.items()},
            "solve_roofline_ideal": ideal,
            "clocks": res["clocks"],
        }
        if res.get("split_check"):
            line["split_check"] = res["split_check"]
        if world == 1 and not args.no_compare:
            if large:
                # the 100k-node BA configuration: its own rate and the FP64 comparison
                ba = gpu_workload(P, torch, "ba100k_jl64", args, 10, 3, local, 1, full=False)
                line["ba100k_jl64"] = {"value": ba["value"], "unit": "RHS/s", "ms_per_step": ba["ms_step"],
                                       "steps": 10, "precision_comparison": precision_comparison(P, torch, ba, args)}
                del ba
            else:
                res2 = gpu_workload(P, torch, args.workload, args, 1, 1, local, 1, full=False)
                line["precision_comparison"] = precision_comparison(P, torch, res2, args)
                del res2
        if world == 1 and not args.no_compare:
            # the accuracy experiment (Sec. 6.4's shape) at two settings of each estimator
            line["accuracy"] = {"ba3000": accuracy_rows(P, torch, ACCURACY_GRAPHS["ba3000"], (0.3, 0.1), (10, 100),
                                                         np.random.default_rng(4)),
                                "note": "every node queried; exact farness from the dense pseudoinverse on the "
                                        "device; `--workload accuracy` runs the full sweep on two graphs"}
        if world == 1 and not args.no_serving:
            line["serving"] = run_serving(P, SERVE_SMALL, n_queries=48, loads=(0.5,))
            line["serving_resident_pivots"] = run_serving(P, SERVE_SMALL, n_queries=48, loads=(0.5,),
                                                          resident=True)
        if world == 1 and not args.no_cpu_baseline:
            threads = oracle_threads()
            if large:
                gL = oracle_graph(wl)
                line["cpu_baseline"], _ = cpu_baseline(wl, threads, gL)
                line["parity"] = parity_large(P, torch, res, gL[0], gL[1], threads)
                del gL
            else:
                line["cpu_baseline"], Zo = cpu_baseline(wl, threads)
                # this run's error against the oracle on the same sample: the JL
                # farness terms of rows 0..7 for the query node (Algorithm 1)
                v = int(wl["nodes"][0])
                f_or = float(((Zo - Zo[:, [v]]) ** 2).sum())
                n0, s0, d0, w0 = make_graph(wl)
                h = P.lap_build_hierarchy(n0, s0, d0, w0)
                f_gpu = float(P.cfc_farness_jl_rows(h, k, 0, CPU_SAMPLE_ROWS, wl["jl_seed"],
                                                    np.array([v], np.int32))[0])
                h.destroy()
                line["parity"] = {"quantity": f"JL farness terms of rows 0-{CPU_SAMPLE_ROWS - 1} for node {v}",
                                  "oracle": f_or, "gpu": f_gpu, "rel_err": abs(f_gpu - f_or) / abs(f_or),
                                  "bound": 1e-6}
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
