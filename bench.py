#!/usr/bin/env python
"""Benchmark of the Steiner-tree hot path on GB300.

One step = one query through the whole path (Voronoi cells, predecessor and
bridge scan, pair compaction, MST, expansion, sorted tree and total) on the
largest single-query workload: an R-MAT scale-26 graph (67M vertices, 2.1G
arcs, weights uniform in [1, 1000]) with 10,000 seeds drawn uniformly from
its largest component (``--workload 2`` runs the 4096 x 4096 grid with 256
seeds, ``--workload 1`` R-MAT 16 with 16 seeds).  Inputs (graph and seed
set) are seeded and synthetic.  The autotuner tunes on another seed set of
the same size from the same pool, never on the timed one.

Printed (rank 0, one JSON line):
  value      trees/s from device time (CUDA events on the library's stream,
             graph resident in HBM), summed over ranks (replicas: each rank
             runs its own queries)
  e2e        trees/s through the C ABI with host seed lists in and host tree
             edges out (copies inside the timed region)
  roofline   the Voronoi SSSP kernel's algorithmic bytes per launch / its
             event-timed duration, against the measured HBM copy bandwidth
  cpu_baseline  the CPU oracle timed on one host core on one whole query
             of the workload (rank 0, N = 1), run in a child process forked
             before any CUDA call so it overlaps the GPU measurement

``--impl reference`` times the CPU oracle itself on the same workload.
Multi-GPU: ``torchrun --nproc-per-node N bench.py --gpus N``; ranks are
independent replicas (queries never exchange data), barrier + max-over-ranks
timing.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = 3            # R-MAT scale 26, 10,000 seeds
GRID = 2                # the 4096^2 grid, 256 seeds
TUNE_SALT = 0x7E57      # seed-set salt of the autotuner's held-out sample
REF_BUDGET_S = 300.0    # reference arm: whole oracle queries within this time
SSSP_SOURCES = ["paper_2205_14503_gb300/csrc/voronoi.cu", "paper_2205_14503_gb300/csrc/common.cuh",
                "paper_2205_14503_gb300/csrc/internal.h"]


def _code_only(src: str) -> str:
    """C/CUDA source without comments and with whitespace collapsed, so a
    comment edit does not void a capture of the same code."""
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return " ".join(src.split())


def sssp_source_hash() -> str:
    h = hashlib.sha256()
    for p in SSSP_SOURCES:
        with open(os.path.join(ROOT, p), encoding="utf-8") as f:
            h.update(_code_only(f.read()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(workload_name: str):
    """DRAM bytes per SSSP launch from the committed ncu summary of this
    workload, or None if it is absent or the kernel source changed since."""
    try:
        text = open(os.path.join(ROOT, "profiles", f"sssp_{workload_name}.md")).read()
    except OSError:
        return None
    m1 = re.search(r"sssp_source_hash:\s*([0-9a-f]+)", text)
    m2 = re.search(r"traffic_bytes_per_launch:\s*([0-9]+)", text)
    if not m1 or not m2 or m1.group(1) != sssp_source_hash():
        return None
    return int(m2.group(1))


def measured_peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(gpu_index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[3:7]):
                if flag.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload(rank: int, side: int | None = None, k: int | None = None, cfg: int = WORKLOAD,
             scale: int | None = None):
    """The benchmark graph, the timed seed set and the autotuner's held-out
    seed set (same size, same pool, another salt).  ``side``/``k`` shrink
    the grid, ``scale``/``k`` the R-MAT graph, for profiling captures (same
    recipe and seed density unless k is given); ``cfg`` picks the
    single-query workload (3 R-MAT 26, the default; 2 the grid; 1 R-MAT 16)."""
    import paper_2205_14503_gb300.workloads as wl
    if scale:
        c = wl.CONFIGS[3]
        g = wl.rmat(scale, 16, (0.57, 0.19, 0.19), c["wmax"], wl.CONFIG_SEED + 3, True)
        pool = wl.largest_cc(g)
        kk = k or max(2, round(c["k"] * 2.0 ** (scale - c["scale"])))
        seeds = wl.sample_distinct(pool, kk, (wl.CONFIG_SEED + 3) ^ 0x51ED)
    elif side:
        g = wl.grid(side, side, 1000, wl.CONFIG_SEED + GRID)
        pool = np.arange(g.n, dtype=np.int32)
        seeds = wl.sample_distinct(pool, k or 64, (wl.CONFIG_SEED + GRID) ^ 0x51ED)
    else:
        g = wl.config_graph(cfg)
        seeds = wl.config_seed_sets(cfg, g)[0]
        pool = np.arange(g.n, dtype=np.int32) if cfg == GRID else wl.largest_cc(g)
    if rank > 0:    # replicas run their own queries of the same size
        seeds = wl.sample_distinct(pool, seeds.size, 0x5EED + cfg + 1000 * rank)
    tune_seeds = wl.sample_distinct(pool, seeds.size, 0x5EED + cfg + TUNE_SALT + 1000 * rank)
    return g, seeds, tune_seeds


def heldout_queries(g, cfg: int, count: int, pool=None):
    """``count`` seed sets drawn like workload ``cfg``'s query stream but
    with other salts: the autotuner's sample, never the timed queries."""
    import paper_2205_14503_gb300.workloads as wl
    c = wl.CONFIGS[cfg]
    pool = wl.largest_cc(g) if pool is None else pool
    base = wl.CONFIG_SEED + cfg + TUNE_SALT
    ks = wl.log_uniform_sizes(count, c["klo"], c["khi"], base ^ 0x517E)
    return [wl.sample_distinct(pool, int(k), base + 7919 * i) for i, k in enumerate(ks)]


def host_info() -> dict:
    ram = None
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemTotal:"):
                    ram = round(int(line.split()[1]) / 2 ** 20, 1)
    except OSError:
        pass
    import platform
    return {"host_cores": os.cpu_count(), "host_ram_gib": ram, "machine": platform.machine()}


def start_oracle_child(g, seeds):
    """Forks a child that times one whole oracle query of (g, seeds) on one
    host core and writes the result to a pipe.  Call before any CUDA call in
    this process (a fork after CUDA initialisation is not safe)."""
    r, w = os.pipe()
    pid = os.fork()
    if pid == 0:        # child: no CUDA here
        os.close(r)
        try:
            import oracle
            t0 = time.perf_counter()
            res = oracle.steiner(g, seeds, want_labels=False)
            dt = time.perf_counter() - t0
            msg = {"seconds": dt, "status": int(res.status), "total": int(res.total),
                   "edges_sha": hashlib.sha256(np.ascontiguousarray(res.edges, np.uint32)
                                               .tobytes()).hexdigest()}
        except Exception as e:      # reported, not raised, in the parent
            msg = {"error": repr(e)}
        data = json.dumps(msg).encode()
        while data:
            data = data[os.write(w, data):]
        os._exit(0)
    os.close(w)
    return pid, r


def finish_oracle_child(child):
    pid, r = child
    chunks = []
    while True:
        b = os.read(r, 65536)
        if not b:
            break
        chunks.append(b)
    os.close(r)
    os.waitpid(pid, 0)
    try:
        return json.loads(b"".join(chunks).decode())
    except ValueError:
        return {"error": "oracle child gave no result"}


def config_dict(g, seeds, cfg: int = WORKLOAD, side: int | None = None,
                scale: int | None = None):
    import paper_2205_14503_gb300.workloads as wl
    if scale:
        name = f"rmat{scale}_k{seeds.size}"
        desc = f"R-MAT scale {scale}, edge factor 16, (a,b,c)=(.57,.19,.19), w~U[1,1000]"
    elif side or cfg == GRID:
        s = int(round(g.n ** 0.5))
        name, desc = f"grid{s}_k{seeds.size}", f"{s}x{s} 4-connected grid, w~U[1,1000]"
    else:
        c = wl.CONFIGS[cfg]
        name = c["name"]
        desc = (f"R-MAT scale {c['scale']}, edge factor 16, (a,b,c)=(.57,.19,.19), "
                f"w~U[1,{c['wmax']}]")
    return {"workload": name, "graph": desc,
            "n": int(g.n), "arcs": int(g.n_arcs), "k": int(seeds.size),
            "l2": f"inputs larger than L2 (adjacency {g.n_arcs * 8 >> 20} MiB, "
                  f"labels {g.n * 4 >> 20}-{g.n * 8 >> 20} MiB)",
            "tuning_seeds": f"held-out set of the same size (salt {TUNE_SALT:#x})"}


METRIC = "Steiner trees/s (Voronoi SSSP + bridge scan + MST + expansion)"


def run_reference(args, world, rank):
    """The oracle itself (the paper ships no code) on the same workload,
    metric and unit: each step is one whole query on one host core.  A
    whole query of the R-MAT 26 workload takes minutes, so the arm times
    whole queries within REF_BUDGET_S (at least one) and states in its line
    how many it ran against the steps asked for; the oracle has nothing to
    warm up, so no warm-up query runs when the budget is that short."""
    if rank != 0:
        return
    g, seeds, _ = workload(0, args.side, args.k, args.workload, args.scale)
    import oracle

    def one():
        t0 = time.perf_counter()
        oracle.steiner(g, seeds, want_labels=False)
        return time.perf_counter() - t0

    # The first query sizes the run: if K + W whole queries fit the budget
    # it was a warm-up and the contract's W, K follow; otherwise it is the
    # first timed step and timing goes on only while the budget lasts.
    t_all = time.perf_counter()
    t1 = one()
    times, warm = [], 0
    if (args.steps + args.warmup) * t1 <= REF_BUDGET_S:
        warm = 1
        for _ in range(args.warmup - 1):
            one()
            warm += 1
        times = [one() for _ in range(args.steps)]
    else:
        times = [t1]
        while (len(times) < args.steps
               and time.perf_counter() - t_all + statistics.mean(times) <= REF_BUDGET_S):
            times.append(one())
    total = sum(times)
    value = len(times) / total
    per_q = total / len(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "trees/s",
            "n_gpus": args.gpus, "steps": len(times), "warmup": warm,
            "ms_per_step": 1e3 * per_q, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": config_dict(g, seeds, args.workload, args.side, args.scale),
            "cpu_baseline": {"kind": "oracle", "value": value, "unit": "trees/s", "cores": 1,
                             "sample": f"{len(times)} whole queries of the workload, "
                                       "single-threaded C oracle", **host_info()},
            "e2e": {"value": value, "unit": "trees/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    if len(times) < args.steps or warm < args.warmup:
        line["requested"] = {"steps": args.steps, "warmup": args.warmup}
        line["note"] = (f"one whole oracle query of this workload takes {per_q:.0f} s here; "
                        f"{args.steps + args.warmup} of them would take "
                        f"{(args.steps + args.warmup) * per_q / 60:.0f} min, so the arm timed "
                        f"{len(times)} whole queries (and {warm} warm-up) within "
                        f"{REF_BUDGET_S:.0f} s")
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_14503_gb300 import steiner as st

    g, seeds, tune_seeds = workload(rank, args.side, args.k, args.workload, args.scale)
    # the CPU baseline runs beside the GPU measurement, in a child forked
    # before this process makes its first CUDA call
    child = (start_oracle_child(g, seeds)
             if world == 1 and rank == 0 and not args.no_cpu_baseline else None)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (no CPU fallback)")
    torch.cuda.set_device(local)
    t0 = time.perf_counter()
    G = st.SteinerGraph(g, device=local)
    load_s = time.perf_counter() - t0
    tuned = None
    if args.tuned:
        # explicit (delta, blocks, local rounds), e.g. for profiling captures
        vals = [int(x) for x in args.tuned.split(",")]
        d, b, lr, lb, fs, tl = vals + [0, 0, 0, 0, -1, 1][len(vals):]
        G.set_param("delta", d)
        G.set_param("sssp_blocks", b)
        G.set_param("local_rounds", lr)
        G.set_param("label_bits", lb)
        G.set_param("far_scan", fs)
        G.set_param("tail", tl)
        tuned = {"delta": d, "sssp_blocks": G.get_param("sssp_blocks"), "local_rounds": lr,
                 "label_bits": lb, "far_scan": fs, "tail": tl}
    elif not args.no_autotune:
        # set-up, untimed: band width, grid size, label width and split mode
        # for this graph, tuned on the held-out seed set
        from paper_2205_14503_gb300 import autotune
        tuned = autotune.tune(G, g, [tune_seeds], cache_path=None, device=local)
    for _ in range(max(args.warmup, 3)):
        r = G.query_detail(seeds, pairs=False)
        if r.status != st.STEINER_OK:
            raise SystemExit(f"warm-up query failed: {st.STATUS_NAMES[r.status]} {st.last_error()}")

    # device-timed pass (graph and seed set resident; per-phase CUDA events)
    barrier(world)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    phase = {k: [] for k in ("ms_init", "ms_voronoi", "ms_bridges", "ms_mst", "ms_tree")}
    launches = 0
    stats = None
    for _ in range(args.steps):
        r = G.query_detail(seeds, pairs=False)
        stats = r.stats
        for k in phase:
            phase[k].append(stats[k])
        launches += stats["gpu_launches"]
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    dev_ms = [sum(phase[k][i] for k in phase) for i in range(args.steps)]
    dev_s = max_over_ranks(sum(dev_ms) / 1e3, world)

    # end-to-end pass through the C ABI: host seeds in, host edges out
    barrier(world)
    torch.cuda.synchronize()
    lat = []
    t_start = time.perf_counter()
    for _ in range(args.steps):
        t0 = time.perf_counter()
        res = G.query(seeds)
        lat.append(time.perf_counter() - t0)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t_start, world)
    barrier(world)
    label_bits = G.get_param("label_bits_last")      # the width the timed queries used
    narrow_reruns = G.get_param("narrow_reruns")
    pull_passes = G.get_param("pull_passes_last")
    tail_iteration = G.get_param("tail_iteration_last")
    G.close()

    if rank != 0:
        return
    total_q = args.steps * world
    value = total_q / dev_s
    n, m_arcs = g.n, g.n_arcs
    sssp_ms = statistics.mean(phase["ms_voronoi"])
    # per SSSP launch (one query): every arc record (8 B) and the head's
    # label once, every row offset and label once; labels are 4 or 8 bytes
    lb = label_bits // 8
    alg_bytes = (8 + lb) * m_arcs + (4 + lb) * n
    peak, peak_kind = measured_peak_hbm()
    achieved = alg_bytes / (sssp_ms / 1e3) / 1e9
    cfgd = config_dict(g, seeds, args.workload, args.side, args.scale)
    traffic = profiled_traffic(cfgd["workload"])
    line = {
        "metric": METRIC, "value": value, "unit": "trees/s", "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": 1e3 * dev_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": cfgd,
        "roofline": {"kernel": "sssp_kernel (Voronoi near/far SSSP)", "bound": "hbm",
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind,
                     "traffic": traffic, "alg_bytes_per_launch": alg_bytes,
                     "alg_bytes_rule": f"(8 + {lb}) B per arc + (4 + {lb}) B per vertex "
                                       f"({label_bits}-bit labels)",
                     "launch_ms": sssp_ms},
        "e2e": {"value": total_q / e2e_s, "unit": "trees/s",
                "h2d_bytes_per_step": int(seeds.size * 4),
                "d2h_bytes_per_step": int(res.edges.shape[0] * 12 + 8),
                "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                "p99_ms": 1e3 * float(np.percentile(lat, 99))},
        "gpu_launches": launches,
        "gteps": (g.n_arcs // 2) / (sssp_ms / 1e3) / 1e9,
        "phase_ms": {k: statistics.mean(v) for k, v in phase.items()},
        "sssp": {"iterations": stats["iterations"], "phases": stats["phases"],
                 "relax_attempts": stats["relax_attempts"],
                 "work_efficiency": stats["relax_attempts"] / m_arcs,
                 "delta": tuned["delta"] if tuned else None,
                 "blocks": tuned["sssp_blocks"] if tuned else None,
                 "local_rounds": tuned["local_rounds"] if tuned else None,
                 "label_bits": label_bits, "narrow_reruns": narrow_reruns,
                 "far_scan": tuned.get("far_scan") if tuned else None,
                 "tail": tuned.get("tail") if tuned else None,
                 "pull_passes": pull_passes, "tail_iteration": tail_iteration,
                 "autotuned": bool(tuned) and not args.tuned},
        "tree": {"edges": int(res.edges.shape[0]), "total": int(res.total)},
        "graph_load_s": load_s,
        "clocks": clocks,
    }
    if child is not None:
        ref = finish_oracle_child(child)
        if "error" in ref:
            line["cpu_baseline"] = {"kind": "oracle", "value": None, "unit": "trees/s",
                                    "cores": 1, "error": ref["error"]}
        else:
            gpu_sha = hashlib.sha256(np.ascontiguousarray(res.edges, np.uint32)
                                     .tobytes()).hexdigest()
            same = bool(ref["total"] == res.total and ref["edges_sha"] == gpu_sha)
            line["cpu_baseline"] = {"kind": "oracle", "value": 1.0 / ref["seconds"],
                                    "unit": "trees/s", "cores": 1,
                                    "sample": "1 whole query of the workload, single-threaded C "
                                              "oracle (run beside the GPU measurement)",
                                    "seconds": ref["seconds"], "matches_gpu": same,
                                    **host_info()}
    print(json.dumps(line), flush=True)


def run_batch_mode(args, world, rank, local):
    """R-MAT scale 22, 64 queries of log-uniform size in [3, 1000] in one
    batched run, against the same queries one at a time (plain path)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2205_14503_gb300.workloads as wl
    from paper_2205_14503_gb300 import steiner as st
    torch.cuda.set_device(local)
    if args.batch_scale:
        # profiling only: an R-MAT graph of another scale, same query recipe
        c = wl.CONFIGS[4]
        g = wl.rmat(args.batch_scale, 16, (0.57, 0.19, 0.19), c["wmax"], wl.CONFIG_SEED + 4, True)
        pool = wl.largest_cc(g)
        ks = wl.log_uniform_sizes(c["queries"], c["klo"], c["khi"], (wl.CONFIG_SEED + 4) ^ 0x517E)
        qs = [wl.sample_distinct(pool, int(k), (wl.CONFIG_SEED + 4 + 0xC0FFEE) + 7919 * i)
              for i, k in enumerate(ks)]
    else:
        g = wl.config_graph(4)
        qs = wl.config_seed_sets(4, g)
    if rank > 0:
        pool = wl.largest_cc(g)
        qs = [wl.sample_distinct(pool, q.size, 0x5EED + 4000 + 97 * rank + i) for i, q in enumerate(qs)]
    G = st.SteinerGraph(g, device=local)
    tuned = btuned = None
    if not args.no_autotune:
        # set-up, untimed, on held-out queries: the graph's single-query
        # settings (the plain comparator) and the batched engine's band width
        from paper_2205_14503_gb300 import autotune
        tq = heldout_queries(g, 4, len(qs))
        tuned = autotune.tune(G, g, tq[:2], cache_path=None, device=local)
        btuned = autotune.tune_batch(G, g, tq)
    for _ in range(max(args.warmup, 3)):
        G.query_batch(qs)
    plain = [G.query(q) for q in qs]
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        rc, res = G.query_batch(qs)
    torch.cuda.synchronize()
    t_batch = max_over_ranks((time.perf_counter() - t0) / args.steps, world)
    G.get_param("batch_reset")
    G.query_batch(qs)
    parts = {k: G.get_param("batch_" + k) / 1e3 for k in ("ms_sssp", "ms_scan", "ms_tail", "ms_admit")}
    t0 = time.perf_counter()
    for q in qs:
        G.query(q)
    t_plain = max_over_ranks(time.perf_counter() - t0, world)
    same = all(a.status == b.status and a.total == b.total and np.array_equal(a.edges, b.edges)
               for a, b in zip(res, plain))
    G.close()
    if rank != 0:
        return
    nq = len(qs) * world
    line = {"metric": "batched Steiner queries/s (64 queries, one batched run)",
            "value": nq / t_batch, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": 1e3 * t_batch,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": f"rmat{args.batch_scale or 22}_batch64", "n": g.n,
                       "arcs": g.n_arcs, "queries": len(qs),
                       "k_range": [3, 1000],
                       "tuned": {k: tuned.get(k) for k in ("delta", "sssp_blocks", "local_rounds",
                                                            "label_bits", "far_scan")}
                       if tuned else None},
            "batch_delta": (btuned or {}).get("batch_delta"),
            "batch_pull": (btuned or {}).get("batch_pull"),
            "plain_queries_per_s": nq / t_plain, "speedup_vs_plain": t_plain / t_batch,
            "identical_to_plain": same, "phase_ms": parts}
    print(json.dumps(line), flush=True)


def run_serve_mode(args, world, rank, local):
    """R-MAT scale 24, a stream of queries with log-uniform size in
    [3, 10000]; saturated throughput (all submitted at once) and p50/p99
    latency at 0.7x that rate (Poisson arrivals); 40 GB per-query budget."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2205_14503_gb300.workloads as wl
    from paper_2205_14503_gb300 import steiner as st
    torch.cuda.set_device(local)
    g = wl.config_graph(5)
    qs = wl.config_seed_sets(5, g)[: args.queries]
    G = st.SteinerGraph(g, device=local)
    h = G.handle
    tuned = btuned = None
    if not args.no_autotune:
        # set-up, untimed, on held-out queries of the same recipe
        from paper_2205_14503_gb300 import autotune
        tq = heldout_queries(g, 5, 64)
        tuned = autotune.tune(G, g, tq[:2], cache_path=None, device=local)
        btuned = autotune.tune_batch(G, g, tq)

    def stream(arrivals):
        st.steiner_serve_start(h, 64, 40 << 30)
        tickets, submit_t, done_t = [], [], {}
        t0 = time.perf_counter()
        pending = set()
        for s, at in zip(qs, arrivals):
            while time.perf_counter() - t0 < at:
                for t in list(pending):
                    rc, _ = st.steiner_poll(h, t)
                    if rc != st.STEINER_PENDING:
                        done_t[t] = time.perf_counter()
                        pending.discard(t)
            rc, t = st.steiner_submit(h, s)
            tickets.append(t)
            submit_t.append(time.perf_counter())
            pending.add(t)
        while pending:
            for t in list(pending):
                rc, _ = st.steiner_poll(h, t)
                if rc != st.STEINER_PENDING:
                    done_t[t] = time.perf_counter()
                    pending.discard(t)
            time.sleep(0.0002)
        wall = time.perf_counter() - t0
        st.steiner_serve_stop(h)
        lat = [done_t[t] - ts for t, ts in zip(tickets, submit_t)]
        return wall, lat

    G.query(qs[0])
    wall_sat, lat_sat = stream([0.0] * len(qs))
    G_yield_div = G.get_param("batch_yield_div")
    qps = len(qs) / wall_sat
    arrivals = wl.poisson_arrivals(len(qs), 0.7 * qps, 0x5EED + 5)
    wall_p, lat_p = stream(arrivals)
    sample = qs[: min(len(qs), args.plain_sample)]
    t0 = time.perf_counter()
    for q in sample:
        G.query(q)
    plain_qps = len(sample) / (time.perf_counter() - t0)
    G.close()
    if rank != 0:
        return
    line = {"metric": "served Steiner queries/s (continuous batching) and p50/p99 time-to-tree",
            "value": qps, "unit": "queries/s", "n_gpus": world, "steps": 1, "warmup": 1,
            "ms_per_step": 1e3 * wall_sat, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "rmat24_serve", "n": g.n, "arcs": g.n_arcs, "queries": len(qs),
                       "k_range": [3, 10000], "budget_bytes": 40 << 30, "slots": 64,
                       "yield_div": G_yield_div,
                       "batch_delta": (btuned or {}).get("batch_delta"),
            "batch_pull": (btuned or {}).get("batch_pull"),
                       "tuned": {k: tuned.get(k) for k in ("delta", "sssp_blocks", "local_rounds",
                                                            "label_bits", "far_scan")}
                       if tuned else None},
            "saturated": {"p50_ms": 1e3 * float(np.percentile(lat_sat, 50)),
                          "p99_ms": 1e3 * float(np.percentile(lat_sat, 99))},
            "poisson_0p7": {"rate_qps": 0.7 * qps, "achieved_qps": len(qs) / wall_p,
                            "p50_ms": 1e3 * float(np.percentile(lat_p, 50)),
                            "p99_ms": 1e3 * float(np.percentile(lat_p, 99))},
            "plain_queries_per_s": plain_qps, "speedup_vs_plain": qps / plain_qps,
            "plain_sample": len(sample)}
    print(json.dumps(line), flush=True)


def run_ablation_mode(args, world, rank, local):
    """Relaxation order (the paper's priority-ordered messages against a
    plain frontier): per single-query workload, the Voronoi phase as a
    Bellman-Ford frontier (one unbounded band), as near/far bands at the
    tuned width with the heavy arcs pushed, pushed or pulled, and pulled
    then followed by the unbounded tail, and with the tuned block-local
    rounds; time, relaxations per arc and iterations of each."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2205_14503_gb300.workloads as wl
    from paper_2205_14503_gb300 import autotune
    from paper_2205_14503_gb300 import steiner as st
    torch.cuda.set_device(local)
    if rank != 0:
        return
    cfgs = [1, 2, 4] + ([3] if args.with_large else [])
    rows = []
    for cfg in cfgs:
        g = wl.config_graph(cfg)
        seeds = wl.config_seed_sets(cfg, g)[0]
        with st.SteinerGraph(g, device=local) as G:
            tuned = autotune.tune(G, g, [seeds], cache_path=None, device=local)
            d, lr_t = tuned["delta"], tuned["local_rounds"]
            # (name, delta, local rounds, heavy-pass form, unbounded tail)
            variants = [("frontier (Bellman-Ford)", 0x7FFFFFFF, 0, 1, 1),
                        ("near/far, heavy arcs pushed", d, 0, 0, 0),
                        ("near/far, heavy arcs pushed or pulled", d, 0, 1, 0),
                        ("near/far, pulled, then unbounded tail", d, 0, 1, 1),
                        ("near/far + block-local rounds", d, lr_t, 1, tuned.get("tail", 1))]
            ref = None
            for name, delta, lr, pull, tail in variants:
                if name.endswith("rounds") and lr == 0:
                    continue
                G.set_param("delta", delta)
                G.set_param("local_rounds", lr)
                G.set_param("pull", pull)
                G.set_param("tail", tail)
                G.query_detail(seeds, pairs=False)
                ms, att, its = [], [], []
                for _ in range(max(1, args.steps)):
                    r = G.query_detail(seeds, pairs=False)
                    ms.append(r.stats["ms_voronoi"])
                    att.append(r.stats["relax_attempts"])
                    its.append(r.stats["iterations"])
                if ref is None:
                    ref = r.total
                assert r.total == ref, "schedules must reach the same tree"
                rows.append({"workload": g.name, "order": name, "delta": delta, "local_rounds": lr,
                             "pull": pull, "tail": tail,
                             "ms_voronoi": statistics.median(ms),
                             "relaxations_per_arc": statistics.mean(att) / g.n_arcs,
                             "iterations": statistics.mean(its), "total": int(r.total)})
        del g
    print(json.dumps({"metric": "Voronoi relaxation-order ablation", "unit": "ms",
                      "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
                      "rows": rows}), flush=True)


def run_weights_mode(args, world, rank, local):
    """Sensitivity to the weight range (the paper's weight-range study):
    R-MAT scale 22 with weights uniform in [1, w_max] for w_max from 100 to
    100,000, one query of 64 seeds from the largest component; the Voronoi
    phase at the autotuned band width and as a plain frontier, with
    relaxations per arc."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2205_14503_gb300.workloads as wl
    from paper_2205_14503_gb300 import autotune
    from paper_2205_14503_gb300 import steiner as st
    torch.cuda.set_device(local)
    if rank != 0:
        return
    rows = []
    for wmax in (100, 1000, 10_000, 100_000):
        g = wl.rmat(22, 16, (0.57, 0.19, 0.19), wmax, wl.CONFIG_SEED + 4, True)
        seeds = wl.sample_distinct(wl.largest_cc(g), 64, wl.CONFIG_SEED + 4 + wmax)
        with st.SteinerGraph(g, device=local) as G:
            tuned = autotune.tune(G, g, [seeds], cache_path=None, device=local)
            row = {"w_max": wmax, "delta": tuned["delta"]}
            ref = None
            for name, delta in (("tuned", tuned["delta"]), ("frontier", 0x7FFFFFFF)):
                G.set_param("delta", delta)
                G.query_detail(seeds, pairs=False)
                ms, att = [], []
                for _ in range(max(1, args.steps)):
                    r = G.query_detail(seeds, pairs=False)
                    ms.append(r.stats["ms_voronoi"])
                    att.append(r.stats["relax_attempts"] / g.n_arcs)
                ref = r.total if ref is None else ref
                assert r.total == ref, "schedules must reach the same tree"
                row[f"{name}_ms"] = statistics.median(ms)
                row[f"{name}_relaxations_per_arc"] = statistics.mean(att)
            row["total"] = int(ref)
            rows.append(row)
        del g
    print(json.dumps({"metric": "Voronoi time vs weight range (R-MAT 22, k = 64)", "unit": "ms",
                      "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
                      "rows": rows}), flush=True)


def run_seeds_mode(args, world, rank, local):
    """Seed-selection strategies (the paper's seed-selection study): R-MAT
    scale 20, k = 100 seeds chosen uniformly, by BFS levels, eccentric and
    proximate (k-BFS); per strategy the device time, D and |E_S|, each tree
    checked against the oracle."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import paper_2205_14503_gb300.workloads as wl
    from paper_2205_14503_gb300 import autotune
    from paper_2205_14503_gb300 import steiner as st
    torch.cuda.set_device(local)
    if rank != 0:
        return
    g = wl.rmat(20, 16, (0.57, 0.19, 0.19), 1000, wl.CONFIG_SEED + 6, True)
    pool = wl.largest_cc(g)
    k, sd = 100, wl.CONFIG_SEED + 6
    sets = {"uniform": wl.sample_distinct(pool, k, sd),
            "bfs_level": wl.seeds_bfs_level(g, pool, k, sd),
            "eccentric": wl.seeds_eccentric(g, pool, k, sd),
            "proximate": wl.seeds_proximate(g, pool, k, sd)}
    rows = []
    with st.SteinerGraph(g, device=local) as G:
        autotune.tune(G, g, [sets["uniform"]], cache_path=None, device=local)
        for name, seeds in sets.items():
            G.query_detail(seeds, pairs=False)
            ms = []
            for _ in range(max(1, args.steps)):
                r = G.query_detail(seeds, pairs=False)
                ms.append(sum(r.stats[x] for x in ("ms_init", "ms_voronoi", "ms_bridges",
                                                   "ms_mst", "ms_tree")))
            ref = oracle.steiner(g, seeds, want_labels=False)
            rows.append({"strategy": name, "ms": statistics.median(ms),
                         "ms_voronoi": r.stats["ms_voronoi"], "total_D": int(r.total),
                         "tree_edges": int(r.edges.shape[0]),
                         "matches_oracle": bool(ref.total == r.total
                                                and np.array_equal(ref.edges, r.edges))})
    print(json.dumps({"metric": "seed-selection strategies (R-MAT 20, k = 100)", "unit": "ms",
                      "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
                      "rows": rows}), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's default band width and grid size")
    ap.add_argument("--tuned", default=None,
                    help="DELTA,BLOCKS,LOCAL_ROUNDS[,LABEL_BITS,FAR_SCAN,TAIL] instead of "
                         "autotuning (BLOCKS 0 = all; LABEL_BITS 0/32/64; FAR_SCAN -1/0/1; "
                         "TAIL 0/1)")
    ap.add_argument("--side", type=int, default=None,
                    help="profiling only: a side x side grid instead of the workload")
    ap.add_argument("--k", type=int, default=None,
                    help="profiling only: seeds for --side / --scale")
    ap.add_argument("--scale", type=int, default=None,
                    help="profiling only: an R-MAT graph of this scale with the R-MAT 26 "
                         "workload's recipe and seed density")
    ap.add_argument("--workload", type=int, default=WORKLOAD, choices=[1, 2, 3],
                    help="plain mode: single-query workload (3 = R-MAT 26 with 10,000 seeds, "
                         "the default; 2 = the 4096^2 grid; 1 = R-MAT 16)")
    ap.add_argument("--batch-scale", type=int, default=None,
                    help="batch mode, profiling only: R-MAT scale instead of 22")
    ap.add_argument("--with-large", action="store_true",
                    help="ablation mode: include the R-MAT scale-26 workload")
    ap.add_argument("--mode", choices=["plain", "batch", "serve", "ablation", "weights", "seeds"],
                    default="plain",
                    help="plain: the single-query workload (default); batch: R-MAT 22 with "
                         "64 batched queries; serve: R-MAT 24 query stream; ablation: "
                         "relaxation order on the single-query workloads; weights: "
                         "sensitivity to the weight range; seeds: seed-selection strategies")
    ap.add_argument("--queries", type=int, default=2000, help="serve mode: stream length")
    ap.add_argument("--plain-sample", type=int, default=200,
                    help="serve mode: queries timed one at a time for the plain comparison")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    try:
        if args.impl == "reference":
            run_reference(args, world, rank)
        elif args.mode == "batch":
            run_batch_mode(args, world, rank, local)
        elif args.mode == "serve":
            run_serve_mode(args, world, rank, local)
        elif args.mode == "ablation":
            run_ablation_mode(args, world, rank, local)
        elif args.mode == "weights":
            run_weights_mode(args, world, rank, local)
        elif args.mode == "seeds":
            run_seeds_mode(args, world, rank, local)
        else:
            run_ours(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
