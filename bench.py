"""Benchmark: k-motif counting with pattern morphing on a scale-20 R-MAT graph.

One step = plan (morph selection + plan compilation) + matching on the GPU +
morph transform for the motif query set, on the scale-20 R-MAT graph (edge
factor 16, a=.57 b=c=.19, seed 2, ~15.7M undirected edges) resident in HBM.
`value` = matches/s = (sum of the requested vertex-induced motif counts) /
device time per step.  The same query set is also run without morphing
(matched as given) under a deadline, for the morphed-vs-direct comparison.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--direct-deadline S] [--workload mc|mc5|fsm|batch|serve|pattern]

N > 1 (torchrun) runs independent replicas, one graph per GPU; the line
reports the whole-job rate (sum over ranks / max time over ranks).
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from pm_inputs import cached_rmat, rmat_edges, uniform_ints  # noqa: E402

SCALE, EDGE_FACTOR, SEED = 20, 16, 2
FALLBACK_HBM_GBS = 6400.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--direct-deadline", type=float, default=30.0)
    ap.add_argument("--no-baseline", action="store_true", help="skip the CPU oracle baseline leg")
    ap.add_argument("--workload", choices=["mc", "mc5", "fsm", "batch", "serve", "pattern", "motifs"],
                    default="mc",
                    help="mc: the timed 4-motif counting line (default); mc5: 5-motif counting "
                         "on the scale-20 graph, morphed vs direct; fsm / batch / serve: one "
                         "measurement line of the other workloads; pattern / motifs: one pattern "
                         "or one k-motif count (profiling targets)")
    ap.add_argument("--motif-k", type=int, default=5, help="motif size of the motifs workload")
    ap.add_argument("--motif-mode", choices=["naive", "direct", "cost"], default="naive",
                    help="morph selection of the motifs workload")
    ap.add_argument("--motif-deadline", type=float, default=0.0, help="deadline of each motifs count (0: none)")
    ap.add_argument("--mc5-direct-deadline", type=float, default=60.0,
                    help="deadline of the whole-graph direct 5-motif count")
    ap.add_argument("--no-mc5", action="store_true", help="leave the 5-motif measurements out of the mc line")
    ap.add_argument("--serve-seconds", type=float, default=5.0)
    ap.add_argument("--batch-scale", type=int, default=SCALE)
    ap.add_argument("--batch-pattern-deadline", type=float, default=30.0)
    ap.add_argument("--batch-total-deadline", type=float, default=240.0)
    ap.add_argument("--serve-kmax", type=int, default=6, help="largest pattern size in serving requests")
    ap.add_argument("--pattern", default="4:63:0",
                    help="pattern workload: k:edge_mask:induced (induced 1 = vertex-induced)")
    ap.add_argument("--scale", type=int, default=18, help="R-MAT scale of the pattern workload")
    ap.add_argument("--seed", type=int, default=7, help="R-MAT seed of the pattern workload")
    ap.add_argument("--family", choices=["auto", "rooted", "free"], default="auto")
    ap.add_argument("--labels", type=int, default=0, help="pattern workload: Zipf(1.2) vertex labels")
    ap.add_argument("--pattern-labels", default="", help="pattern workload: comma-separated vertex labels")
    ap.add_argument("--op", choices=["count", "support"], default="count")
    return ap.parse_args()


def connected_classes(k):
    """Connected k-vertex graph classes as canonical edge masks (via the
    library: one vertex-induced query per class is what motif counting asks)."""
    # canonical masks of connected graphs are produced by brute force here so the
    # bench does not depend on the oracle for its own arm
    import itertools
    pairs = [(a, b) for a in range(k) for b in range(a + 1, k)]
    idx = {p: i for i, p in enumerate(pairs)}
    perms = list(itertools.permutations(range(k)))
    seen = set()
    out = []
    for mask in range(1 << len(pairs)):
        best = min(sum(1 << idx[(min(p[a], p[b]), max(p[a], p[b]))]
                       for i, (a, b) in enumerate(pairs) if mask >> i & 1) for p in perms)
        if best in seen:
            continue
        seen.add(best)
        adj = {v: set() for v in range(k)}
        for i, (a, b) in enumerate(pairs):
            if best >> i & 1:
                adj[a].add(b)
                adj[b].add(a)
        comp, stack = {0}, [0]
        while stack:
            v = stack.pop()
            for w in adj[v] - comp:
                comp.add(w)
                stack.append(w)
        if len(comp) == k:
            out.append(best)
    return sorted(out, key=lambda m: (bin(m).count("1"), m))


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for key in ("hbm_gbs", "hbm_GBps", "hbm"):
                if key in d:
                    return float(d[key]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, mx, reasons = [], [], set()
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
                for i, nm in enumerate(names):
                    if r[3 + i].lower().startswith("active"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                pass
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return world, rank, local


def allreduce_max(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def traffic_record(kernel):
    """DRAM bytes per launch of `kernel` on this workload from the committed
    ncu summary (profiles/traffic.json), valid only while the kernel's source
    files are unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(kernel)
    if not rec:
        return None
    for src, sha in rec["sources"].items():
        f = os.path.join(ROOT, "paper_2012_04553_b300", "csrc", src)
        if not os.path.exists(f) or hashlib.sha256(open(f, "rb").read()).hexdigest() != sha:
            return None
    return rec


def cpu_oracle_sample(n, src, dst, ks, budget_s=12.0, seed=11, per_root_s=0.25, sample=4096,
                      all_core=True):
    """The oracle as it stands (direct vertex-induced counting) on a bounded
    sample of the same workload: roots drawn uniformly over all n vertices
    (every degree; a root's occurrences are those whose highest-ranked vertex
    it is), each counted single-threaded under a per-root wall-clock budget
    until budget_s is spent; roots whose budget runs out are recorded (with
    their degree) and left out.  The completed roots are then counted again
    in one call on all host cores.  Returns the all-core matches/s, the
    single-thread matches/s, the roots and the per-root occurrence sums."""
    import oracle
    # host cores this process may use (the oracle's single-thread calls pin
    # OpenMP to one thread, so the all-core pass asks for them explicitly)
    ncores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    og = oracle.prepare_graph(n, src, dst)
    order = uniform_ints(seed, 9, sample, 0, n)
    _, first = np.unique(order, return_index=True)
    order = order[np.sort(first)]
    done, timed_out, matches, t_single, t0 = [], [], 0, 0.0, time.time()
    for r in order:
        if time.time() - t0 > budget_s:
            break
        oracle.set_budget(per_root_s)
        t1 = time.time()
        try:
            c = sum(sum(oracle.motif_counts_direct(og, k, roots=np.array([r], np.int32), threads=1))
                    for k in ks)
        except oracle.OracleTimeout:
            timed_out.append(int(og.degree[r]))
            continue
        finally:
            oracle.set_budget(0)
        t_single += time.time() - t1
        done.append(int(r))
        matches += c
    roots = np.array(sorted(done), dtype=np.int32)
    out = {"unit": "matches/s", "kind": "oracle", "roots": roots, "matches": matches,
           "single_thread": {"value": matches / t_single if t_single > 0 else 0.0, "cores": 1,
                             "seconds": round(t_single, 3)}}
    value, cores = out["single_thread"]["value"], 1
    if all_core and len(roots):
        t1 = time.time()
        c_all = sum(sum(oracle.motif_counts_direct(og, k, roots=roots, threads=ncores)) for k in ks)
        t_all = time.time() - t1
        assert c_all == matches
        value, cores = matches / t_all, ncores
        out["all_core"] = {"value": value, "cores": cores, "seconds": round(t_all, 3)}
    deg_done = og.degree[roots] if len(roots) else np.zeros(1, np.int64)
    out.update({"value": value, "cores": cores,
                "sample": f"{len(order[:len(done) + len(timed_out)])} roots drawn uniformly over all "
                          f"{n} vertices of the same graph (occurrences whose highest-ranked vertex is a "
                          f"sampled root), {'+'.join(str(k) for k in ks)}-motifs direct; "
                          f"{len(done)} completed (max degree {int(deg_done.max())}), "
                          f"{len(timed_out)} exceeded the {per_root_s:g} s per-root budget "
                          f"(degrees {sorted(timed_out)[-8:]}); single-thread pass "
                          f"{t_single:.1f} s, then the completed roots on all cores",
                "roots_timed_out_degrees": sorted(timed_out)})
    return out


def run_reference(args, world, rank):
    """Reference arm: the CPU oracle on the same workload, bounded samples
    (a fresh uniform root sample per step, all host cores)."""
    if rank != 0:
        return
    n = 1 << SCALE
    src, dst = cached_rmat(SCALE, EDGE_FACTOR, SEED)
    ks = [4]
    budget = max(3.0, 90.0 / max(1, args.steps + args.warmup))
    steps = []
    for i in range(args.warmup + args.steps):
        r = cpu_oracle_sample(n, src, dst, ks, budget_s=budget, seed=11 + i, per_root_s=0.5)
        if i >= args.warmup:
            steps.append(r)
    value = float(np.mean([r["value"] for r in steps]))
    line = {
        "impl": "reference", "metric": metric_name(args), "value": value, "unit": "matches/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": budget * 1000.0, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": workload_config(args),
        "cpu_baseline": {"value": value, "unit": "matches/s", "cores": steps[0]["cores"],
                         "kind": "oracle", "sample": steps[0]["sample"]},
        "e2e": {"value": value, "unit": "matches/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def metric_name(args):
    return "4-motif counting matches/s (morphed), R-MAT scale 20"


def workload_config(args):
    return {"workload": "4-motif counting: all connected "
                        f"vertex-induced unlabeled patterns, naive morph to edge-induced patterns, "
                        f"on R-MAT scale {SCALE} (2^{SCALE} vertices), edge factor {EDGE_FACTOR}, "
                        f"a=0.57 b=c=0.19 d=0.05, seed {SEED}, degree-ordered int32 CSR, 128-bit counts",
            "l2": "CSR (~134 MB) exceeds the 126 MB L2 and a 512 MB buffer is written between steps",
            "parallelism": "replicas" if args.gpus > 1 else "single GPU"}


def run_fsm(args):
    """3-edge FSM with MNI support, threshold 20,000, on R-MAT scale 18 (ef 16,
    seed 3) with 16 vertex labels drawn Zipf(1.2) (seed 4): wall time of the
    whole level-wise mining, morphed (edge-induced candidates from
    vertex-induced superpatterns) and direct."""
    import torch
    import paper_2012_04553_b300 as pm
    from pm_inputs import zipf_labels
    n = 1 << 18
    src, dst = cached_rmat(18, 16, 3)
    labels = zipf_labels(n, 16, s=1.2, seed=4)
    g = pm.Graph(n, src, dst, labels)
    out = {}
    for name, mode in (("morphed", pm.MORPH_NAIVE), ("direct", pm.MORPH_NONE)):
        pm.fsm(g, 3, 20000, mode=mode)                      # warm-up (autotuning cached)
        torch.cuda.synchronize()
        t0 = time.time()
        pats, sup, freq = pm.fsm(g, 3, 20000, mode=mode)
        torch.cuda.synchronize()
        out[name] = {"wall_s": time.time() - t0, "candidates": len(pats),
                     "frequent": int(sum(freq)),
                     "frequent_3edge": int(sum(f for (k, m, l), f in zip(pats, freq) if bin(m).count("1") == 3))}
    line = {"metric": "3-edge FSM wall time (morphed), R-MAT scale 18, 16 Zipf labels, MNI >= 20000",
            "value": out["morphed"]["wall_s"], "unit": "s", "higher_is_better": False,
            "n_gpus": 1, "dtype": "int64", "data": "synthetic", "morphed": out["morphed"],
            "direct": out["direct"],
            "config": {"workload": "3-edge frequent subgraph mining, MNI support, threshold 20000, "
                                   "R-MAT scale 18 ef 16 seed 3, 16 labels Zipf(1.2) seed 4"}}
    print(json.dumps(line), flush=True)


def run_batch(args):
    """512 random connected 3-6 vertex patterns (half vertex-, half
    edge-induced; seed 5) counted with one plan on the scale-20 graph, the
    alternative set chosen by the cost-based optimizer, the set-operation
    plans in one persistent launch per pattern size (the decomposable
    edge-induced patterns by the decomposition kernels after them), replayed
    from a captured CUDA graph with a deadline per pattern counted from its
    launch's start: per-query status."""
    import torch
    import paper_2012_04553_b300 as pm
    from pm_inputs import random_patterns
    scale = args.batch_scale
    n = 1 << scale
    src, dst = cached_rmat(scale, EDGE_FACTOR, SEED)
    g = pm.Graph(n, src, dst)
    pats = random_patterns(512, seed=5)
    qs = [pm.make_pattern(k, m, ind) for k, m, ind in pats]
    t0 = time.time()
    plan = pm.Plan(g, qs, mode=pm.MORPH_COST)   # cost-based selection (Section 4.1), shared patterns once
    t_plan = time.time() - t0
    plan.set_launch(pm.LAUNCH_SINGLE)     # one persistent launch per pattern size for the set-operation plans
    t0 = time.time()
    fam = plan.autotune()
    plan.capture_each(timeout_per_pattern_s=args.batch_pattern_deadline,
                      timeout_total_s=args.batch_total_deadline)
    t_tune = time.time() - t0
    torch.cuda.synchronize()
    t0 = time.time()
    counts, status = plan.count_each()
    torch.cuda.synchronize()
    wall = time.time() - t0
    ok = [i for i, st in enumerate(status) if st == pm.PM_OK]
    by_k = {}
    for (k, m, ind), st in zip(pats, status):
        e = by_k.setdefault(str(k), {"queries": 0, "ok": 0})
        e["queries"] += 1
        e["ok"] += int(st == pm.PM_OK)
    line = {"metric": f"batched 512-pattern counting wall time, R-MAT scale {scale}", "value": wall,
            "unit": "s", "higher_is_better": False, "n_gpus": 1, "dtype": "int64",
            "data": "synthetic", "n_matched": plan.n_matched,
            "matched_families": {name: int(sum(f == code for f in fam)) for name, code in
                                 (("rooted", pm.PLANS_ROOTED), ("free", pm.PLANS_FREE),
                                  ("decomposition", pm.PLANS_DECOMP))},
            "queries_ok": len(ok), "queries_deadline": len(qs) - len(ok), "by_size": by_k,
            "patterns_per_s_completed": len(ok) / wall if wall > 0 else None,
            "plan_s": t_plan, "autotune_and_capture_s": t_tune, "launches": plan.last_launches(),
            "config": {"workload": "512 random connected patterns of 3-6 vertices (uniform over sizes, "
                                   "alternating vertex-/edge-induced, seed 5), cost-based morph selection "
                                   "(30 s of sampling, estimates beyond), one plan, one persistent launch "
                                   "per pattern size, captured CUDA graph with a deadline of "
                                   f"{args.batch_pattern_deadline:g} s per pattern from its launch's start "
                                   f"({args.batch_total_deadline:g} s in all), R-MAT scale {scale} ef 16 "
                                   "seed 2"}}
    print(json.dumps(line), flush=True)


def run_serve(args):
    """Poisson stream (200 req/s) of requests of 1-64 random 3-6 vertex
    patterns against R-MAT graphs of scale 16, 20 and 22 (ef 16; the scale-22
    graph carries 8 labels Zipf(1.2) and its queries label each vertex with
    probability 1/2), through the serving loop."""
    import paper_2012_04553_b300 as pm
    from pm_inputs import poisson_arrivals, random_patterns, uniform_ints, zipf_labels, uniform01
    specs = [(16, 16, 61, None), (20, 16, 2, None), (22, 16, 62, 8)]
    graphs = []
    for sc, ef, sd, nl in specs:
        src, dst = cached_rmat(sc, ef, sd)
        lab = zipf_labels(1 << sc, nl, s=1.2, seed=63) if nl else None
        graphs.append(pm.Graph(1 << sc, src, dst, lab))
    arrivals = poisson_arrivals(200.0, args.serve_seconds, seed=6)
    nreq = len(arrivals)
    sizes = uniform_ints(6, 40, nreq, 1, 65)
    which = uniform_ints(6, 41, nreq, 0, 3)
    pool = random_patterns(int(sizes.sum()), kmax=args.serve_kmax, seed=64)
    nv = sum(k for k, _, _ in pool)
    label_draw = zipf_labels(nv, 8, s=1.2, seed=66)            # one label per query vertex
    coin = uniform01(65, 0, np.arange(nv, dtype=np.uint64))    # labeled with probability 1/2
    srv = pm.Server(graphs, workers_per_graph=2, max_batch_patterns=256,
                    hbm_budget_bytes=100 << 30, batch_timeout_s=0.5, batch_total_s=2.0,
                    family=pm.PLANS_QUICK, request_timeout_s=2.0)
    ids, at, vat, t0 = [], 0, 0, time.time()
    for i in range(nreq):
        wait = arrivals[i] - (time.time() - t0)
        if wait > 0:
            time.sleep(wait)
        qs = []
        for k, m, ind in pool[at:at + sizes[i]]:
            labels = None
            if which[i] == 2:
                labels = [int(label_draw[vat + v]) if coin[vat + v] < 0.5 else -1 for v in range(k)]
            vat += k
            qs.append(pm.make_pattern(k, m, ind, labels))
        at += int(sizes[i])
        ids.append((srv.submit(int(which[i]), qs), len(qs)))
    lats, ok_pat, ok_q, statuses = [], 0, 0, {}
    for rid, nq in ids:
        done, counts, lat, st, qst = srv.wait(rid, per_query=True)
        lats.append(lat)
        statuses[st] = statuses.get(st, 0) + 1
        if st == pm.PM_OK:
            ok_pat += nq
        ok_q += sum(x == pm.PM_OK for x in qst)
    wall = time.time() - t0
    stats = srv.stats()
    srv.close()
    line = {"metric": "serving p50/p99 request latency and patterns/s (Poisson 200 req/s)",
            "value": float(np.percentile(lats, 50)), "unit": "s", "higher_is_better": False,
            "p50_s": float(np.percentile(lats, 50)), "p99_s": float(np.percentile(lats, 99)),
            "patterns_per_s_completed": ok_pat / wall,
            "query_patterns_per_s_ok": ok_q / wall, "query_patterns_ok": int(ok_q),
            "query_patterns": int(sizes.sum()), "requests": nreq,
            "status_counts": {str(k): v for k, v in statuses.items()}, "server": stats,
            "n_gpus": 1, "data": "synthetic",
            "config": {"workload": f"Poisson 200 req/s for {args.serve_seconds:.0f} s, 1-64 random "
                                   f"3-{args.serve_kmax} vertex "
                                   "patterns per request, R-MAT scale 16/20/22 ef 16 (scale 22 with 8 "
                                   "Zipf(1.2) labels, half the query vertices labeled), naive morph, "
                                   "quick plan family (no autotuning), 2 workers per graph, batches of "
                                   "at most 256 patterns, 0.5 s deadline per matched pattern, 2 s per "
                                   "batch, 2 s per request from submission (requests queued longer are "
                                   "shed unrun)"}}
    print(json.dumps(line), flush=True)


def simple_degrees(n, src, dst):
    """Degree of every vertex of the simple graph of an edge list (self-loops
    and duplicate edges dropped, either direction), by caller id."""
    a = np.minimum(src, dst).astype(np.int64)
    b = np.maximum(src, dst).astype(np.int64)
    keep = a != b
    key = np.unique(a[keep] * n + b[keep])
    return np.bincount(key // n, minlength=n) + np.bincount(key % n, minlength=n)


def mc5_measurements(pm, g, n, stream=None, direct_s=60.0, reps=2):
    """5-motif counting (the 21 connected vertex-induced unlabeled patterns),
    morphed vs direct:
    * whole graph, morphed: one plan over the 21 vertex-induced patterns with
      naive morphing (Theorem 3.1 / Corollary 3.1 over the 21 edge-induced
      patterns, all counted by the decomposition kernels); one untimed run
      (list and counter allocation), then `reps` timed runs; per-pattern
      device time of the edge-induced group;
    * whole graph, direct: the 21 vertex-induced patterns matched by
      set-operation plans under `direct_s`;
    * the R-MAT scale-12 ef-8 graph: both ways to completion, counts
      compared."""
    import torch
    masks = connected_classes(5)
    vq = [pm.make_pattern(5, m, pm.VERTEX_INDUCED) for m in masks]

    def timed(plan, deadline, runs):
        out = []
        for _ in range(runs):
            torch.cuda.synchronize()
            t0 = time.time()
            try:
                c = plan.count(stream=stream, timeout_s=deadline)
                torch.cuda.synchronize()
                out.append((time.time() - t0, [str(x) for x in c]))
            except pm.PMTimeout:
                return None, time.time() - t0
        return out, None

    morphed = pm.Plan(g, vq, mode=pm.MORPH_NAIVE)
    fam = morphed.autotune(stream=stream)
    timed(morphed, 0.0, 1)                                  # allocation run
    runs, _ = timed(morphed, 0.0, reps)
    names = {0: "rooted", 1: "free", 3: "decomposition"}
    whole = {"wall_s": round(min(t for t, _ in runs), 4), "runs_s": [round(t, 4) for t, _ in runs],
             "vertex_induced_counts": runs[-1][1], "n_matched": morphed.n_matched,
             "matched_families": sorted({names.get(f, f) for f in fam}),
             "group_device_ms": round(max(morphed.pattern_ms()), 3), "launches": morphed.last_launches()}
    direct = pm.Plan(g, vq, mode=pm.MORPH_NONE)
    res, out_after = timed(direct, direct_s, 1)
    if res is None:
        whole_direct = {"timed_out_after_s": round(out_after, 3), "deadline_s": direct_s}
    else:
        whole_direct = {"wall_s": round(res[0][0], 3), "counts_equal_morphed": res[0][1] == whole["vertex_induced_counts"]}
    # a graph on which direct matching finishes too
    ss, sd = rmat_edges(12, 8, seed=SEED)
    gs = pm.Graph(1 << 12, ss, sd)
    small = {"graph": "R-MAT scale 12, ef 8, seed 2"}
    for name, mode in (("morphed", pm.MORPH_NAIVE), ("direct", pm.MORPH_NONE)):
        plan = pm.Plan(gs, vq, mode=mode)
        plan.autotune(stream=stream)
        if mode == pm.MORPH_NAIVE:
            timed(plan, 0.0, 1)                             # allocation run
        r, _ = timed(plan, 0.0, reps if mode == pm.MORPH_NAIVE else 1)   # direct: tens of seconds, once
        small[name] = {"wall_s": round(min(t for t, _ in r), 5), "counts": r[-1][1]}
    small["counts_equal"] = small["morphed"]["counts"] == small["direct"]["counts"]
    small["speedup_morphed_over_direct"] = round(small["direct"]["wall_s"] / small["morphed"]["wall_s"], 2)
    return {"whole_graph_morphed": whole, "whole_graph_direct": whole_direct, "small_graph": small}


def run_mc5(args):
    """5-motif counting on the scale-20 graph, morphed vs direct (one line)."""
    import paper_2012_04553_b300 as pm
    n = 1 << SCALE
    src, dst = cached_rmat(SCALE, EDGE_FACTOR, SEED)
    g = pm.Graph(n, src, dst)
    res = mc5_measurements(pm, g, n, direct_s=args.mc5_direct_deadline)
    line = {"metric": "5-motif counting, morphed vs direct, R-MAT scale 20",
            "unit": "s", "higher_is_better": False, "n_gpus": 1, "dtype": "int64", "data": "synthetic",
            "value": res["whole_graph_morphed"]["wall_s"], "mc5": res,
            "config": {"workload": "5-motif counting (21 connected vertex-induced unlabeled patterns), "
                                   f"R-MAT scale {SCALE} ef {EDGE_FACTOR} seed {SEED}"}}
    print(json.dumps(line), flush=True)


def run_motifs(args):
    """k-motif counting (all connected vertex-induced k-vertex patterns,
    naive morph, direct or cost-based selection) on R-MAT (scale, ef 16,
    seed): one count that allocates the plan's scratch, then one timed count
    (a deadline, if given, applies to both)."""
    import torch
    import paper_2012_04553_b300 as pm
    src, dst = cached_rmat(args.scale, 16, args.seed)
    g = pm.Graph(1 << args.scale, src, dst)
    mode = {"naive": pm.MORPH_NAIVE, "direct": pm.MORPH_NONE, "cost": pm.MORPH_COST}[args.motif_mode]
    plan = pm.Plan(g, [pm.make_pattern(args.motif_k, m, pm.VERTEX_INDUCED) for m in connected_classes(args.motif_k)],
                   mode=mode)
    plan.autotune()
    try:
        plan.count(timeout_s=args.motif_deadline)
    except pm.PMTimeout:
        pass
    torch.cuda.synchronize()
    t0 = time.time()
    try:
        counts = plan.count(timeout_s=args.motif_deadline)
        res = {"value": time.time() - t0, "counts": [str(c) for c in counts]}
    except pm.PMTimeout:
        res = {"value": None, "timed_out_after_s": round(time.time() - t0, 3), "deadline_s": args.motif_deadline}
    torch.cuda.synchronize()
    print(json.dumps({"metric": f"{args.motif_k}-motif count ({args.motif_mode}), wall time", "unit": "s",
                      **res, "launches": plan.last_launches(), "scale": args.scale, "seed": args.seed}),
          flush=True)


def run_pattern(args):
    """One pattern on R-MAT (scale, ef 16, seed), matched as given: device
    time of the matching kernels (profiling target).  With --labels L the
    graph carries L Zipf(1.2) labels (seed + 1) and the pattern's vertices
    take labels from --pattern-labels; --op support collects MNI domains."""
    import torch
    import paper_2012_04553_b300 as pm
    from pm_inputs import zipf_labels
    k, mask, ind = (int(x) for x in args.pattern.split(":"))
    src, dst = cached_rmat(args.scale, 16, args.seed)
    n = 1 << args.scale
    labels = zipf_labels(n, args.labels, s=1.2, seed=args.seed + 1) if args.labels else None
    plab = [int(x) for x in args.pattern_labels.split(",")] if args.pattern_labels else None
    g = pm.Graph(n, src, dst, labels)
    op = pm.OP_SUPPORT if args.op == "support" else pm.OP_COUNT
    plan = pm.Plan(g, [pm.make_pattern(k, mask, ind, plab)], op=op, mode=pm.MORPH_NONE)
    plan.select({"auto": pm.PLANS_AUTO, "rooted": pm.PLANS_ROOTED, "free": pm.PLANS_FREE}[args.family])
    counts = plan.support(threshold=0)[0] if op == pm.OP_SUPPORT else plan.count()
    print(json.dumps({"metric": "single-pattern count, kernel time", "value": plan.last_kernel_ms(),
                      "unit": "ms", "count": str(counts[0]), "pattern": args.pattern,
                      "scale": args.scale, "seed": args.seed, "family": args.family}), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.workload != "mc":
        if rank == 0:
            {"fsm": run_fsm, "batch": run_batch, "serve": run_serve, "mc5": run_mc5,
             "pattern": run_pattern, "motifs": run_motifs}[args.workload](args)
        return
    import torch
    import paper_2012_04553_b300 as pm

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = 1 << SCALE
    src, dst = cached_rmat(SCALE, EDGE_FACTOR, SEED)
    ks = [4]
    queries = [pm.make_pattern(k, m, pm.VERTEX_INDUCED) for k in ks for m in connected_classes(k)]
    g = pm.Graph(n, src, dst, device=local)
    info = g.info()
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def step():
        plan = pm.Plan(g, queries, mode=pm.MORPH_NAIVE)
        counts = plan.count(stream=stream)
        return plan, counts

    for _ in range(max(3, args.warmup)):
        step()
    plan0 = pm.Plan(g, queries, mode=pm.MORPH_NAIVE)
    counts_i, alg_bytes = plan0.count_instrumented(stream=stream)
    pattern_bytes = plan0.pattern_bytes()

    # timed region: K steps, each bracketed by events on the launch stream
    sampler = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    sampler.start()
    times, kernel_ms, per_pattern_ms, counts = [], [], [], None
    for _ in range(args.steps):
        flush.fill_(1)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        plan, counts = step()
        ev1.record(stream)
        torch.cuda.synchronize()
        times.append(ev0.elapsed_time(ev1))
        kernel_ms.append(plan.last_kernel_ms())
        per_pattern_ms.append(plan.pattern_ms())
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    assert counts == counts_i, "instrumented and timed runs disagree"
    ms_step = allreduce_max(float(np.mean(times)), world)
    matches = sum(counts)
    total_matches = allreduce_sum(matches, world)
    value = total_matches / (ms_step / 1000.0)

    # end to end through the public API from pinned host buffers: graph load
    # (host preparation + upload), planning with autotuning on the fresh
    # graph, the count, the result read back
    src_t = torch.from_numpy(src).pin_memory()
    dst_t = torch.from_numpy(dst).pin_memory()
    e2e_times, phases = [], []
    for _ in range(max(1, min(args.steps, 2))):
        torch.cuda.synchronize()
        t0 = time.time()
        g2 = pm.Graph(n, src_t.numpy(), dst_t.numpy(), device=local, stream=stream)
        t1 = time.time()
        p2 = pm.Plan(g2, queries, mode=pm.MORPH_NAIVE)
        p2.autotune(stream=stream)
        t2 = time.time()
        c2 = p2.count(stream=stream)
        torch.cuda.synchronize()
        t3 = time.time()
        e2e_times.append(t3 - t0)
        phases.append((t1 - t0, t2 - t1, t3 - t2))
        p2.free()
        g2.free()
        assert c2 == counts
    e2e_s = allreduce_max(float(np.mean(e2e_times)), world)
    ph = np.mean(np.array(phases), axis=0)
    h2d = 8 * (n + 1) * 2 + 4 * 2 * info["m"] + 96 * plan0.n_plans
    d2h = 16 * plan0.n_matched + 24

    # direct (no morphing) under a deadline
    direct = {}
    dplan = pm.Plan(g, queries, mode=pm.MORPH_NONE)
    torch.cuda.synchronize()
    t0 = time.time()
    try:
        dc = dplan.count(stream=stream, timeout_s=args.direct_deadline)
        direct = {"wall_s": time.time() - t0, "counts_equal_morphed": dc == counts}
    except pm.PMTimeout:
        direct = {"timed_out_after_s": round(time.time() - t0, 3), "deadline_s": args.direct_deadline}

    peak, peak_kind = read_peaks()
    roof = dominant_roofline(pm, plan0, per_pattern_ms, pattern_bytes, peak, peak_kind, stream)
    roof["whole_step"] = {"algorithmic_bytes": int(alg_bytes),
                          "launch_sequence_ms": round(float(np.mean(kernel_ms)), 3)}
    line = {
        "metric": metric_name(args), "value": value, "unit": "matches/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic", "config": workload_config(args),
        "counts": [str(c) for c in counts],
        "morphed_wall_s": ms_step / 1000.0,
        "direct": direct,
        "roofline": roof,
        "e2e": {"value": total_matches / e2e_s, "unit": "matches/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "wall_s": e2e_s,
                "phases_s": {"load_and_upload": round(float(ph[0]), 3),
                             "plan_and_autotune": round(float(ph[1]), 3),
                             "count_and_readback": round(float(ph[2]), 3)}},
        "gpu_launches": args.steps * plan.last_launches(),
        "clocks": clocks,
        "graph": {"n": info["n"], "m": info["m"], "max_degree": info["max_degree"]},
    }
    if rank == 0 and not args.no_mc5:
        line["mc5"] = mc5_measurements(pm, g, n, stream=stream, direct_s=args.mc5_direct_deadline)
    if rank == 0 and world == 1 and not args.no_baseline:
        base = cpu_oracle_sample(n, src, dst, ks)
        roots = base.pop("roots")
        sample_matches = base.pop("matches")
        if len(roots):
            # the library's exact count on the same roots; the whole-graph
            # oracle time is extrapolated by the sample's share of occurrences
            gpu_sample = sum(pm.Plan(g, queries, mode=pm.MORPH_NAIVE).count_roots(roots, stream=stream))
            base["sample_counts_equal_library"] = gpu_sample == sample_matches
            if sample_matches > 0 and "all_core" in base:
                share = sample_matches / float(matches)
                base["extrapolation"] = {
                    "kind": "extrapolation (not measured): all-core oracle time on the sample "
                            "divided by the sample's share of all occurrences",
                    "sample_share_of_occurrences": share,
                    "whole_graph_seconds": base["all_core"]["seconds"] / share}
        line["cpu_baseline"] = base
    if rank == 0:
        print(json.dumps(line), flush=True)


def kernel_of(family, kind, pm):
    if family == pm.PLANS_DECOMP:
        return "decomposition: tri_kernel, mirror_kernel, local_warp_kernel, local_block_kernel, ve_kernel"
    return {0: "match_kernel", 1: "wedge_heavy_kernel+wedge_pairs_kernel", 2: "clique_kernel"}[kind]


def dominant_roofline(pm, plan, per_pattern_ms, pattern_bytes, peak, peak_kind, stream):
    """Roofline of the matched pattern whose launches take the most device
    time in a step (per-pattern CUDA events on the launch stream; the
    decomposed patterns' passes are timed as one group): its kernels, its
    algorithmic bytes (instrumented run of the same plan) over its own
    average time."""
    fam = plan.autotune(stream=stream)
    rooted = plan.export_plans(pm.PLANS_ROOTED)
    mats = plan.matched_patterns()
    ms = np.mean(np.array(per_pattern_ms), axis=0)
    j = int(np.argmax(ms))
    kind = 0
    if fam[j] == pm.PLANS_ROOTED:
        kinds = [int(r["kind"]) for r in rooted if int(r["counter"]) == j]
        kind = kinds[0] if len(kinds) == 1 else 0
    k, mask, induced, labels = mats[j]
    b = int(pattern_bytes[j])
    achieved = b / (ms[j] / 1000.0) / 1e9 if ms[j] > 0 and b > 0 else None
    name = kernel_of(fam[j], kind, pm)
    trec = traffic_record(name.split(":")[0])
    share = float(ms[j] / ms.sum()) if ms.sum() > 0 else None
    fam_name = {pm.PLANS_ROOTED: "rooted", pm.PLANS_FREE: "free", pm.PLANS_DECOMP: "decomposition"}[fam[j]]
    return {"bound": "hbm", "achieved": round(achieved, 2) if achieved else None, "peak": peak,
            "unit": "GB/s", "frac": round(achieved / peak, 5) if achieved else None,
            "peak_source": peak_kind,
            "traffic": trec["dram_bytes_per_launch"] if trec else None,
            "traffic_frac": (round(trec["dram_bytes_per_launch"] / (ms[j] / 1000.0) / 1e9 / peak, 5)
                             if trec else None),
            "kernel": name,
            "pattern": {"k": k, "edge_mask": mask, "induced": induced, "family": fam_name,
                        "decomposed_patterns_in_group": int(sum(f == pm.PLANS_DECOMP for f in fam))
                        if fam[j] == pm.PLANS_DECOMP else None},
            "kernel_ms": round(float(ms[j]), 3), "share_of_step_device_time": share,
            "algorithmic_bytes_per_launch": b,
            "per_pattern_ms": [round(float(x), 3) for x in ms],
            "per_pattern_algorithmic_bytes": [int(x) for x in pattern_bytes]}


if __name__ == "__main__":
    main()
