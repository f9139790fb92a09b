"""Benchmark: warm-start APSP updates/s at n = 8192 (directed complete graph,
int32 weights uniform in [1, 1e6]), mixed updates (25 % node add, 25 % node
removal, 25 % edge decrease w -> floor(w/2), 25 % edge increase w -> 4w,
uniform random targets), one library call per update.

A step is a batch of --updates mixed updates.  `value` is updates per second
with every input already in device memory (CUDA events on the library's
stream); `e2e` is the same metric through the C ABI with host buffers (the new
nodes' weight vectors copied host -> device inside the timed region, and a
device -> host read of query results at the end of every step).  Also
reported: the GPU cold blocked Floyd-Warshall on the final graph, the
dominant kernel's roofline, and the CPU oracle's throughput on a bounded
sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
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
sys.path.insert(0, ROOT)

import synth  # noqa: E402

N = 8192
CAP = 8192 + 256
W_LO, W_HI = 1, 10**6
SEED = 2
METRIC = "warm-start APSP updates/s at n=8192 vs GPU cold FW; sweep HBM GB/s vs peak"
UNIT = "updates/s"
WORKLOAD = "n=8192 directed complete graph, int32 weights U[1,1e6], mixed updates 25% add / 25% remove / 25% decrease (w/2) / 25% increase (4w), uniform targets, one call per update"
# kernels that read the whole of D once per launch on this workload (the
# insertion's reduction reads only its candidate rows here, see k_insert_reduce)
SWEEP_KERNELS = ("insert_relax", "detect_remove")
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of each
# sweep at this workload, from an ncu capture of the same kernels taken in a
# separate run (mean of two launches); a sweep whose code changes must be
# captured again before its figure is used
SWEEP_TRAFFIC = {"insert_relax": 275.10e6, "detect_remove": 274.96e6}
TRAFFIC_SOURCE = "ncu capture of the same kernel on this workload, separate run (not this run)"


def rank_seed(rank: int) -> int:
    """Each replica (one process per GPU) updates its own graph."""
    return SEED + 1000 * rank


def job_ms(ms: float, dist=None, device="cuda") -> float:
    """The job's time is its slowest rank's: max over ranks."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(updates_per_rank: int, world: int, ms: float) -> float:
    """Whole-job updates/s: the updates of all ranks over the slowest rank's time."""
    return updates_per_rank * world / (ms / 1000.0)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def plan_ops(total: int, seed: int, tight: bool = False, W=None):
    """Concrete op list (slot ids and weights) from the seeded update stream,
    simulating slot assignment (lowest free slot) and the weight mirror on the
    host, so no per-update host work happens inside the timed region.  With
    `tight`, every edge update takes the lightest out-edge of its source (a
    shortest path, so increases are never trivial and decreases sweep)."""
    if W is None:
        W = synth.complete_digraph_i32(N, W_LO, W_HI, seed)
    alive = np.zeros(CAP, dtype=bool)
    alive[:N] = True
    Wm = np.full((CAP, CAP), synth.INF_I32, dtype=np.int32)
    Wm[:N, :N] = W
    ups = synth.mixed_updates(N, total, seed, capacity=CAP, w_lo=W_LO, w_hi=W_HI, cap=1 << 26, tight=tight)
    ops = []
    for up in ups:
        live = np.flatnonzero(alive)
        if up.kind == synth.ADD:
            iw = np.full(CAP, synth.INF_I32, np.int32)
            ow = np.full(CAP, synth.INF_I32, np.int32)
            iw[live] = up.in_w[:len(live)]
            ow[live] = up.out_w[:len(live)]
            dead = np.flatnonzero(~alive)
            p = int(dead[0])
            Wm[:, p] = np.where(alive, iw, synth.INF_I32)
            Wm[p, :] = np.where(alive, ow, synth.INF_I32)
            Wm[p, p] = 0
            alive[p] = True
            ops.append(("add", iw, ow))
        elif up.kind == synth.REMOVE:
            k = int(live[up.a])
            alive[k] = False
            Wm[k, :] = synth.INF_I32
            Wm[:, k] = synth.INF_I32
            ops.append(("remove", k))
        else:
            u, v = int(live[up.a]), int(live[up.b])
            if up.tight:
                row = np.where(alive, Wm[u].astype(np.int64), synth.INF_I32)
                row[u] = synth.INF_I32
                v = int(np.argmin(row))
            w0 = int(Wm[u, v])
            w = w0 // 2 if up.kind == synth.DECREASE else min(w0 * 4, up.cap)
            Wm[u, v] = w
            ops.append((up.kind, u, v, w))
    return W, ops


def step_queries(ops, U: int, steps, qpairs):
    """Per step, the pair-query batch issued after the step's updates: the
    pairs `qpairs` taken modulo the live slots as the host's own simulation of
    the lowest-free-slot rule sees them (no device read needed)."""
    alive = np.zeros(CAP, dtype=bool)
    alive[:N] = True
    out = {}
    last = max(steps) + 1
    for s in range(last):
        for op in ops[s * U:(s + 1) * U]:
            if op[0] == "add":
                alive[int(np.flatnonzero(~alive)[0])] = True
            elif op[0] == "remove":
                alive[op[1]] = False
        if s in steps:
            live = np.flatnonzero(alive)
            out[s] = live[qpairs % len(live)].astype(np.int32)
    return out


def fw_cpu_timings(sizes_all=(256, 1024, 2048, 4096), sizes_one=(256, 1024, 2048)):
    """The oracle's Floyd-Warshall (C, OpenMP over rows) on the host cores, all
    threads and one thread, in a child process per setting (the thread count
    is fixed when OpenMP starts); best of 3 below n = 2048, one run above."""
    code = r"""
import json, sys, time
sys.path.insert(0, %r)
import synth
from oracle import apsp as O
out = {}
for n in %r:
    W = synth.complete_digraph_i32(n, 1, 10**6, 2)
    best = None
    for _ in range(3 if n < 2048 else 1):
        t = time.perf_counter(); O.fw(W); dt = time.perf_counter() - t
        best = dt if best is None else min(best, dt)
    out[n] = best
print(json.dumps({"threads": O.num_threads(), "s": out}))
"""
    res = {}
    for label, sizes, env_threads in (("all_cores", sizes_all, None), ("one_thread", sizes_one, "1")):
        env = dict(os.environ)
        if env_threads:
            env["OMP_NUM_THREADS"] = env_threads
        r = subprocess.run([sys.executable, "-c", code % (ROOT, list(sizes))], capture_output=True, text=True,
                           env=env, timeout=600)
        if r.returncode != 0:
            res[label] = {"error": r.stderr.strip().splitlines()[-1] if r.stderr.strip() else "failed"}
            continue
        d = json.loads(r.stdout.strip().splitlines()[-1])
        res[label] = {"threads": d["threads"], "seconds": {str(k): round(v, 4) for k, v in d["s"].items()}}
    one = res.get("one_thread", {}).get("seconds", {})
    if "2048" in one:
        res["one_thread"]["extrapolated_n3"] = {"4096": round(one["2048"] * 8, 2), "8192": round(one["2048"] * 64, 1)}
    allc = res.get("all_cores", {}).get("seconds", {})
    if "4096" in allc:
        res["all_cores"]["extrapolated_n3"] = {"8192": round(allc["4096"] * 8, 2)}
    return res


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, dev: int):
        self.dev = dev
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"apsp_bench_clocks_{os.getpid()}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_rate(W, rows: int):
    """The oracle (dense Dijkstra per source, C + OpenMP) recomputing `rows`
    source rows of the APSP matrix of the graph; scaled to one full update
    (all N rows)."""
    from oracle import apsp as O
    src = synth.uniform_int(SEED, 31, rows, 0, N - 1)
    t0 = time.perf_counter()
    O.dijkstra_rows(W, src)
    dt = time.perf_counter() - t0
    per_update = dt * N / rows
    return 1.0 / per_update, O.num_threads(), dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    W = synth.complete_digraph_i32(N, W_LO, W_HI, SEED)
    # a bounded sample per step: about 2560 source rows over the whole timed
    # run, at least 64 a step so the oracle's per-call setup stays amortised
    rows = max(64, min(128, 2560 // max(1, args.steps)))
    for _ in range(args.warmup):
        cpu_oracle_rate(W, rows)
    rates, times, cores = [], [], 1
    for _ in range(args.steps):
        r, cores, dt = cpu_oracle_rate(W, rows)
        rates.append(r)
        times.append(dt)
    value = len(rates) / sum(1.0 / r for r in rates)
    sample = f"{rows} of {N} source rows per step (dense Dijkstra per row), scaled x{N // rows} to one full recomputation per update"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_case(case: str):
    """The workload's graph plus a few fixed updates, for profiler captures:
    "removals" removes nodes 7115 (about 5k affected pairs) and 5533 (about
    284k), "inserts" adds two nodes with the workload's weight distribution,
    "paths" answers two batches of 4096 uniform path queries (Algorithm 7)."""
    import torch
    from paper_2412_15122_gb300 import Graph, build
    build.build()
    W = synth.complete_digraph_i32(N, W_LO, W_HI, SEED)
    g = Graph(W, CAP)
    if case == "removals":
        for k in (7115, 5533):
            g.remove_node(k)
            g.sync()
            st = g.stats()
            print(json.dumps({"op": "remove", "node": k, "pairs": st["affected_pairs"], "rows": st["affected_rows"],
                              "passes": st["passes"], "warm_us": st["warm_total_us"]}))
    elif case == "paths":
        uv = np.stack([synth.uniform_int(SEED, 80, 4096, 0, N - 1), synth.uniform_int(SEED, 81, 4096, 0, N - 1)], 1)
        for _ in range(2):
            _, lens = g.query_paths(uv.astype(np.int32), stride=64)
        print(json.dumps({"op": "paths", "queries": 4096, "mean_nodes": float(np.mean(lens))}))
    else:
        for t in range(2):
            iw = synth.uniform_int(SEED, 60 + t, CAP, W_LO, W_HI).astype(np.int32)
            ow = synth.uniform_int(SEED, 70 + t, CAP, W_LO, W_HI).astype(np.int32)
            p = g.add_node(iw, ow)
            g.sync()
            print(json.dumps({"op": "add", "slot": p}))
    g.close()
    torch.cuda.synchronize()


TYPE_FEATURE = {"remove": 1.0 / 3.0, "increase": 1.0}


def _euclid_stream(n0, count, seed, fractions, capacity):
    """Update stream for an undirected Euclidean graph: rank-based node
    references from synth.mixed_updates; a new node is a new uniform point
    (its weights are drawn when it is applied)."""
    return synth.mixed_updates(n0, count, seed, fractions=fractions, tight=True, capacity=capacity, stream=90)


class _Tracked:
    """A graph plus the host mirror of its weights (and, for Euclidean
    graphs, its points) that the update streams of the dispatch study need."""

    def __init__(self, Graph, W, cap, euclid, pts=None):
        self.g = Graph(W, cap, undirected=euclid)
        n = W.shape[0]
        self.W = np.full((cap, cap), synth.INF_I32, np.int32)
        self.W[:n, :n] = W
        self.alive = np.zeros(cap, bool)
        self.alive[:n] = True
        self.euclid = euclid
        self.pts = np.zeros((cap, 2))
        if pts is not None:
            self.pts[:n] = pts

    def apply(self, up, seed, t):
        """Issues one update; returns (kind, relative weight change)."""
        g, live = self.g, np.flatnonzero(self.alive)
        if up.kind == synth.ADD:
            cap = len(self.alive)
            iw = np.full(cap, synth.INF_I32, np.int32)
            ow = iw.copy()
            if self.euclid:
                w, pnt = synth.new_point_weights_i32(self.pts[live], seed, 5000 + t)
                iw[live] = w
                ow[live] = w
            else:
                iw[live] = up.in_w[:len(live)]
                ow[live] = up.out_w[:len(live)]
            slot = g.add_node(iw, ow)
            if self.euclid:
                self.pts[slot] = pnt
            self.W[:, slot] = np.where(self.alive, iw, synth.INF_I32)
            self.W[slot, :] = np.where(self.alive, ow, synth.INF_I32)
            self.W[slot, slot] = 0
            self.alive[slot] = True
            return "add", 0.0
        if up.kind == synth.REMOVE:
            k = int(live[up.a])
            g.remove_node(k)
            self.alive[k] = False
            self.W[k, :] = synth.INF_I32
            self.W[:, k] = synth.INF_I32
            return "remove", 0.0
        u, v = int(live[up.a]), int(live[up.b])
        if up.tight:   # the lightest out-edge of u is always a shortest path
            row = np.where(self.alive, self.W[u].astype(np.int64), synth.INF_I32)
            row[u] = synth.INF_I32
            v = int(np.argmin(row))
        w0 = int(self.W[u, v])
        w = w0 // 2 if up.kind == synth.DECREASE else min(max(1, w0) * 4, 1 << 26)
        g.update_edge(u, v, w)
        self.W[u, v] = w
        if self.euclid:
            self.W[v, u] = w
        return up.kind, ((w - w0) / max(1, w0) if up.kind == synth.INCREASE else 0.0)


def run_dispatch_study(args):
    """Cost-model study (warm/cold dispatch): samples from real warm updates
    at n in {1024, ..., 8192} on directed uniform and undirected Euclidean
    graphs (features as the device computes them, labels = measured log2
    microseconds of the warm repair and of the cold Floyd-Warshall at that
    size), training on 80 %, held-out loss and decision accuracy on 20 %, then
    total device time of the update stream on an n=16384 undirected Euclidean
    graph under the delta rule, the model, always-warm and always-cold."""
    import torch
    from paper_2412_15122_gb300 import Graph, build
    from paper_2412_15122_gb300 import apsp as A
    build.build()
    t_start = time.perf_counter()
    arm_list = [a for a in args.study_arms.split(",") if a]
    sizes = (1024, 2048, 4096, 8192)
    per = max(50, args.study_samples // (2 * len(sizes))) if "model" in arm_list else 0
    X, Y = [], []
    for euclid in ((False, True) if per else ()):
        for n in sizes:
            seed = 300 + n + (1 if euclid else 0)
            if euclid:
                W, pts0 = synth.euclidean_undirected_i32(n, seed)
                cap = n + 64
                pts = np.zeros((cap, 2))
                pts[:n] = pts0
            else:
                W = synth.complete_digraph_i32(n, 1, 10**6, seed)
                cap, pts = n + 64, None
            tg = _Tracked(Graph, W, cap, euclid, pts[:n] if euclid else None)
            g = tg.g
            # cold label: the blocked FW at this size
            g.recompute()
            g.sync()
            t0 = time.perf_counter()
            g.recompute()
            g.sync()
            cold_us = (time.perf_counter() - t0) * 1e6
            g.set_dispatch("warm")
            # adds balance removals so the graph keeps its size
            mix = (0.35, 0.35, 0.0, 0.3)
            ups = _euclid_stream(n, per * 3, seed, mix, cap) if euclid else \
                synth.mixed_updates(n, per * 3, seed, fractions=mix, w_lo=1, w_hi=10**6,
                                    tight=True, capacity=cap, stream=91)
            got = 0
            for t, up in enumerate(ups):
                kind, dw = tg.apply(up, seed, t)
                if kind not in TYPE_FEATURE:
                    continue
                st = g.stats()
                if st["path"] != "warm":
                    continue
                nb = st["n_live"] + (1 if kind == "remove" else 0)
                nb = max(2, nb)
                X.append([TYPE_FEATURE[kind], np.log2(nb), dw, st["affected_pairs"] / (nb * nb),
                          st["affected_rows"] / max(1, nb - 1), st["affected_rows"] / nb])
                Y.append([np.log2(max(1.0, st["warm_total_us"])), np.log2(cold_us)])
                got += 1
                if got >= per:
                    break
            g.close()
    train_s = train_loss = held_loss = acc = None
    P = None
    tr = te = ()
    if per:
        X = np.asarray(X, np.float32)
        Y = np.asarray(Y, np.float32)
        order = np.argsort(synth.u64(7, 7, len(X)))
        cut = int(0.8 * len(X))
        tr, te = order[:cut], order[cut:]
        t_train = time.perf_counter()
        P, train_loss = A.apsp_model_train(X[tr], Y[tr], epochs=80, batch=256, lr=2e-3, seed=5)
        train_s = time.perf_counter() - t_train
        held_loss, _ = A.apsp_model_loss_grad(P, X[te], Y[te])
        pred = A.apsp_model_predict(P, X[te])
        acc = float(np.mean((pred[:, 0] <= pred[:, 1]) == (Y[te, 0] <= Y[te, 1])))

    # ---- the four arms on n = 16384 undirected Euclidean updates -------------
    n = 16384
    W, pts0 = synth.euclidean_undirected_i32(n, 3)
    cap = n + 64
    ups = _euclid_stream(n, args.study_updates, 3, (0.1, 0.4, 0.1, 0.4), cap)
    arms = {}
    finals = {}
    lists = {}
    for arm in arm_list:
        tg = _Tracked(Graph, W, cap, True, pts0)
        g = tg.g
        if arm == "delta":
            g.set_dispatch("delta", 0.5)
        elif arm == "model":
            g.set_model(P)
            g.set_dispatch("model")
        elif arm in ("warm_exact_list", "warm_direct_filter", "warm_algorithm12"):
            # Experiment IV's question: how much of Corollary 3's list is
            # Algorithm 12's (pairs whose distance really grows); what the
            # direct-edge filter keeps of it; and Algorithm 12 applied before
            # the repair
            g.set_dispatch("warm")
            g.set_exact_list(True)
            g.set_list_mode({"warm_exact_list": "corollary3", "warm_direct_filter": "direct_edge",
                             "warm_algorithm12": "algorithm12"}[arm])
        else:
            g.set_dispatch(arm)
        g.sync()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        paths = {}
        for t, up in enumerate(ups):
            kind = tg.apply(up, 3, t)[0]
            st = g.stats()
            paths[st["path"]] = paths.get(st["path"], 0) + 1
            if arm.startswith("warm_") and kind in ("remove", "increase") and st["grown_pairs"] >= 0:
                L = lists.setdefault(arm, {}).setdefault(kind, {"updates": 0, "listed_pairs": 0, "alg12_pairs": 0,
                                                                "listed_rows": 0, "alg12_rows": 0})
                L["updates"] += 1
                L["listed_pairs"] += st["affected_pairs"]
                L["alg12_pairs"] += st["grown_pairs"]
                L["listed_rows"] += st["affected_rows"]
                L["alg12_rows"] += st["grown_rows"]
        g.sync()
        arms[arm] = {"seconds": time.perf_counter() - t0, "paths": paths}
        finals[arm] = torch.from_numpy(g.D()).cuda()
        alive, Wf = tg.alive.copy(), tg.W
        g.close()
    ref_arm = arm_list[0]
    same = all(torch.equal(finals[ref_arm], finals[a]) for a in finals)
    # 64 sampled rows of the final matrix against the oracle's Dijkstra
    from oracle import apsp as O
    Dw = finals[ref_arm].cpu().numpy()
    m = Dw.shape[0]
    live = np.flatnonzero(alive[:m])
    rows = live[synth.uniform_int(3, 77, 64, 0, len(live) - 1)]
    ref = O.dijkstra_rows(Wf[:m, :m], rows, alive=alive[:m])
    ok_rows = bool(np.array_equal(O.to_i32(ref)[:, live], Dw[rows][:, live]))
    print(json.dumps({
        "study": "warm/cold dispatch", "samples": int(len(X)), "train": int(len(tr)), "held_out": int(len(te)),
        "sizes": list(sizes), "graphs": ["directed complete U[1,1e6]", "undirected Euclidean round(1e4 d)"],
        "model_train_seconds": train_s, "train_loss": train_loss, "held_out_loss": held_loss,
        "held_out_decision_accuracy": acc,
        "eval": {"workload": f"n={n} undirected Euclidean, {len(ups)} updates (10% add, 40% remove, "
                             "10% decrease, 40% increase on lightest out-edges)", "arms": arms,
                 "identical_final_D": bool(same), "sampled_rows_match_oracle": ok_rows,
                 "affected_lists": lists},
        "wall_seconds": time.perf_counter() - t_start}))


def _batch_workload(n_graphs, per, dtype, seed):
    """Graphs with n ~ U[64, 2048] and `per` ordered mixed updates each
    (25 % of each kind, uniform targets), as concrete per-graph items."""
    sizes = synth.uniform_int(seed, 3, n_graphs, 64, 2048)
    graphs, items = [], []
    for gi, n in enumerate(sizes):
        n = int(n)
        cap = n + per
        if dtype == "f32":
            W = synth.lognormal_digraph_f32(n, seed + gi)
            ups = synth.mixed_updates(n, per, seed + gi, capacity=cap, weights="lognormal", stream=11)
            inf, npdt = np.float32(np.inf), np.float32
        else:
            W = synth.complete_digraph_i32(n, 1, 1000, seed + gi)
            ups = synth.mixed_updates(n, per, seed + gi, capacity=cap, w_lo=1, w_hi=1000, stream=11)
            inf, npdt = synth.INF_I32, np.int32
        Wm = np.full((cap, cap), inf, W.dtype)
        Wm[:n, :n] = W
        alive = np.zeros(cap, bool)
        alive[:n] = True
        its = []
        for up in ups:
            live = np.flatnonzero(alive)
            if up.kind == synth.ADD:
                iw = np.full(cap, inf, npdt)
                ow = np.full(cap, inf, npdt)
                iw[live] = up.in_w[:len(live)]
                ow[live] = up.out_w[:len(live)]
                p = int(np.flatnonzero(~alive)[0])
                Wm[:, p] = np.where(alive, iw, inf)
                Wm[p, :] = np.where(alive, ow, inf)
                Wm[p, p] = 0
                alive[p] = True
                its.append((gi, "add", iw, ow))
            elif up.kind == synth.REMOVE:
                k = int(live[up.a])
                alive[k] = False
                Wm[k, :] = inf
                Wm[:, k] = inf
                its.append((gi, "remove", k))
            else:
                u, v = int(live[up.a]), int(live[up.b])
                w0 = Wm[u, v]
                if dtype == "f32":
                    w = np.float32(w0 / 2) if up.kind == synth.DECREASE else np.float32(w0 * 4)
                else:
                    w = int(w0) // 2 if up.kind == synth.DECREASE else min(int(w0) * 4, 1 << 26)
                Wm[u, v] = w
                its.append((gi, "edge", u, v, float(w)))
        graphs.append((W, cap))
        items.append(its)
    return graphs, items


def run_batch_study(args):
    """Batched execution: 512 directed complete graphs, n ~ U[64, 2048],
    16 ordered mixed updates each, applied (a) by one persistent batch
    launch, (b) by one library call per update, (c) as a cold Floyd-Warshall
    of every graph; int32 U[1, 1000] and fp32 lognormal(0, 1) weights."""
    import torch
    from paper_2412_15122_gb300 import Batch, Graph, build
    build.build()
    per = 16
    out = {"study": "batched execution", "graphs": args.study_graphs, "updates_per_graph": per,
           "workload": "directed complete graphs, n ~ U[64, 2048], mixed updates 25% each kind, uniform targets"}
    for dtype in ("i32", "f32"):
        specs, items = _batch_workload(args.study_graphs, per, dtype, 40 if dtype == "i32" else 41)
        n_upd = sum(len(x) for x in items)
        flat = [it for its in items for it in its]
        # (a) batched: one persistent launch (a replayed CUDA graph), timed for
        # each CTA width on fresh copies of the graphs; the fastest is kept
        per_width = {}
        G = None
        for width in (128, 256, 512):
            if G is not None:
                for g in G:
                    g.close()
            G = [Graph(W, cap) for W, cap in specs]
            for g in G:
                g.sync()
            b = Batch()
            b.set_width(width)
            # warm-up: capture the executor's graph on a copy of the first graph
            gw = Graph(specs[0][0], specs[0][1])
            b.run([gw], items[0])
            gw.close()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            b.run(G, flat)
            per_width[width] = time.perf_counter() - t0
            binfo = b.info()
            b.close()
        best_w = min(per_width, key=per_width.get)
        batch_s = per_width[best_w]
        # (b) one call per update
        S = [Graph(W, cap) for W, cap in specs]
        for g in S:
            g.sync()
        t0 = time.perf_counter()
        for gi, its in enumerate(items):
            g = S[gi]
            for it in its:
                if it[1] == "add":
                    g.add_node(it[2], it[3])
                elif it[1] == "remove":
                    g.remove_node(it[2])
                else:
                    g.update_edge(it[2], it[3], it[4])
        for g in S:
            g.sync()
        single_s = time.perf_counter() - t0
        # identical results, graph by graph (int32 exact, fp32 within 1e-5)
        worst = 0.0
        for g, s in zip(G, S):
            a, c = torch.from_numpy(g.D()).cuda(), torch.from_numpy(s.D()).cuda()
            if dtype == "i32":
                worst = max(worst, float((a != c).sum().item()))
            else:
                fin = torch.isfinite(c)
                rel = ((a[fin] - c[fin]).abs() / c[fin].abs().clamp_min(1e-30)).max().item() if fin.any() else 0.0
                worst = max(worst, rel)
        # (c) cold FW of every graph (the state after the updates)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for g in G:
            g.recompute()
        for g in G:
            g.sync()
        cold_s = time.perf_counter() - t0
        for g in G + S:
            g.close()
        out[dtype] = {"updates": n_upd, "batched_seconds": batch_s, "batched_updates_per_s": n_upd / batch_s,
                      "batched_seconds_per_width": per_width, "best_width": best_w,
                      "graph_replays_last_executor": binfo["graph_replays"],
                      "single_call_seconds": single_s, "single_call_updates_per_s": n_upd / single_s,
                      "cold_fw_all_graphs_seconds": cold_s,
                      ("mismatched_entries" if dtype == "i32" else "max_rel_diff"): worst}
    print(json.dumps(out))


def run_ratio_study(args):
    """Experiments I and II of the paper on the GPU: on directed complete
    graphs (int32 U[1, 1e6]) of N = 1000, 2000, 3000, 5000 nodes, the time of a
    warm-start update divided by a cold Floyd-Warshall of the updated graph,
    r = APSP_warm / APSP_cold (Eq. (equ:ratioo)); 20 random node removals
    (Experiment I) and 20 random edge modifications to a new U[1, 1e6] weight
    (Experiment II) per size, each timed alone with CUDA events."""
    import torch
    from paper_2412_15122_gb300 import Graph, build
    build.build()
    out = {"study": "warm/cold ratios (Experiments I and II)",
           "workload": "directed complete graphs, int32 U[1,1e6]; random node removal / random edge to a new U[1,1e6] weight",
           "sizes": {}}
    stream = torch.cuda.Stream()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1)

    for n in (1000, 2000, 3000, 5000):
        W = synth.complete_digraph_i32(n, W_LO, W_HI, 900 + n)
        g = Graph(W, n + 32, stream=stream)
        g.sync()
        for _ in range(3):   # warm-up of every kernel
            g.recompute()
        g.sync()
        reps = args.study_reps
        ks = synth.uniform_int(901, n, reps, 0, n - 1)
        rm, ed = [], []
        alive = np.ones(n, dtype=bool)
        for t in range(reps):
            live = np.flatnonzero(alive)
            k = int(live[ks[t] % len(live)])
            warm = timed(lambda: g.remove_node(k))
            alive[k] = False
            cold = timed(g.recompute)
            rm.append(warm / cold)
        uv = synth.uniform_int(902, n, 2 * reps, 0, n - 1)
        nw = synth.uniform_int(903, n, reps, W_LO, W_HI)
        for t in range(reps):
            live = np.flatnonzero(alive)
            u, v = int(live[uv[2 * t] % len(live)]), int(live[uv[2 * t + 1] % len(live)])
            if u == v:
                v = int(live[(uv[2 * t + 1] + 1) % len(live)])
            warm = timed(lambda: g.update_edge(u, v, int(nw[t])))
            cold = timed(g.recompute)
            ed.append(warm / cold)
        g.close()
        out["sizes"][str(n)] = {"removal_ratio_mean": float(np.mean(rm)), "removal_ratio_sd": float(np.std(rm)),
                                "edge_ratio_mean": float(np.mean(ed)), "edge_ratio_sd": float(np.std(ed)),
                                "reps": reps}
    print(json.dumps(out))


def run_path_study(args):
    """Warm-start path queries (Algorithm 7) on directed complete graphs with
    int32 weights U[1, 1e6]: uniform random pairs, answered in batches through
    apsp_query_paths and one at a time through apsp_query_path.  The CPU side
    times the oracle's Algorithm 7 and its dense Dijkstra per query (the
    paper's cold comparison) at n = 2048."""
    import torch
    from paper_2412_15122_gb300 import Graph, build
    from paper_2412_15122_gb300 import apsp as A
    build.build()
    from oracle import apsp as O
    hbm, peak_kind = peaks()
    out = {"study": "path queries", "workload": "directed complete graph, int32 U[1,1e6], uniform pairs",
           "gpu": {}}
    nq = args.study_queries
    for n in (2048, 8192):
        W = synth.complete_digraph_i32(n, W_LO, W_HI, 20 + n)
        g = Graph(W, n + 256)
        g.sync()
        uv = np.stack([synth.uniform_int(21, n, nq, 0, n - 1), synth.uniform_int(22, n, nq, 0, n - 1)], 1)
        uv = uv.astype(np.int32)
        for _ in range(3):
            g.query_paths(uv, stride=64)
        A.apsp_profile_enable(g.h, True)
        A.apsp_profile_reset(g.h)
        reps = 5
        t0 = time.perf_counter()
        for _ in range(reps):
            _, lens = g.query_paths(uv, stride=64)
        api_s = (time.perf_counter() - t0) / reps
        prof = A.apsp_profile_read(g.h)
        A.apsp_profile_enable(g.h, False)
        kl, kms = prof.get("path_query", (0, 0.0))
        kern_s = kms / 1000.0 / max(1, kl)
        span = g.info()["n_slots"]
        lat = []
        for q in range(200):
            u, v = int(uv[q, 0]), int(uv[q, 1])
            t1 = time.perf_counter()
            g.query_path(u, v, 64)
            lat.append(time.perf_counter() - t1)
        algo_bytes = 8.0 * span * nq          # row u of D and row v of D^T per query
        out["gpu"][str(n)] = {
            "queries": nq, "api_queries_per_s": nq / api_s, "kernel_us_per_batch": kern_s * 1e6,
            "kernel_queries_per_s": nq / kern_s if kern_s > 0 else None,
            "kernel_read_gbs": algo_bytes / kern_s / 1e9 if kern_s > 0 else None,
            "kernel_read_frac_of_peak": (algo_bytes / kern_s / 1e9) / hbm if kern_s > 0 else None,
            "peak": f"{hbm} GB/s {peak_kind}", "single_query_us_p50": 1e6 * statistics.median(lat),
            "mean_path_nodes": float(np.mean(lens)), "block_tier_launches": prof.get("path_query_block", (0, 0))[0],
            "wide_tier_launches": prof.get("path_query_wide", (0, 0))[0]}
        g.close()
        torch.cuda.synchronize()
    # CPU oracle at n = 2048: Algorithm 7 vs dense Dijkstra per query
    n = 2048
    W = synth.complete_digraph_i32(n, W_LO, W_HI, 20 + n)
    M = O.fw(W)
    alive = np.ones(n, dtype=bool)
    uv = np.stack([synth.uniform_int(23, n, 20, 0, n - 1), synth.uniform_int(24, n, 20, 0, n - 1)], 1)
    t0 = time.perf_counter()
    for u, v in uv:
        O.warm_shortest_path(M, W, alive, int(u), int(v))
    warm = (time.perf_counter() - t0) / len(uv)
    t0 = time.perf_counter()
    for u, _ in uv:
        O.dijkstra_rows(W, [int(u)])
    cold = (time.perf_counter() - t0) / len(uv)
    out["cpu_oracle_n2048"] = {"queries": len(uv), "alg7_ms_per_query": warm * 1e3,
                               "dijkstra_ms_per_query": cold * 1e3, "warm_over_cold": warm / cold,
                               "note": "oracle code as it stands (numpy / C), not tuned"}
    print(json.dumps(out))


class _ServeState:
    """Host view of one resident graph for generating valid requests: live
    slots (lowest-free-slot rule for adds) and the current edge weights."""

    def __init__(self, W, cap):
        self.n0, self.cap = W.shape[0], cap
        self.W0 = W
        self.alive = np.zeros(cap, bool)
        self.alive[:self.n0] = True
        self.mods = {}
        self.added = {}   # slot -> (in_w, out_w) of a node added later

    def weight(self, u, v):
        if (u, v) in self.mods:
            return self.mods[(u, v)]
        if v in self.added:
            return int(self.added[v][0][u])
        if u in self.added:
            return int(self.added[u][1][v])
        return int(self.W0[u, v])


def _serve_requests(states, count, seed, stream):
    """count requests: 70 % edge updates (half halve, half x4), 20 % node
    add / remove (half each), 10 % distance queries; graph and targets
    uniform."""
    pick = synth.uniform_int(seed, stream, count, 0, len(states) - 1)
    kind = synth.uniform_f64(seed, stream + 1, count)
    r = synth.u64(seed, stream + 2, 2 * count)
    reqs = []
    for q in range(count):
        gi = int(pick[q])
        st = states[gi]
        live = np.flatnonzero(st.alive)
        a = int(r[2 * q] % np.uint64(len(live)))
        b = int(r[2 * q + 1] % np.uint64(len(live) - 1))
        b += b >= a
        u, v = int(live[a]), int(live[b])
        k = kind[q]
        if k < 0.10:
            reqs.append((gi, "query", u, v))
            continue
        if k < 0.20:
            if len(live) < st.cap:
                iw = np.full(st.cap, synth.INF_I32, np.int32)
                ow = np.full(st.cap, synth.INF_I32, np.int32)
                iw[live] = synth.uniform_int(seed, 100000 + 2 * q + stream, len(live), 1, 10**6)
                ow[live] = synth.uniform_int(seed, 100001 + 2 * q + stream, len(live), 1, 10**6)
                p = int(np.flatnonzero(~st.alive)[0])
                st.alive[p] = True
                st.added[p] = (iw, ow)
                for key in [kk for kk in st.mods if p in kk]:
                    del st.mods[key]
                reqs.append((gi, "add", iw, ow))
                continue
            k = 0.25
        if k < 0.30:
            st.alive[u] = False
            reqs.append((gi, "remove", u))
        else:
            w0 = st.weight(u, v)
            w = w0 // 2 if k < 0.65 else min(w0 * 4, 1 << 26)
            st.mods[(u, v)] = w
            reqs.append((gi, "edge", u, v, float(w)))
    return reqs


def run_serve_study(args):
    """Serving: 64 resident directed complete graphs (16 each of n = 1024,
    2048, 4096, 8192; int32 U[1, 1e6]); Poisson arrivals swept from 10 % to
    110 % of the measured capacity; p50 / p99 latency and throughput; a tight
    HBM budget that forces queuing; and the alone-vs-in-the-mix identity
    (graphs replayed alone give the same matrices)."""
    from paper_2412_15122_gb300 import Graph, build
    from paper_2412_15122_gb300 import apsp as A
    build.build()
    sizes = [n for n in (1024, 2048, 4096, 8192) for _ in range(args.serve_per_size)]
    specs, graphs, states = [], [], []
    t_gen = time.perf_counter()
    for k, n in enumerate(sizes):
        W = synth.complete_digraph_i32(n, 1, 10**6, 500 + k)
        cap = n + 64
        specs.append((W, cap))
        graphs.append(Graph(W, cap))
        states.append(_ServeState(W, cap))
    gen_s = time.perf_counter() - t_gen
    small = args.serve_small_slots
    history = [[] for _ in graphs]
    hs = [g.h for g in graphs]

    def run(reqs, arrivals, budget=0.0):
        res = A.apsp_serve(hs, reqs, arrivals, hbm_budget_bytes=budget, small_max_slots=small)
        for q, it in enumerate(reqs):
            history[it[0]].append(it)
        lat = res["done_s"] - np.asarray(arrivals)
        span = float(res["done_s"].max() - np.asarray(arrivals).min())
        return {"requests": len(reqs), "ok": int((res["status"] == 0).sum()),
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "throughput_per_s": len(reqs) / span, "waves": int(res["wave"].max() + 1)}, res

    N = args.serve_requests
    stream = 10
    # warm-up: lets the batched kernel's width autotuner settle on this mix
    warm_rounds = 0
    while small > 0 and A.apsp_batch_tuned_width(A.APSP_I32, small) == 0 and warm_rounds < 6:
        reqs = _serve_requests(states, N, 5, stream)
        stream += 10
        run(reqs, np.zeros(len(reqs)))
        warm_rounds += 1
    # capacity: everything arrives at once
    reqs = _serve_requests(states, N, 5, stream)
    stream += 10
    cal, _ = run(reqs, np.zeros(len(reqs)))
    C = cal["throughput_per_s"]
    sweep = {}
    for frac in (0.1, 0.5, 0.9, 1.1):
        reqs = _serve_requests(states, N, 5, stream)
        stream += 10
        gaps = -np.log1p(-synth.uniform_f64(5, stream + 7, N)) / (frac * C)
        sweep[f"{frac:.1f}"], _ = run(reqs, np.cumsum(gaps))
    # tight budget: about four of the smallest graphs per wave
    reqs = _serve_requests(states, N, 5, stream)
    stream += 10
    gaps = -np.log1p(-synth.uniform_f64(5, stream + 7, N)) / (0.5 * C)
    budget = 4 * 3 * (1024 + 128) ** 2 * 4.0
    tight, _ = run(reqs, np.cumsum(gaps), budget)
    # alone vs in the mix: the n=1024 graphs replayed alone
    same = True
    for gi in range(args.serve_per_size):
        W, cap = specs[gi]
        g = Graph(W, cap)
        for it in history[gi]:
            if it[1] == "add":
                g.add_node(it[2], it[3])
            elif it[1] == "remove":
                g.remove_node(it[2])
            elif it[1] == "edge":
                g.update_edge(it[2], it[3], it[4])
        same &= bool(np.array_equal(g.D(), graphs[gi].D()))
        g.close()
    for g in graphs:
        g.close()
    print(json.dumps({
        "study": "serving", "graphs": len(sizes), "sizes": [1024, 2048, 4096, 8192], "per_size": args.serve_per_size,
        "mix": "70% edge updates (half halve, half x4), 20% node add/remove (half each), 10% queries; uniform graph and targets",
        "batched_graphs": f"capacity <= {small} in the persistent batched kernel (one CTA per graph), larger via one call "
                          "per update",
        "warm_up_rounds": warm_rounds, "batch_width": A.apsp_batch_tuned_width(A.APSP_I32, small) if small > 0 else None,
        "capacity_requests_per_s": C, "calibration": cal, "poisson_sweep_fraction_of_capacity": sweep,
        "tight_budget": {"budget_bytes": budget, "at_fraction": 0.5, **tight},
        "alone_vs_mix_identical_n1024": same, "setup_seconds": gen_s}))


def run_minimax_study(args):
    """Minimax (bottleneck) distances: warm against cold per update.  Directed
    complete graphs with int32 weights U[1, 1e6] (n = 1024 and 4096); the same
    seeded removals, tight-edge increases and decreases go to two graphs, one
    always warm and one always cold ((min, max) Floyd-Warshall); each update
    is timed with CUDA events on the library's stream; the matrices are
    compared after every update."""
    import torch
    from paper_2412_15122_gb300 import Graph, build
    build.build()
    stream = torch.cuda.Stream()
    out = {}
    for n in (1024, 4096):
        cap = n + 32
        W = synth.complete_digraph_i32(n, 1, 10**6, 900 + n)
        gw = Graph(W, cap, stream=stream, minimax=True)
        gc = Graph(W, cap, stream=stream, minimax=True)
        gw.set_dispatch("warm")
        gc.set_dispatch("cold")
        Wm = np.full((cap, cap), synth.INF_I32, np.int32)
        Wm[:n, :n] = W
        alive = np.zeros(cap, bool)
        alive[:n] = True
        ups = synth.mixed_updates(n, args.study_updates, 900 + n, fractions=(0.0, 0.34, 0.33, 0.33), tight=True,
                                  capacity=cap, stream=95)
        rec = {}
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for up in ups:
            live = np.flatnonzero(alive)
            if up.kind == synth.REMOVE:
                k = int(live[up.a])
                call = lambda g, k=k: g.remove_node(k)
                alive[k] = False
                Wm[k, :] = Wm[:, k] = synth.INF_I32
            else:
                u = int(live[up.a])
                row = np.where(alive, Wm[u].astype(np.int64), synth.INF_I32)
                row[u] = synth.INF_I32
                v = int(np.argmin(row))
                w = int(Wm[u, v]) // 2 if up.kind == synth.DECREASE else int(Wm[u, v]) * 4 + 1
                call = lambda g, u=u, v=v, w=w: g.update_edge(u, v, w)
                Wm[u, v] = w
            times = []
            for g in (gw, gc):
                e0.record(stream)
                call(g)
                e1.record(stream)
                g.sync()
                times.append(e0.elapsed_time(e1))
            st = gw.stats()
            r = rec.setdefault(up.kind, {"count": 0, "warm_ms": 0.0, "cold_ms": 0.0, "pairs": 0, "cost": 0.0,
                                         "passes": 0, "warm_faster": 0})
            r["count"] += 1
            r["warm_ms"] += times[0]
            r["cold_ms"] += times[1]
            r["pairs"] += st["affected_pairs"]
            r["cost"] += st["cost"]
            r["passes"] += st["passes"]
            r["warm_faster"] += times[0] < times[1]
        same = bool(np.array_equal(gw.D(), gc.D()))
        gw.close()
        gc.close()
        for r in rec.values():
            c = max(1, r["count"])
            for f in ("warm_ms", "cold_ms", "pairs", "cost", "passes"):
                r["avg_" + f] = round(r.pop(f) / c, 4)
        out[str(n)] = {"per_type": rec, "warm_and_cold_identical": same}
    print(json.dumps({"study": "minimax", "updates_per_size": args.study_updates,
                      "workload": "directed complete graphs, int32 U[1, 1e6], minimax distances; removals, "
                                  "lightest-out-edge increases (x4 + 1) and decreases (halved)",
                      "results": out}))


def detailed_pass(Graph, A, W, ops, stream, profile=False):
    """Replays `ops` on a fresh graph, one wait per update: per update type
    the count, the library's statistics and the device time of the update
    (CUDA events on the library's stream around its call), for all updates
    and for the non-trivial ones (path not "trivial" / "none").  With
    `profile`, also the per-kernel totals of the pass."""
    import torch
    g = Graph(W, CAP, stream=stream)
    if profile:
        A.apsp_profile_enable(g.h, True)
        A.apsp_profile_reset(g.h)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = {}
    for op in ops:
        e0.record(stream)
        issue_op(A, g, op, None)
        e1.record(stream)
        st = g.stats()
        ms = e0.elapsed_time(e1)
        k = stats.setdefault(st["op"], {"count": 0, "paths": {}, "pairs": 0, "rows": 0, "passes": 0,
                                         "sweep_rows": 0, "max_pairs": 0, "pairs_rechecked": 0,
                                         "warm_pass1_us": 0.0, "warm_total_us": 0.0, "device_ms": 0.0,
                                         "nontrivial": 0, "nontrivial_ms": 0.0, "warm": 0, "warm_pairs": 0})
        k["count"] += 1
        k["paths"][st["path"]] = k["paths"].get(st["path"], 0) + 1
        k["pairs"] += st["affected_pairs"]
        k["rows"] += st["affected_rows"]
        k["passes"] += st["passes"]
        k["sweep_rows"] += st["sweep_rows"]
        k["pairs_rechecked"] += st["pairs_rechecked"]
        k["warm_pass1_us"] += st["warm_pass1_us"]
        k["warm_total_us"] += st["warm_total_us"]
        k["max_pairs"] = max(k["max_pairs"], st["affected_pairs"])
        k["device_ms"] += ms
        if st["path"] not in ("trivial", "none"):
            k["nontrivial"] += 1
            k["nontrivial_ms"] += ms
        if st["path"] == "warm":
            k["warm"] += 1
            k["warm_pairs"] += st["affected_pairs"]
    prof = A.apsp_profile_read(g.h) if profile else {}
    span = g.info()["n_slots"]
    g.close()
    for k in stats.values():
        c = max(1, k["count"])
        for f in ("pairs", "rows", "passes", "sweep_rows", "pairs_rechecked"):
            k["avg_" + f] = round(k.pop(f) / c, 2)
        w = max(1, k["warm"])
        k["avg_warm_pass1_us"] = round(k.pop("warm_pass1_us") / w, 2)
        k["avg_warm_total_us"] = round(k.pop("warm_total_us") / w, 2)
        k["avg_warm_pairs"] = round(k.pop("warm_pairs") / w, 1)
        k["device_ms"] = round(k["device_ms"], 3)
        k["updates_per_s"] = round(k["count"] / (k["device_ms"] / 1000.0), 1) if k["device_ms"] > 0 else None
        k["nontrivial_ms"] = round(k["nontrivial_ms"], 3)
        k["nontrivial_updates_per_s"] = (round(k["nontrivial"] / (k["nontrivial_ms"] / 1000.0), 1)
                                         if k["nontrivial_ms"] > 0 else None)
    return stats, prof, span


def issue_op(A, g, op, device_vecs):
    """One library call for one planned update."""
    if op[0] == "add":
        if device_vecs is not None:
            A.apsp_add_node_device(g.h, device_vecs[id(op)][0], device_vecs[id(op)][1])
        else:
            A.apsp_add_node(g.h, op[1], op[2])
    elif op[0] == "remove":
        A.apsp_remove_node(g.h, op[1])
    else:
        A.apsp_update_edge(g.h, op[1], op[2], op[3], A.APSP_I32)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--updates", type=int, default=100, help="updates per step")
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-rows", type=int, default=1024)
    ap.add_argument("--no-stats", action="store_true")
    ap.add_argument("--tight-updates", type=int, default=1000, help="updates of the tight-edge mix (0: skip)")
    ap.add_argument("--no-fw-cpu", action="store_true", help="skip the host Floyd-Warshall timings")
    ap.add_argument("--case", choices=["removals", "inserts", "paths"],
                    help="run a small fixed case of the workload (for profiler captures) and exit")
    ap.add_argument("--study-graphs", type=int, default=512)
    ap.add_argument("--serve-per-size", type=int, default=16)
    ap.add_argument("--serve-requests", type=int, default=1000)
    ap.add_argument("--serve-small-slots", type=int, default=0,
                    help="serving: graphs of capacity <= this go through the batched kernel (one CTA per graph); "
                         "0: every graph one call per update on its own stream")
    ap.add_argument("--study-queries", type=int, default=4096)
    ap.add_argument("--study-reps", type=int, default=20)
    ap.add_argument("--study", choices=["dispatch", "batch", "serve", "paths", "ratios", "minimax"],
                    help="dispatch: train the warm/cold cost model and compare it with the delta rule, "
                         "always-warm and always-cold on n=16384 undirected Euclidean updates")
    ap.add_argument("--study-updates", type=int, default=100)
    ap.add_argument("--study-arms", default="delta,model,warm,cold,warm_exact_list,warm_direct_filter,warm_algorithm12",
                    help="dispatch study: comma-separated arms to run")
    ap.add_argument("--study-samples", type=int, default=20000)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.case:
        return run_case(args.case)
    if args.study == "dispatch":
        return run_dispatch_study(args)
    if args.study == "batch":
        return run_batch_study(args)
    if args.study == "serve":
        return run_serve_study(args)
    if args.study == "paths":
        return run_path_study(args)
    if args.study == "ratios":
        return run_ratio_study(args)
    if args.study == "minimax":
        return run_minimax_study(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_2412_15122_gb300 import Graph, build
    from paper_2412_15122_gb300 import apsp as A
    build.build()

    seed = rank_seed(rank)
    total = (args.warmup + args.steps) * args.updates
    W, ops = plan_ops(total, seed)
    ops_value = ops_e2e = ops          # the same workload, replayed on a fresh graph for e2e
    stream = torch.cuda.Stream()
    hbm, peak_kind = peaks()

    def issue(g, op, device_vecs):
        issue_op(A, g, op, device_vecs)

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    # ---- value: inputs resident in HBM ----------------------------------------
    U = args.updates
    dvec = {id(op): (torch.from_numpy(op[1]).cuda(), torch.from_numpy(op[2]).cuda())
            for op in ops_value if op[0] == "add"}

    def device_pass(profile: bool, want_clocks: bool):
        g = Graph(W, CAP, stream=stream)
        torch.cuda.synchronize()
        for s in range(args.warmup):
            for op in ops_value[s * U:(s + 1) * U]:
                issue(g, op, dvec)
        g.sync()
        if profile:
            A.apsp_profile_enable(g.h, True)
            A.apsp_profile_reset(g.h)
        launches0 = g.launches()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        clk = Clocks(local) if want_clocks else None
        if clk:
            clk.__enter__()
        ev0.record(stream)
        for s in range(args.warmup, args.warmup + args.steps):
            for op in ops_value[s * U:(s + 1) * U]:
                issue(g, op, dvec)
        ev1.record(stream)
        g.sync()
        barrier()
        if clk:
            clk.__exit__(None, None, None)
        ms = ev0.elapsed_time(ev1)
        nl = g.launches() - launches0
        prof = A.apsp_profile_read(g.h) if profile else {}
        cold = None
        if not profile:
            # cold FW on the final graph (the comparison baseline)
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            g.recompute()
            c1.record(stream)
            g.sync()
            cold = c0.elapsed_time(c1)
        span = g.info()["n_slots"]
        g.close()
        return ms, nl, prof, cold, span, clk

    ms, gpu_launches, _, cold_ms, span, clk = device_pass(profile=False, want_clocks=True)
    ms = job_ms(ms, dist)
    n_updates = args.steps * U * world
    value = job_value(args.steps * U, world, ms)
    prof_ms, _, prof, _, _, _ = device_pass(profile=True, want_clocks=False)

    # ---- statistics of the workload (untimed, one wait per update) -----------
    stats = {}
    if rank == 0 and not args.no_stats:
        stats, _, _ = detailed_pass(Graph, A, W, ops_value[: (args.warmup + args.steps) * U], stream)

    # ---- the tight-edge mix: every edge update on a shortest path -------------
    tight = None
    if rank == 0 and not args.no_stats and args.tight_updates > 0:
        _, tops = plan_ops(args.tight_updates, seed + 7, tight=True, W=W)
        gt = Graph(W, CAP, stream=stream)
        torch.cuda.synchronize()
        t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0e.record(stream)
        for op in tops:
            issue(gt, op, None)
        t1e.record(stream)
        gt.sync()
        tight_ms = t0e.elapsed_time(t1e)
        gt.close()
        tstats, tprof, tspan = detailed_pass(Graph, A, W, tops, stream, profile=True)
        tight = {"workload": f"the same graph and mix, {args.tight_updates} updates, every edge update on the "
                             "lightest out-edge of a uniform node (a shortest path: increases are never trivial)",
                 "value": args.tight_updates / (tight_ms / 1000.0), "unit": UNIT, "ms": tight_ms,
                 "per_type": tstats,
                 "kernels": {k: {"launches": v[0], "total_ms": round(v[1], 3)} for k, v in sorted(tprof.items())}}
        dec = tstats.get("decrease")
        if dec and "decrease_sweep" in tprof and tprof["decrease_sweep"][1] > 0:
            nl, tot = tprof["decrease_sweep"]
            b = 4.0 * tspan * dec["avg_sweep_rows"] * dec["count"]      # rows swept x one row of D each
            tight["decrease_sweep_roofline"] = {"bound": "hbm", "achieved": b / (tot / 1000.0) / 1e9, "peak": hbm,
                                                "unit": "GB/s", "frac": b / (tot / 1000.0) / 1e9 / hbm,
                                                "bytes_per_launch": b / max(1, nl), "launches": nl,
                                                "avg_launch_us": 1000.0 * tot / max(1, nl)}
        inc = tstats.get("increase")
        if inc and inc.get("avg_warm_pass1_us", 0) > 0:
            l2 = A.apsp_probe_l2_read_gbs()
            b = 4.0 * tspan * inc["avg_warm_pairs"]
            tight["increase_repair_roofline"] = {
                "bound": "l2", "kernel": "k_repair_p1, first re-relaxation pass (tight increases)",
                "achieved": b / (inc["avg_warm_pass1_us"] * 1e-6) / 1e9, "peak": l2, "unit": "GB/s",
                "frac": b / (inc["avg_warm_pass1_us"] * 1e-6) / 1e9 / l2, "bytes_per_increase": b,
                "pass1_us_per_increase": inc["avg_warm_pass1_us"], "warm_total_us": inc["avg_warm_total_us"]}
    del dvec

    # ---- e2e: host buffers through the C ABI ---------------------------------
    g = Graph(W, CAP, stream=stream)
    qpairs = np.stack([synth.uniform_int(seed, 41, 16, 0, N - 1), synth.uniform_int(seed, 42, 16, 0, N - 1)], 1)
    h2d = 0
    for s in range(args.warmup):
        for op in ops_e2e[s * U:(s + 1) * U]:
            issue(g, op, None)
    g.sync()
    # the query pairs of every step, from the host's own slot simulation
    quv = step_queries(ops_e2e, U, set(range(args.warmup, args.warmup + args.steps)), qpairs)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(stream)
    d2h = 0
    for s in range(args.warmup, args.warmup + args.steps):
        for op in ops_e2e[s * U:(s + 1) * U]:
            issue(g, op, None)
            if op[0] == "add":
                h2d += op[1].nbytes + op[2].nbytes
        uv = quv[s]
        h2d += uv.nbytes
        res = g.query_batch(uv)
        d2h += res.nbytes
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    wall_ms = (time.perf_counter() - t0) * 1000
    e2e_ms = job_ms(e2e_ms, dist)
    e2e_value = job_value(args.steps * U, world, e2e_ms)
    g.close()

    # ---- roofline of the dominant sweep kernel --------------------------------
    top = max(prof.items(), key=lambda kv: kv[1][1]) if prof else ("none", (0, 0.0))
    sweep = {k: v for k, v in prof.items() if k in SWEEP_KERNELS}
    rk = max(sweep.items(), key=lambda kv: kv[1][1]) if sweep else None
    roofline = None
    if rk:
        name, (nl, tot_ms) = rk
        bytes_per_launch = 4.0 * span * span      # one full read of D (span x span int32)
        achieved = bytes_per_launch / (tot_ms / nl / 1000.0) / 1e9
        roofline = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                    "frac": achieved / hbm, "peak_kind": f"{peak_kind} copy bandwidth",
                    "traffic": SWEEP_TRAFFIC.get(name), "traffic_source": TRAFFIC_SOURCE,
                    "bytes_per_launch": bytes_per_launch, "launches": nl,
                    "avg_launch_us": 1000 * tot_ms / nl}

    # cold FW against the CUDA cores' measured min-plus issue rate (ALU bound)
    fw_roofline = None
    if cold_ms:
        peak_ops = A.apsp_probe_addmin_rate(A.APSP_I32)
        fw_ops = float(span) ** 3 / (cold_ms / 1000.0)
        fw_roofline = {"bound": "alu", "kernel": "fw_phase1/2/3", "achieved": fw_ops / 1e9, "peak": peak_ops / 1e9,
                       "unit": "Gpair-op/s", "frac": fw_ops / peak_ops,
                       "peak_kind": "measured: register-tile probe of min(a + b, c), int32 (apsp_probe_addmin_rate)",
                       "work": "span^3 add-min pairs"}

    # the dominant kernel (warm repair): its first pass against the measured L2
    # read bandwidth (its reads are served by L2: rows and columns of a
    # 1024-column window of x stay resident)
    repair_roofline = None
    rm = stats.get("remove") if stats else None
    if rm and rm.get("avg_warm_pass1_us", 0) > 0:
        l2 = A.apsp_probe_l2_read_gbs()
        p1_bytes = 4.0 * span * rm["avg_pairs"]       # a column slice of every listed pair over all x
        p1_gbs = p1_bytes / (rm["avg_warm_pass1_us"] * 1e-6) / 1e9
        repair_roofline = {"bound": "l2", "kernel": "k_repair_p1, first re-relaxation pass (removals)", "achieved": p1_gbs,
                           "peak": l2, "unit": "GB/s", "frac": p1_gbs / l2,
                           "peak_kind": "measured: L2 read probe (apsp_probe_l2_read_gbs)",
                           "bytes_per_removal": p1_bytes, "pass1_us_per_removal": rm["avg_warm_pass1_us"]}

    fw_cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.no_fw_cpu:
        fw_cpu = fw_cpu_timings()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, cores, dt = cpu_oracle_rate(W, args.cpu_rows)
        cpu = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_rows} of {N} source rows of the initial graph by dense Dijkstra "
                         f"({dt:.1f} s), scaled x{N // args.cpu_rows} to one full recomputation per update"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N, "capacity": CAP, "updates_per_step": U,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (D alone is 268 MB)"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d // args.steps,
                    "d2h_bytes_per_step": d2h // args.steps, "wall_ms": wall_ms},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "clocks": clk.summary(),
            "gpu_launches": gpu_launches,
            "cold_fw_ms": cold_ms,
            "cold_fw_roofline": fw_roofline,
            "repair_roofline": repair_roofline,
            "roofline_note": ("roofline: the dominant HBM-bound kernel (a full streaming pass over D); the kernel with "
                              "the most total time is the warm repair, whose first pass is served by L2 and is "
                              "reported against the measured L2 read bandwidth in repair_roofline"),
            "profiled_pass_ms": prof_ms,
            "update_stats": stats,
            "tight_mix": tight,
            "fw_cpu": fw_cpu,
            "warm_updates_per_cold_fw": value * cold_ms / 1000.0,
            "top_kernel": {"name": top[0], "launches": top[1][0], "total_ms": top[1][1]},
            "kernels": {k: {"launches": v[0], "total_ms": round(v[1], 3)} for k, v in sorted(prof.items())},
        }
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
