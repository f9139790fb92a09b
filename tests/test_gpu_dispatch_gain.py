"""What the learned warm / cold dispatch gains over Algorithm 5's fixed
threshold on Cost.

Workload where the two paths genuinely compete: node removals on small
directed complete graphs (n = 128 .. 512) with int32 weights in [0, 3]
(ties everywhere, Cost near 1) or in [1, 1000].  Measured on GB300, the cold
Floyd-Warshall wins most n = 128 removals with weights [0, 3] while the warm
repair wins by 2-3x at n = 256 .. 512 with the same Cost of 1, so no
threshold on Cost alone can pick both right; the network also sees n and
the list size.

1. Training labels come from the library itself: every removal runs on two
   graphs, one always warm and one always cold, each timed with CUDA events;
   the features are the ones the device computes at its decision point.
2. The crossover delta is measured on the same samples: the threshold on Cost
   with the least total time (Algorithm 5's rule at its best setting).
3. The network is trained on the GPU (apsp_model_train).
4. On held-out graphs (other seeds) each removal again runs always warm and
   always cold, and on a graph using the model and one using the delta rule
   at the crossover.  Both rules are charged the measured time of the path
   they chose, so the comparison is free of timing noise; the model's total
   must not exceed the delta rule's.  Every graph ends with the same matrix,
   which equals the oracle's Floyd-Warshall.
"""
import math

import numpy as np
import pytest

import synth
from oracle import apsp as O

pytestmark = pytest.mark.gpu

SIZES = (128, 192, 256, 384, 512)
WEIGHTS = ((0, 3), (1, 1000))


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2412_15122_gb300 import Graph, build
    from paper_2412_15122_gb300 import apsp as A
    build.build()
    stream = torch.cuda.Stream()
    return torch, Graph, A, stream


def _removals(env, n, lo, hi, seed, count, extra_modes=()):
    """Runs `count` seeded removals on graphs that are always warm, always cold
    and one per extra mode; returns per removal (features, warm ms, cold ms,
    {mode: path}) and the graphs' final matrices."""
    torch, Graph, A, stream = env
    W = synth.complete_digraph_i32(n, lo, hi, seed)
    cap = n + 8
    modes = [("warm", 1.0), ("cold", 1.0)] + list(extra_modes)
    gs = []
    for m, delta in modes:
        g = Graph(W, cap, stream=stream)
        if m == "model":
            g.set_model(delta)              # `delta` holds the network's parameters here
            g.set_dispatch("model", 1.0)
        else:
            g.set_dispatch(m, delta)
        gs.append(g)
    alive = np.zeros(cap, bool)
    alive[:n] = True
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rows = []
    for t in range(count):
        live = np.flatnonzero(alive)
        N = len(live)
        k = int(live[synth.uniform_int(seed, 100 + t, 1, 0, N - 1)[0]])
        ms, paths = [], {}
        for (m, _), g in zip(modes, gs):
            e0.record(stream)
            g.remove_node(k)
            e1.record(stream)
            g.sync()
            ms.append(e0.elapsed_time(e1))
            paths[m] = g.stats()["path"]
        st = gs[0].stats()
        feat = [1.0 / 3.0, math.log2(N), 0.0, st["affected_pairs"] / float(N * N), st["cost"],
                st["affected_rows"] / float(N)]
        rows.append((feat, ms[0], ms[1], paths))
        alive[k] = False
    Ds = [g.D() for g in gs]
    for g in gs:
        g.close()
    Wm = np.full((cap, cap), synth.INF_I32, np.int32)
    Wm[:n, :n] = W
    m = Ds[0].shape[0]
    ref = O.to_i32(O.fw(Wm[:m, :m], alive[:m]))
    live = np.flatnonzero(alive[:m])
    for D in Ds:
        assert np.array_equal(D[np.ix_(live, live)], ref[np.ix_(live, live)])
    return rows, Ds


def test_model_dispatch_no_worse_than_delta_rule_at_measured_crossover(env):
    torch, Graph, A, stream = env
    # 1. training samples (labels: log2 of microseconds, warm and cold)
    X, Y, costs, tw, tc = [], [], [], [], []
    for n in SIZES:
        for (lo, hi) in WEIGHTS:
            for seed in (1, 2):
                rows, _ = _removals(env, n, lo, hi, 1000 * seed + n + hi, 10)
                for feat, w_ms, c_ms, _ in rows:
                    X.append(feat)
                    Y.append([math.log2(max(w_ms, 1e-3) * 1000.0), math.log2(max(c_ms, 1e-3) * 1000.0)])
                    costs.append(feat[4])
                    tw.append(w_ms)
                    tc.append(c_ms)
    costs, tw, tc = np.array(costs), np.array(tw), np.array(tc)
    assert (tc < tw).any() and (tw < tc).any(), "warm and cold must each win somewhere"
    # 2. the measured crossover: Algorithm 5's threshold with the least total time
    cands = np.unique(np.concatenate([[0.0, 1.0], costs]))
    totals = [np.where(costs > d, tc, tw).sum() for d in cands]
    delta = float(cands[int(np.argmin(totals))])
    # 3. train the network on the GPU
    params, loss = A.apsp_model_train(np.array(X, np.float32), np.array(Y, np.float32), epochs=400, batch=32,
                                      lr=3e-3, seed=5)
    assert np.isfinite(loss)
    # 4. held-out graphs: both rules charged the measured time of their choice
    tot_model = tot_delta = tot_warm = tot_cold = tot_best = 0.0
    for n in (128, 256, 512):
        for (lo, hi) in WEIGHTS:
            rows, _ = _removals(env, n, lo, hi, 7000 + n + hi, 10, [("model", params), ("delta", delta)])
            for _, w_ms, c_ms, paths in rows:
                pick = {m: (c_ms if paths[m] == "cold" else w_ms) for m in ("model", "delta")}
                tot_model += pick["model"]
                tot_delta += pick["delta"]
                tot_warm += w_ms
                tot_cold += c_ms
                tot_best += min(w_ms, c_ms)
    print(f"crossover delta {delta:.3f}; held-out totals (ms): model {tot_model:.3f}, delta rule {tot_delta:.3f}, "
          f"always warm {tot_warm:.3f}, always cold {tot_cold:.3f}, best possible {tot_best:.3f}")
    assert tot_model <= tot_delta * 1.02 + 1e-3
