"""Batched execution (one persistent launch for many graphs) against the
oracle and against the one-call-per-update path."""
import numpy as np
import pytest

import synth
from oracle import apsp as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2412_15122_gb300 import apsp, build
    build.build()
    return apsp


def _graph_and_updates(n, cap, seed, count, dtype, tight):
    if dtype == "f32":
        W = synth.lognormal_digraph_f32(n, seed)
        ups = synth.mixed_updates(n, count, seed, capacity=cap, weights="lognormal", tight=tight, stream=11)
    else:
        W = synth.complete_digraph_i32(n, 1, 1000, seed)
        ups = synth.mixed_updates(n, count, seed, capacity=cap, w_lo=1, w_hi=1000, tight=tight, stream=11)
    return W, ups


def _items_for(gi, ups, Wm, alive, cap, dtype):
    """Concrete items with slot ids, tracking the weight mirror and liveness
    the way the library assigns slots (lowest free slot)."""
    items = []
    inf = np.float32(np.inf) if dtype == "f32" else synth.INF_I32
    npdt = np.float32 if dtype == "f32" else np.int32
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
            items.append((gi, "add", iw, ow))
        elif up.kind == synth.REMOVE:
            k = int(live[up.a])
            alive[k] = False
            Wm[k, :] = inf
            Wm[:, k] = inf
            items.append((gi, "remove", k))
        else:
            u, v = int(live[up.a]), int(live[up.b])
            if up.tight:
                row = np.where(alive, Wm[u], inf).astype(np.float64)
                row[u] = np.inf
                v = int(np.argmin(row))
            w0 = Wm[u, v]
            w = (w0 // 2 if dtype == "i32" else np.float32(w0 / 2)) if up.kind == synth.DECREASE else \
                (min(int(w0) * 4, 1 << 26) if dtype == "i32" else np.float32(w0 * 4))
            Wm[u, v] = w
            items.append((gi, "edge", u, v, float(w)))
    return items


@pytest.mark.parametrize("dtype", ["i32", "f32"])
@pytest.mark.parametrize("tight", [False, True])
def test_batch_matches_oracle_and_single_calls(lib, dtype, tight):
    from paper_2412_15122_gb300 import Batch, Graph
    sizes = [40, 97, 130, 257]
    graphs, singles, items, mirrors = [], [], [], []
    for gi, n in enumerate(sizes):
        cap = n + 24
        W, ups = _graph_and_updates(n, cap, 100 + gi + (50 if tight else 0), 16, dtype, tight)
        g = Graph(W, cap)
        s = Graph(W, cap)
        inf = np.float32(np.inf) if dtype == "f32" else synth.INF_I32
        Wm = np.full((cap, cap), inf, W.dtype)
        Wm[:n, :n] = W
        alive = np.zeros(cap, bool)
        alive[:n] = True
        its = _items_for(gi, ups, Wm, alive, cap, dtype)
        graphs.append(g)
        singles.append(s)
        items += its
        mirrors.append((Wm, alive))
    # interleave the graphs' items (per-graph order is what counts)
    order = sorted(range(len(items)), key=lambda q: (q % 7, q))
    per_graph = {}
    for q in range(len(items)):
        per_graph.setdefault(items[q][0], []).append(q)
    mixed = []
    pos = {gi: 0 for gi in per_graph}
    for q in order:
        gi = items[q][0]
        mixed.append(items[per_graph[gi][pos[gi]]])
        pos[gi] += 1
    b = Batch()
    ids = b.run(graphs, mixed)
    assert (ids[[m[1] == "add" for m in mixed]] >= 0).all()
    for gi, (g, s) in enumerate(zip(graphs, singles)):
        for it in items:
            if it[0] != gi:
                continue
            if it[1] == "add":
                s.add_node(it[2], it[3])
            elif it[1] == "remove":
                s.remove_node(it[2])
            else:
                s.update_edge(it[2], it[3], it[4])
        Wm, alive = mirrors[gi]
        m = g.info()["n_slots"]
        Db, Ds = g.D(), s.D()
        np.testing.assert_array_equal(g.W()[:m, :m], Wm[:m, :m])
        np.testing.assert_array_equal(g.alive()[:m].astype(bool), alive[:m])
        ref = O.fw(Wm[:m, :m], alive[:m])
        live = np.flatnonzero(alive[:m])
        if dtype == "i32":
            np.testing.assert_array_equal(Db[np.ix_(live, live)], O.to_i32(ref)[np.ix_(live, live)])
            np.testing.assert_array_equal(Db, Ds)
        else:
            r = ref[np.ix_(live, live)]
            d = Db[np.ix_(live, live)].astype(np.float64)
            fin = np.isfinite(r)
            assert (np.isfinite(d) == fin).all()
            assert (np.abs(d[fin] - r[fin]) <= 1e-5 * np.abs(r[fin]) + 1e-6).all()
        g.close()
        s.close()
    b.close()


def test_batch_rejects_invalid_item_without_changes(lib):
    from paper_2412_15122_gb300 import ApspError, Batch, Graph
    W = synth.complete_digraph_i32(50, 1, 100, 3)
    g = Graph(W, 64)
    D0 = g.D().copy()
    b = Batch()
    with pytest.raises(ApspError):
        b.run([g], [(0, "remove", 5), (0, "remove", 5)])   # second removal of a dead node
    np.testing.assert_array_equal(g.D(), D0)
    assert g.alive()[5] == 1
    with pytest.raises(ApspError):
        b.run([g], [(0, "edge", 1, 2, -3.0)])
    b.run([g], [])
    b.close()
    g.close()


def test_batch_then_single_calls_continue(lib):
    from paper_2412_15122_gb300 import Batch, Graph
    W = synth.complete_digraph_i32(64, 1, 100, 9)
    g = Graph(W, 80)
    b = Batch()
    b.run([g], [(0, "remove", 3), (0, "edge", 4, 5, 1.0)])
    g.remove_node(10)   # the single-graph path sees the batch's state
    # the test's own copy of the weights after the three updates
    Wm = np.full((80, 80), synth.INF_I32, np.int32)
    Wm[:64, :64] = W
    alive = np.zeros(80, bool)
    alive[:64] = True
    for k in (3, 10):
        alive[k] = False
        Wm[k, :] = Wm[:, k] = synth.INF_I32
    Wm[4, 5] = 1
    m = g.info()["n_slots"]
    assert np.array_equal(g.alive()[:m].astype(bool), alive[:m])
    live = np.flatnonzero(alive[:m])
    ref = O.to_i32(O.fw(Wm[:m, :m], alive[:m]))
    np.testing.assert_array_equal(g.D()[np.ix_(live, live)], ref[np.ix_(live, live)])
    b.close()
    g.close()


def _workload(seed, sizes, per):
    """Graphs of the given sizes with `per` mixed updates each (int32 U[1, 1000])."""
    specs, items = [], []
    for gi, n in enumerate(sizes):
        cap = n + 24
        W, ups = _graph_and_updates(n, cap, seed + gi, per, "i32", False)
        Wm = np.full((cap, cap), synth.INF_I32, np.int32)
        Wm[:n, :n] = W
        alive = np.zeros(cap, bool)
        alive[:n] = True
        specs.append((W, cap))
        items += _items_for(gi, ups, Wm, alive, cap, "i32")
    return specs, items


def test_batch_widths_give_identical_results_and_replay_graphs(lib):
    # Every CTA width gives the same int32 matrices; repeated launches of one
    # executor replay its captured CUDA graph with new parameters.
    from paper_2412_15122_gb300 import Batch, Graph
    specs, items = _workload(300, [70, 129, 200], 12)
    ref = None
    for width in (128, 256, 512):
        graphs = [Graph(W, cap) for W, cap in specs]
        b = Batch()
        b.set_width(width)
        half = len(items) // 2
        first = [it for it in items[:half]]
        b.run(graphs, first)
        b.run(graphs, items[half:])
        info = b.info()
        assert info["launches"] == 2 and info["graph_captures"] == 1 and info["graph_replays"] == 2
        assert info["last_width"] == width and info["fixed_width"] == width
        Ds = [g.D() for g in graphs]
        if ref is None:
            ref = Ds
        else:
            for a, c in zip(ref, Ds):
                np.testing.assert_array_equal(a, c)
        for g in graphs:
            g.close()
        b.close()


def test_batch_autotuner_settles_on_a_width(lib):
    # Batches of enough work (>= 2^20 span^2) in one size bucket: after two
    # samples of each width the tuner keeps one of them.
    from paper_2412_15122_gb300 import Batch, Graph
    from paper_2412_15122_gb300 import apsp as A
    specs, items = _workload(400, [600, 700, 760, 640], 8)
    graphs = [Graph(W, cap) for W, cap in specs]
    Wm = [g.W() for g in graphs]
    b = Batch()
    settled_before = A.apsp_batch_tuned_width(A.APSP_I32, 784)
    widths = []
    for rep in range(8):
        # the same edge items again (weights toggled back and forth) keep the work per batch alike
        its = [it for it in items if it[1] == "edge"]
        if rep % 2:
            its = [(gi, "edge", u, v, float(Wm[gi][u, v])) for (gi, _, u, v, _) in its]
        b.run(graphs, its)
        widths.append(b.info()["last_width"])
    tuned = A.apsp_batch_tuned_width(A.APSP_I32, 784)
    assert tuned in (128, 256, 512)
    if settled_before == 0:
        assert set(widths[:6]) == {128, 256, 512}     # each width measured first
    assert widths[-1] == tuned
    for g in graphs:
        g.close()
    b.close()


@pytest.mark.parametrize("dtype", ["i32", "f32"])
@pytest.mark.parametrize("width", [256, 512])
def test_batch_teams_for_large_graphs(lib, dtype, width):
    # Graphs of n >= 384 go to teams of CTAs (a team barrier between steps,
    # scratch in global memory), the others to single CTAs, in one launch:
    # results equal one call per update (int32 bit for bit, fp32 within
    # 1e-5) and the oracle (every entry up to n = 1100, 64 sampled rows at
    # n = 2048).  Two launches in a row on one executor (the second replays
    # the captured graph and reuses the team scratch).
    from paper_2412_15122_gb300 import Batch, Graph
    sizes = [2048, 1100, 700, 400, 150, 90]
    graphs, singles, mirrors, per = [], [], [], []
    for gi, n in enumerate(sizes):
        cap = n + 24
        W, ups = _graph_and_updates(n, cap, 900 + gi, 24, dtype, gi % 2 == 0)
        graphs.append(Graph(W, cap))
        singles.append(Graph(W, cap))
        inf = np.float32(np.inf) if dtype == "f32" else synth.INF_I32
        Wm = np.full((cap, cap), inf, W.dtype)
        Wm[:n, :n] = W
        alive = np.zeros(cap, bool)
        alive[:n] = True
        per.append(_items_for(gi, ups, Wm, alive, cap, dtype))
        mirrors.append((Wm, alive))
    b = Batch()
    b.set_width(width)
    for half in (0, 1):
        its = [it for p in per for it in p[12 * half:12 * (half + 1)]]
        b.run(graphs, its)
        for it in its:
            s = singles[it[0]]
            if it[1] == "add":
                s.add_node(it[2], it[3])
            elif it[1] == "remove":
                s.remove_node(it[2])
            else:
                s.update_edge(it[2], it[3], it[4])
    assert b.info()["graph_replays"] == 2
    for gi, (g, s) in enumerate(zip(graphs, singles)):
        Db, Ds = g.D(), s.D()
        Wm, alive = mirrors[gi]
        m = Db.shape[0]
        live = np.flatnonzero(alive[:m])
        if dtype == "i32":
            np.testing.assert_array_equal(Db, Ds, err_msg=f"graph {gi}")
        else:
            fin = np.isfinite(Ds)
            assert np.array_equal(np.isfinite(Db), fin)
            assert (np.abs(Db[fin] - Ds[fin]) <= 1e-5 * np.abs(Ds[fin]) + 1e-6).all()
        if sizes[gi] <= 1100:
            ref = O.fw(Wm[:m, :m], alive[:m])[np.ix_(live, live)]
        else:
            pick = live[synth.uniform_int(gi, 9, 64, 0, len(live) - 1)]
            ref = O.dijkstra_rows(Wm[:m, :m], pick, alive[:m])[:, live]
            live_rows = pick
        rows = live if sizes[gi] <= 1100 else live_rows
        got = Db[np.ix_(rows, live)].astype(np.float64)
        if dtype == "i32":
            np.testing.assert_array_equal(got, O.to_i32(ref), err_msg=f"graph {gi} vs oracle")
        else:
            fin = np.isfinite(ref)
            assert np.array_equal(np.isfinite(got), fin)
            assert (np.abs(got[fin] - ref[fin]) <= 1e-5 * np.abs(ref[fin]) + 1e-6).all()
        g.close()
        s.close()
    b.close()
