"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Int32 results must be bit-exact; fp32 results within 1e-5 relative of the
fp64 oracle.  The oracle side keeps its own copy of the weights in slot space
and recomputes the APSP matrix of the updated graph from scratch.
"""
import numpy as np
import pytest

import synth
from oracle import apsp as O

pytestmark = pytest.mark.gpu

F32_RTOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    from paper_2412_15122_gb300 import build
    build.build()


def G(*a, **k):
    from paper_2412_15122_gb300 import Graph
    return Graph(*a, **k)


class Mirror:
    """Oracle-side state: weights in slot space and the live mask."""

    def __init__(self, W, cap, undirected=False):
        n = W.shape[0]
        self.fp = W.dtype == np.float32
        self.inf = np.float32(np.inf) if self.fp else np.int32(synth.INF_I32)
        self.W = np.full((cap, cap), self.inf, dtype=W.dtype)
        self.W[:n, :n] = W
        self.alive = np.zeros(cap, dtype=bool)
        self.alive[:n] = True
        self.und = undirected
        self.cap = cap

    def add(self, in_w, out_w):
        p = O.lowest_free_slot(self.alive)
        live = self.alive.copy()
        self.W[:, p] = np.where(live, in_w, self.inf)
        self.W[p, :] = np.where(live, out_w, self.inf)
        self.W[p, p] = 0
        self.alive[p] = True
        return p

    def remove(self, k):
        self.alive[k] = False
        self.W[k, :] = self.inf
        self.W[:, k] = self.inf

    def edge(self, u, v, w):
        self.W[u, v] = w
        if self.und:
            self.W[v, u] = w

    def live(self):
        return np.flatnonzero(self.alive)

    def expected(self, m):
        return O.fw(self.W[:m, :m], self.alive[:m])


def assert_same(g, mir, tag=""):
    D = g.D()
    m = D.shape[0]
    ref = mir.expected(m)
    if mir.fp:
        Df = D.astype(np.float64)
        inf_ok = np.array_equal(np.isinf(Df), np.isinf(ref))
        fin = np.isfinite(ref)
        err = np.abs(Df[fin] - ref[fin]) <= F32_RTOL * np.abs(ref[fin]) + 1e-30
        assert inf_ok and err.all(), f"{tag}: fp32 mismatch, max rel err " \
            f"{np.max(np.abs(Df[fin] - ref[fin]) / np.maximum(np.abs(ref[fin]), 1e-30)) if fin.any() else 0}"
    else:
        got = D
        exp = O.to_i32(ref)
        if not np.array_equal(got, exp):
            bad = np.argwhere(got != exp)
            i, j = bad[0]
            raise AssertionError(f"{tag}: {len(bad)} entries differ, first ({i},{j}) got {got[i, j]} expected {exp[i, j]}")


def make_graph(n, seed, fp=False, undirected=False, lo=1, hi=1000, p_missing=0.0):
    if fp:
        W = synth.lognormal_digraph_f32(n, seed)
    else:
        W = synth.complete_digraph_i32(n, lo, hi, seed)
    if p_missing > 0:
        m = synth.uniform_f64(seed, 77, n * n).reshape(n, n) < p_missing
        np.fill_diagonal(m, False)
        W = W.copy()
        W[m] = np.inf if fp else synth.INF_I32
    if undirected:
        W = np.minimum(W, W.T)
    return W


def apply(g, mir, up: synth.Update, rng_stream=0):
    """Apply one generated update to both sides; returns a tag."""
    live = mir.live()
    if up.kind == synth.ADD:
        in_w = np.full(mir.cap, mir.inf, dtype=mir.W.dtype)
        out_w = np.full(mir.cap, mir.inf, dtype=mir.W.dtype)
        in_w[live] = up.in_w[:len(live)]
        out_w[live] = up.out_w[:len(live)] if not mir.und else up.in_w[:len(live)]
        if mir.und:
            out_w = in_w.copy()
        p = g.add_node(in_w, out_w)
        q = mir.add(in_w, out_w)
        assert p == q
        return f"add {p}"
    if up.kind == synth.REMOVE:
        k = int(live[up.a])
        g.remove_node(k)
        mir.remove(k)
        return f"remove {k}"
    u = int(live[up.a])
    if up.tight:
        row = mir.W[u].astype(np.float64).copy()
        row[~mir.alive] = np.inf
        row[u] = np.inf
        v = int(np.argmin(row))
    else:
        v = int(live[up.b])
    w0 = mir.W[u, v]
    if up.kind == synth.DECREASE:
        w = np.float32(w0 / 2) if mir.fp else np.int32(w0 // 2)
    else:
        w = np.float32(w0 * 4) if mir.fp else np.int32(min(int(w0) * 4, up.cap))
    g.update_edge(u, v, w)
    mir.edge(u, v, w)
    return f"{up.kind} ({u},{v}) {w0}->{w}"


# ---------------------------------------------------------------------------

INIT_CASES = [(n, fp, und, pm) for n in (1, 2, 3, 31, 33, 130, 257) for fp in (False, True)
              for und in (False, True) for pm in (0.0, 0.5)]


@pytest.mark.parametrize("n,fp,und,pm", INIT_CASES)
def test_init_floyd_warshall_matches_oracle(n, fp, und, pm):
    W = make_graph(n, 3 + n, fp=fp, undirected=und, lo=0, hi=50, p_missing=pm)
    g = G(W, n + 5, undirected=und)
    assert_same(g, Mirror(W, n + 5, und), "init")
    g.close()


@pytest.mark.parametrize("tight", [False, True])
def test_plain_method_chain_n256(tight):
    # n = 256 directed complete graph, int32 weights U[1, 1000], D from the
    # CPU Floyd-Warshall handed in; then one add, one removal, one decrease
    # (halved) and one increase (x4), each checked bit-exact.
    n, cap = 256, 320
    W = synth.complete_digraph_i32(n, 1, 1000, seed=1)
    D0 = O.to_i32(O.fw(W))
    g = G(W, cap, D=D0)
    mir = Mirror(W, cap)
    assert_same(g, mir, "init (given D)")
    ups = [synth.Update(synth.ADD, in_w=synth.uniform_int(1, 10, n, 1, 1000).astype(np.int32),
                        out_w=synth.uniform_int(1, 11, n, 1, 1000).astype(np.int32)),
           synth.Update(synth.REMOVE, a=int(synth.uniform_int(1, 12, 1, 0, n)[0])),
           synth.Update(synth.DECREASE, a=5, b=77, tight=tight),
           synth.Update(synth.INCREASE, a=9, b=140, tight=tight)]
    for up in ups:
        tag = apply(g, mir, up)
        assert_same(g, mir, tag)
        st = g.stats()
        assert st["op"] == up.kind
    g.close()


SEQ = [(n, fp, und, tight, seed) for n in (40, 200) for fp in (False, True) for und in (False, True)
       for tight in (False, True) for seed in (1,)] + [(513, False, False, True, 2), (300, True, False, True, 3)]


@pytest.mark.parametrize("n,fp,und,tight,seed", SEQ)
def test_mixed_update_sequences(n, fp, und, tight, seed):
    W = make_graph(n, seed, fp=fp, undirected=und, lo=0 if not fp else 1, hi=200)
    cap = n + 24
    g = G(W, cap, undirected=und)
    mir = Mirror(W, cap, und)
    ups = synth.mixed_updates(n, 30, seed, tight=tight, capacity=cap, w_lo=0, w_hi=200,
                              weights="lognormal" if fp else "int")
    for t, up in enumerate(ups):
        tag = apply(g, mir, up)
        assert_same(g, mir, f"step {t}: {tag}")
    g.close()


@pytest.mark.parametrize("mode", ["warm", "cold", "delta"])
@pytest.mark.parametrize("und", [False, True])
def test_dispatch_modes_give_identical_results(mode, und):
    n = 150
    W = make_graph(n, 9, undirected=und, lo=1, hi=30)
    cap = n + 10
    g = G(W, cap, undirected=und)
    g.set_dispatch(mode, 0.2)
    mir = Mirror(W, cap, und)
    for t, up in enumerate(synth.mixed_updates(n, 16, 9, fractions=(0.1, 0.45, 0.0, 0.45), tight=True,
                                               capacity=cap, w_lo=1, w_hi=30)):
        tag = apply(g, mir, up)
        assert_same(g, mir, f"{mode} step {t}: {tag}")
        st = g.stats()
        if mode == "cold" and st["op"] in ("remove", "increase"):
            assert st["path"] in ("cold", "trivial")
        if mode == "warm":
            assert st["path"] != "cold"
    g.close()


def test_worked_example_need_update_list_on_gpu():
    import json, os
    spec = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_example.json")))
    names = spec["nodes"]
    ix = {c: i for i, c in enumerate(names)}
    W = np.full((4, 4), synth.INF_I32, dtype=np.int32)
    np.fill_diagonal(W, 0)
    for a, b, w in spec["undirected_edges"]:
        W[ix[a], ix[b]] = W[ix[b], ix[a]] = w
    for node, rows, cost in (("C", 0, 0.0), ("B", 3, 1.0)):
        g = G(W, 4, undirected=True)
        g.remove_node(ix[node])
        st = g.stats()
        assert st["affected_rows"] == rows
        assert st["affected_pairs"] == sum(len(v) for v in spec[f"remove_{node}"]["need_update_list"].values())
        assert abs(st["cost"] - cost) < 1e-6
        mir = Mirror(W, 4, True)
        mir.remove(ix[node])
        assert_same(g, mir, f"remove {node}")
        g.close()


def pair_set(lst):
    """{i: [j, ...]} (the oracle's lists) -> set of (i, j)."""
    return {(int(i), int(j)) for i, js in lst.items() for j in js}


def device_pairs(g):
    """The device's list of the last update as a set; no pair listed twice."""
    ij = g.last_list()
    s = {(int(a), int(b)) for a, b in ij}
    assert len(s) == len(ij), "a pair is listed twice"
    return s


@pytest.mark.parametrize("case", ["uniform1", "uniform2", "uniform3", "euclid", "euclid_fp"])
def test_affected_set_matches_oracle_need_update_list(case):
    # The device detection lists exactly the need_update_list of Section 3.2,
    # pair by pair: removals on a directed uniform graph and on a tie-heavy
    # undirected Euclidean graph (rounded distances, weights <= 40), three
    # removals in a row each.
    n = 180
    und = case.startswith("euclid")
    if und:
        W, _ = synth.euclidean_undirected_i32(n, 31, scale=40.0)
    else:
        W = synth.complete_digraph_i32(n, 1, 100, int(case[-1]))
    if case == "euclid_fp":
        W = np.where(W >= synth.INF_I32, np.inf, W).astype(np.float32) * np.float32(0.25)
    g = G(W, n, undirected=und)
    g.set_dispatch("warm")
    mir = Mirror(W, n, und)
    for t in range(3):
        live = mir.live()
        M = mir.expected(n)
        k = int(live[synth.uniform_int(len(case), 5 + t, 1, 0, len(live) - 1)[0]])
        kept = O.need_update_list(M, mir.alive, k)
        g.remove_node(k)
        mir.remove(k)
        st = g.stats()
        want = pair_set(kept)
        if case == "euclid_fp":
            # fp32 lists by the conservative slack test: a superset of the
            # exact list, its extra pairs tight within the 2^-8 slack
            got = device_pairs(g)
            assert want <= got
            for (i, j) in got - want:
                via, d = M[i, k] + M[k, j], M[i, j]
                assert via <= d * (1 + 2.0 ** -7), (i, j, via, d)
        else:
            assert device_pairs(g) == want
            assert st["affected_rows"] == sum(1 for v in kept.values() if v)
        assert st["affected_pairs"] == len(g.last_list())
        assert_same(g, mir, f"{case} remove {k}")
    g.close()


def _direct_edge_pairs(lst, Wx, M):
    return sum(1 for i, js in lst.items() for j in js if Wx[i, j] != M[i, j])


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("undirected", [False, True])
@pytest.mark.parametrize("list_mode", ["corollary3", "direct_edge", "algorithm12"])
def test_exact_list_matches_oracle_algorithm12(seed, undirected, list_mode):
    # Small integer weights (0..4) make ties common, so Corollary 3 lists many
    # pairs whose distance does not grow; Algorithm 12's list drops them.  The
    # device's list is Corollary 3's, Corollary 3's minus the pairs whose direct
    # edge is a shortest path, or Algorithm 12's, by list mode; the measured
    # Algorithm 12 list and the matrices are the same in every mode.
    n, cap = 60, 64
    W = make_graph(n, 700 + seed, undirected=undirected, lo=0, hi=4, p_missing=0.2)
    g = G(W, cap, undirected=undirected)
    g.set_exact_list(True)
    g.set_list_mode(list_mode)
    mir = Mirror(W, cap, undirected)
    assert g.stats()["grown_pairs"] == -1            # init: not a removal or increase
    for t in range(4):
        live = mir.live()
        M = mir.expected(cap)
        k = int(live[synth.uniform_int(seed, 90 + t, 1, 0, len(live) - 1)[0]])
        alg12 = O.need_update_list_alg12(M, mir.W, mir.alive, k)
        cor3 = O.need_update_list(M, mir.alive, k)
        Wx = O.exact(mir.W, mir.alive)
        g.remove_node(k)
        mir.remove(k)
        st = g.stats()
        got = device_pairs(g)
        if list_mode == "direct_edge":
            assert got == {(i, j) for (i, j) in pair_set(cor3) if Wx[i, j] != M[i, j]}
            assert st["affected_pairs"] == _direct_edge_pairs(cor3, Wx, M)
        elif list_mode == "algorithm12":   # the device list is Algorithm 12's (n < 126: no pair stays unchecked)
            assert got == pair_set(alg12)
            assert st["affected_rows"] == sum(1 for v in alg12.values() if v)
        else:
            assert got == pair_set(cor3)
        assert st["affected_pairs"] == len(got)
        assert st["grown_pairs"] == sum(len(v) for v in alg12.values())
        assert st["grown_rows"] == sum(1 for v in alg12.values() if v)
        N = len(live)
        assert abs(st["grown_cost"] - st["grown_rows"] / (N - 1)) < 1e-6
        assert_same(g, mir, f"remove {k}")
    # an edge increase on a tight edge: the list is the pairs whose distance grows
    live = mir.live()
    u = int(live[3])
    row = np.where(mir.alive, mir.W[u].astype(np.int64), 1 << 40)
    row[u] = 1 << 40
    v = int(np.argmin(row))
    before = mir.expected(cap)
    w_old = mir.W[u, v]
    w = int(mir.W[u, v]) * 4 + 3
    cand = O.edge_affected_pairs(before, mir.alive, u, v, int(w_old), undirected)
    g.update_edge(u, v, w)
    mir.edge(u, v, w)
    after = mir.expected(cap)
    st = g.stats()
    Wx = O.exact(mir.W, mir.alive)                   # the new weight: the changed edge is never dropped
    grown = (after > before) & np.outer(mir.alive, mir.alive)
    np.fill_diagonal(grown, False)
    got = device_pairs(g)
    cand_set = {(int(i), int(j)) for (i, j) in cand}
    if list_mode == "direct_edge":
        assert got == {(i, j) for (i, j) in cand_set if Wx[i, j] != before[i, j]}
    elif list_mode == "algorithm12":
        assert got == {(int(i), int(j)) for i, j in np.argwhere(grown)}
    else:
        assert got == cand_set
    assert st["affected_pairs"] == len(got)
    assert st["grown_pairs"] == int(grown.sum())
    assert st["grown_rows"] == int(grown.any(1).sum())
    assert_same(g, mir, "increase")
    g.close()


def test_insert_every_node_from_empty_graph():
    # Algorithm 1's warm start used from scratch: n insertions give FW.
    n = 70
    W = make_graph(n, 21, lo=0, hi=40, p_missing=0.3)
    g = G(np.zeros((0, 0), np.int32), n)
    mir = Mirror(np.zeros((0, 0), np.int32), n)
    for p in range(n):
        in_w = np.full(n, synth.INF_I32, np.int32)
        out_w = np.full(n, synth.INF_I32, np.int32)
        in_w[:p] = W[:p, p]
        out_w[:p] = W[p, :p]
        q = g.add_node(in_w, out_w)
        assert q == p == mir.add(in_w, out_w)
    assert_same(g, mir, "all inserted")
    ref = O.to_i32(O.fw(W))
    assert np.array_equal(g.D(), ref)
    g.close()


def test_errors_and_slot_reuse():
    from paper_2412_15122_gb300 import ApspError
    n, cap = 20, 21
    W = synth.complete_digraph_i32(n, 1, 50, 4)
    g = G(W, cap)
    mir = Mirror(W, cap)
    full = np.ones(cap, np.int32)
    p = g.add_node(full, full)
    mir.add(full, full)
    assert p == 20
    with pytest.raises(ApspError) as e:
        g.add_node(full, full)
    assert e.value.status == 4                           # no free slot
    with pytest.raises(ApspError) as e:
        g.update_edge(3, 3, 5)
    assert e.value.status == 1
    with pytest.raises(ApspError) as e:
        g.update_edge(3, 4, -1)
    assert e.value.status == 3
    g.remove_node(5)
    mir.remove(5)
    with pytest.raises(ApspError) as e:
        g.remove_node(5)
    assert e.value.status == 2
    with pytest.raises(ApspError) as e:
        g.update_edge(5, 4, 1)
    assert e.value.status == 2
    q = g.add_node(full * 3, full * 2)                   # the dead slot is reused
    assert q == 5 == mir.add(full * 3, full * 2)
    assert_same(g, mir, "reuse")
    g.update_edge(1, 2, synth.INF_I32)                   # delete an edge
    mir.edge(1, 2, synth.INF_I32)
    assert_same(g, mir, "delete edge")
    g.update_edge(2, 9, 0)                               # zero weight
    mir.edge(2, 9, 0)
    assert_same(g, mir, "zero weight")
    for k in list(mir.live())[:-1]:                      # down to one live node
        g.remove_node(int(k))
        mir.remove(int(k))
        assert_same(g, mir, f"remove {k}")
    g.close()


def test_float_nan_rejected_and_queries():
    from paper_2412_15122_gb300 import ApspError
    W = synth.lognormal_digraph_f32(30, 5)
    g = G(W, 32)
    with pytest.raises(ApspError) as e:
        g.update_edge(1, 2, np.float32(np.nan))
    assert e.value.status == 1
    ref = O.fw(W)
    uv = np.array([[0, 1], [5, 7], [29, 0], [3, 3]], dtype=np.int32)
    got = g.query_batch(uv)
    for (u, v), x in zip(uv, got):
        assert abs(float(x) - ref[u, v]) <= F32_RTOL * abs(ref[u, v])
        assert abs(float(g.query(int(u), int(v))) - ref[u, v]) <= F32_RTOL * abs(ref[u, v])
    g.close()


def test_device_inputs_for_add_node():
    import torch
    n, cap = 64, 80
    W = synth.complete_digraph_i32(n, 1, 100, 6)
    g = G(W, cap)
    mir = Mirror(W, cap)
    iw = synth.uniform_int(6, 1, cap, 1, 100).astype(np.int32)
    ow = synth.uniform_int(6, 2, cap, 1, 100).astype(np.int32)
    p = g.add_node(torch.from_numpy(iw).cuda(), torch.from_numpy(ow).cuda())
    assert p == mir.add(iw, ow)
    assert_same(g, mir, "device add")
    # the host mirror of the weights learned the new node: an edge update on it works
    g.update_edge(p, 3, int(mir.W[p, 3]) * 4)
    mir.edge(p, 3, mir.W[p, 3] * 4)
    assert_same(g, mir, "edge on device-added node")
    g.close()


@pytest.mark.parametrize("fp", [False, True])
def test_scale_n8192_sampled_rows(fp):
    # n = 8192 directed complete graph: GPU cold FW at init, then mixed updates;
    # 64 seeded source rows (plus the rows of touched nodes) checked by Dijkstra.
    n, cap = 8192, 8192 + 256
    W = synth.lognormal_digraph_f32(n, 2) if fp else synth.complete_digraph_i32(n, 1, 10**6, 2)
    g = G(W, cap)
    mir = Mirror(W, cap)
    touched = set()
    for up in synth.mixed_updates(n, 12, 2, capacity=cap, w_lo=1, w_hi=10**6, tight=True,
                                  weights="lognormal" if fp else "int"):
        tag = apply(g, mir, up)
        touched.update(int(x) for x in tag.replace("(", " ").replace(")", " ").replace(",", " ").split()
                       if x.isdigit() and int(x) < cap)
    m = g.info()["n_slots"]
    live = mir.live()
    rows = sorted(set(int(x) for x in live[synth.uniform_int(2, 9, 64, 0, len(live) - 1)]) |
                  (touched & set(int(x) for x in live)))
    ref = O.dijkstra_rows(mir.W[:m, :m], rows, mir.alive[:m])
    D = g.D()
    for r, row in zip(rows, ref):
        if fp:
            fin = np.isfinite(row)
            assert np.array_equal(np.isfinite(D[r]), fin)
            assert np.all(np.abs(D[r][fin] - row[fin]) <= F32_RTOL * np.abs(row[fin]))
        else:
            assert np.array_equal(D[r], O.to_i32(row)), f"row {r}"
    g.close()


@pytest.mark.parametrize("fp", [False, True])
def test_chunked_repair_n2048_full_check(fp):
    # Several x-chunks per pass-1 evaluation, so different warps relax the same
    # pair concurrently; wide rows (sources of tight edges) make it frequent.
    n, cap = 2048, 2048 + 32
    W = synth.lognormal_digraph_f32(n, 12) if fp else synth.complete_digraph_i32(n, 1, 10**6, 12)
    g = G(W, cap)
    mir = Mirror(W, cap)
    for up in synth.mixed_updates(n, 24, 12, fractions=(0.1, 0.3, 0.1, 0.5), capacity=cap, w_lo=1, w_hi=10**6,
                                  tight=True, weights="lognormal" if fp else "int"):
        apply(g, mir, up)
    assert_same(g, mir, "after 24 updates")
    g.close()


def test_config2_workload_n4096_full_matrix():
    # The benchmark's workload at the largest size the oracle checks in full:
    # n = 4096 directed complete graph, int32 U[1, 1e6], 100 mixed updates
    # (25 % each kind, uniform targets, half of the edge updates on tight
    # edges), then every entry against the oracle's Floyd-Warshall.
    n, cap = 4096, 4096 + 128
    W = synth.complete_digraph_i32(n, 1, 10**6, 42)
    g = G(W, cap)
    mir = Mirror(W, cap)
    for t, up in enumerate(synth.mixed_updates(n, 100, 42, capacity=cap, w_lo=1, w_hi=10**6, cap=1 << 26)):
        if up.kind in (synth.DECREASE, synth.INCREASE) and t % 2:
            up.tight = True
        apply(g, mir, up)
    assert_same(g, mir, "after 100 mixed updates")
    g.close()


def test_graphs_of_different_sizes_coexist():
    """A smaller graph created later must not restrict the launches of a
    larger one (per-function launch limits are process-wide)."""
    import synth
    from oracle import apsp as O
    from paper_2412_15122_gb300 import Graph, build
    build.build()
    Wb = synth.complete_digraph_i32(700, 1, 1000, 71)
    big = Graph(Wb, 720)
    mir = Mirror(Wb, 720)                            # the test's own copy of the weights
    small = Graph(synth.complete_digraph_i32(40, 1, 1000, 72), 48)
    big.remove_node(5)
    mir.remove(5)
    big.update_edge(3, 9, 1)
    mir.edge(3, 9, 1)
    big.update_edge(10, 11, 4000)
    mir.edge(10, 11, 4000)
    iw = synth.uniform_int(73, 1, 720, 1, 1000).astype(np.int32)
    ow = synth.uniform_int(73, 2, 720, 1, 1000).astype(np.int32)
    p = big.add_node(iw, ow)
    assert p == mir.add(iw, ow)
    small.remove_node(3)
    assert np.array_equal(big.alive().astype(bool), mir.alive[:big.info()["n_slots"]])
    assert_same(big, mir, "big graph beside a small one")
    big.close()
    small.close()
