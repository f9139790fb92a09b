"""Pins for the CPU oracle: it is checked here against things other than itself.

* the definition of a shortest path distance, by two independent brute-force
  enumerations of loop-free paths (DFS and permutations), n <= 7;
* closed forms (directed cycle, unit-weight complete graph, path graph);
* the worked example of Section 3.2 (tests/golden/worked_example.json);
* invariants every APSP matrix satisfies;
* planted mistakes in copies of the oracle's functions, which these pins must catch.
"""
import itertools
import json
import os

import numpy as np
import pytest

import synth
from oracle import apsp as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def rand_graph(n, seed, lo=0, hi=9, p_missing=0.0, undirected=False, fp=False):
    if fp:
        W = synth.lognormal_digraph_f32(n, seed)
    else:
        W = synth.complete_digraph_i32(n, lo, hi, seed)
    if p_missing > 0:
        m = synth.uniform_f64(seed, 99, n * n).reshape(n, n) < p_missing
        np.fill_diagonal(m, False)
        W = W.copy()
        W[m] = np.inf if fp else synth.INF_I32
    if undirected:
        W = np.minimum(W, W.T)
    return W


CASES = [dict(n=n, seed=s, p_missing=pm, undirected=u, fp=fp)
         for n in (1, 2, 3, 5, 7) for s in (1, 2) for pm in (0.0, 0.4)
         for u in (False, True) for fp in (False, True)]


def close(a, b):
    if O.is_float(a):
        return np.allclose(a, b, rtol=1e-12, atol=0) and np.array_equal(np.isinf(a), np.isinf(b))
    return np.array_equal(a, b)


@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
def test_solvers_match_brute_force(case, oracle_lib):
    W = rand_graph(**case)
    B = O.brute_force_apsp(W)
    assert close(B, O.itertools_paths_min(W))
    assert close(O.fw(W), B)
    assert close(O.fw_python(W), B)
    assert close(O.dijkstra_rows(W, range(W.shape[0])), B)


def test_dead_slots_take_part_in_no_path(oracle_lib):
    W = rand_graph(7, 3)
    alive = np.array([1, 0, 1, 1, 0, 1, 1], dtype=bool)
    D = O.fw(W, alive)
    live = np.flatnonzero(alive)
    B = O.brute_force_apsp(W[np.ix_(live, live)])
    assert np.array_equal(D[np.ix_(live, live)], B)
    assert np.all(D[~alive, :] == O.INF) and np.all(D[:, ~alive] == O.INF)


def test_closed_form_directed_cycle(oracle_lib):
    # Directed cycle 0 -> 1 -> ... -> n-1 -> 0 with weights w_i: the only path
    # i -> j follows the cycle, so D[i][j] = sum of w from i up to j - 1.
    n = 300
    w = synth.uniform_int(5, 0, n, 0, 1000)
    W = np.full((n, n), synth.INF_I32, dtype=np.int32)
    np.fill_diagonal(W, 0)
    for i in range(n):
        W[i, (i + 1) % n] = w[i]
    pre = np.concatenate([[0], np.cumsum(np.concatenate([w, w]))])
    expect = np.empty((n, n), dtype=np.int64)
    for i in range(n):
        for j in range(n):
            jj = j if j >= i else j + n
            expect[i, j] = pre[jj] - pre[i]
    assert np.array_equal(O.fw(W), expect)
    assert np.array_equal(O.dijkstra_rows(W, [0, 17, n - 1]), expect[[0, 17, n - 1]])


def test_closed_form_unit_complete_and_path(oracle_lib):
    n = 200
    W = np.ones((n, n), dtype=np.int32)
    np.fill_diagonal(W, 0)
    D = O.fw(W)
    assert np.array_equal(D, 1 - np.eye(n, dtype=np.int64))
    # undirected path graph with unit weights: D[i][j] = |i - j|
    P = np.full((n, n), synth.INF_I32, dtype=np.int32)
    np.fill_diagonal(P, 0)
    idx = np.arange(n - 1)
    P[idx, idx + 1] = 1
    P[idx + 1, idx] = 1
    D = O.fw(P)
    assert np.array_equal(D, np.abs(np.arange(n)[:, None] - np.arange(n)[None, :]))


def test_invariants_hold_and_catch_errors(oracle_lib):
    W = rand_graph(40, 4, lo=1, hi=50, p_missing=0.3)
    alive = np.ones(40, dtype=bool)
    D = O.fw(W)
    assert O.check_invariants(W, D, alive) == []
    bad = D.copy()
    i, j = 3, 7
    bad[i, j] += 1                     # too large: no first edge is tight
    assert O.check_invariants(W, bad, alive)
    bad = D.copy()
    finite = np.argwhere((D > 0) & (D < O.INF))
    i, j = finite[0]
    bad[i, j] -= 1                     # too small: not achievable
    assert O.check_invariants(W, bad, alive)


# ---------------------------------------------------------------------------
# Worked example of Section 3.2
# ---------------------------------------------------------------------------

def worked_example():
    g = json.load(open(os.path.join(GOLD, "worked_example.json")))
    names = g["nodes"]
    ix = {c: i for i, c in enumerate(names)}
    n = len(names)
    W = np.full((n, n), synth.INF_I32, dtype=np.int32)
    np.fill_diagonal(W, 0)
    for a, b, w in g["undirected_edges"]:
        W[ix[a], ix[b]] = W[ix[b], ix[a]] = w
    return g, names, ix, W


def test_worked_example_need_update_lists_and_costs(oracle_lib):
    g, names, ix, W = worked_example()
    alive = np.ones(len(names), dtype=bool)
    M = O.fw(W)
    for node in ("C", "B"):
        spec = g[f"remove_{node}"]
        lst = O.need_update_list(M, alive, ix[node])
        got = {names[i]: sorted(names[j] for j in js) for i, js in lst.items()}
        assert got == {k: sorted(v) for k, v in spec["need_update_list"].items()}
        assert O.cost_of_remove(lst, len(names)) == spec["cost"]
        a2 = alive.copy()
        a2[ix[node]] = False
        M2 = O.brute_force_apsp(W, a2)
        for a, b in spec.get("changed_pairs", []):
            assert M2[ix[a], ix[b]] != M[ix[a], ix[b]]
        for a, b in spec["unchanged_pairs"]:
            assert M2[ix[a], ix[b]] == M[ix[a], ix[b]]


# ---------------------------------------------------------------------------
# Section 3.1 (adding a node) and Algorithm 1's warm start as a cold solver
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("undirected", [False, True])
def test_add_node_matches_brute_force(seed, undirected, oracle_lib):
    n = 7
    W = rand_graph(n, seed, lo=0, hi=12, p_missing=0.2 * (seed % 2), undirected=undirected)
    p = seed % n
    alive = np.ones(n, dtype=bool)
    alive[p] = False
    M = O.fw(W, alive)
    M2 = O.add_node(M, alive, p, W[:, p], W[p, :])
    assert np.array_equal(M2, O.brute_force_apsp(W))


def test_add_node_float(oracle_lib):
    W = rand_graph(7, 11, fp=True)
    alive = np.ones(7, dtype=bool)
    alive[2] = False
    M2 = O.add_node(O.fw(W, alive), alive, 2, W[:, 2], W[2, :])
    assert close(M2, O.brute_force_apsp(W))


def test_inserting_every_node_from_empty_equals_fw(oracle_lib):
    # Algorithm 1 used cold: start from the empty graph and add the nodes one
    # at a time with the warm start of Section 3.1; the end result is the APSP
    # matrix of the whole graph.
    n = 60
    W = rand_graph(n, 8, lo=0, hi=100, p_missing=0.5)
    alive = np.zeros(n, dtype=bool)
    M = O.exact(W, alive)
    for p in synth.u64(8, 3, n).argsort():
        M = O.add_node(M, alive, int(p), W[:, p], W[p, :])
        alive[p] = True
    assert np.array_equal(M, O.fw(W))


# ---------------------------------------------------------------------------
# Algorithms 5 and 6
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("delta", [0.0, 1.0])
def test_remove_node_alg5_matches_brute_force(seed, delta, oracle_lib):
    n = 7
    W = rand_graph(n, seed + 20, lo=0, hi=6, undirected=bool(seed % 2))
    alive = np.ones(n, dtype=bool)
    M = O.fw(W)
    k = seed % n
    M2, alive2, info = O.remove_node_alg5(W, M, alive, k, delta)
    assert np.array_equal(M2, O.brute_force_apsp(W, alive2))
    # every pair whose distance changed was in need_update_list (Corollary 3)
    for i, j in zip(*np.nonzero(M2 != M)):
        if alive2[i] and alive2[j]:
            assert j in info["list"][int(i)]


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("factor", ["halve", "x4", "delete", "zero"])
def test_modify_edge_alg6_matches_brute_force(seed, factor, oracle_lib):
    n = 7
    und = bool(seed % 2)
    W = rand_graph(n, seed + 40, lo=1, hi=9, undirected=und)
    alive = np.ones(n, dtype=bool)
    M = O.fw(W)
    u, v = seed % n, (seed * 3 + 1) % n
    if u == v:
        v = (v + 1) % n
    w = {"halve": W[u, v] // 2, "x4": W[u, v] * 4, "delete": synth.INF_I32, "zero": 0}[factor]
    M2, W2 = O.modify_edge_alg6(W, M, alive, (u, v), w, delta=0.5, undirected=und)
    assert np.array_equal(M2, O.brute_force_apsp(W2))


@pytest.mark.parametrize("seed", range(6))
def test_edge_affected_set_covers_every_change(seed, oracle_lib):
    n = 7
    und = bool(seed % 2)
    W = rand_graph(n, seed + 60, lo=0, hi=5, undirected=und)
    M = O.fw(W)
    alive = np.ones(n, dtype=bool)
    # the lightest out-edge of u is always a shortest path
    u = seed % n
    row = W[u].astype(np.int64).copy()
    row[u] = 1 << 40
    v = int(np.argmin(row))
    aff = O.edge_affected_pairs(M, alive, u, v, int(W[u, v]), und)
    assert (u, v) in aff
    W2 = W.copy()
    W2[u, v] = W[u, v] * 4 + 3
    if und:
        W2[v, u] = W2[u, v]
    M2 = O.brute_force_apsp(W2)
    for i, j in zip(*np.nonzero(M2 != M)):
        assert (int(i), int(j)) in aff


# ---------------------------------------------------------------------------
# Planted mistakes: copies of oracle functions with one plausible bug each
# must fail the pins above.
# ---------------------------------------------------------------------------

def test_planted_transposed_operand_in_corollary1_is_caught(oracle_lib):
    def add_node_bad(M, alive, p, in_w, out_w):
        live = np.flatnonzero(alive)
        out_row = np.full(M.shape[0], O.INF, dtype=np.int64)
        in_col = np.full(M.shape[0], O.INF, dtype=np.int64)
        for r in live:
            out_row[r] = np.min(out_w[live].astype(np.int64) + M[r, live])   # M[r,t] instead of M[t,r]
            in_col[r] = np.min(M[r, live] + in_w[live].astype(np.int64))
        M2 = M.copy()
        for i in live:
            M2[i, live] = np.minimum(M[i, live], in_col[i] + out_row[live])
        M2[p, :], M2[:, p], M2[p, p] = out_row, in_col, 0
        return M2

    caught = 0
    for seed in range(6):
        W = rand_graph(7, seed, lo=1, hi=12)
        alive = np.ones(7, dtype=bool)
        alive[0] = False
        M2 = add_node_bad(O.fw(W, alive), alive, 0, W[:, 0], W[0, :])
        caught += not np.array_equal(M2, O.brute_force_apsp(W))
    assert caught > 0


def test_planted_dropped_theorem3_term_is_caught(oracle_lib):
    caught = 0
    for seed in range(6):
        W = rand_graph(7, seed, lo=1, hi=12)
        alive = np.ones(7, dtype=bool)
        alive[3] = False
        M = O.fw(W, alive)
        good = O.add_node(M, alive, 3, W[:, 3], W[3, :])
        bad = M.copy()                      # Theorem 3 step left out: only row/col p written
        bad[3, :], bad[:, 3] = good[3, :], good[:, 3]
        caught += not np.array_equal(bad, O.brute_force_apsp(W))
    assert caught > 0


def test_planted_wrong_tightness_and_cost_are_caught(oracle_lib):
    g, names, ix, W = worked_example()
    M = O.fw(W)
    alive = np.ones(4, dtype=bool)
    k = ix["B"]
    # strict test written the wrong way round: a tight pair counted as unneeded
    lst_bad = {i: [j for j in range(4) if j not in (i, k) and M[i, j] < M[i, k] + M[k, j]]
               for i in range(4) if i != k}
    assert {names[i]: sorted(names[j] for j in v) for i, v in lst_bad.items()} != g["remove_B"]["need_update_list"]
    # Cost over N instead of N - 1
    lst = O.need_update_list(M, alive, k)
    assert sum(1 for v in lst.values() if v) / 4 != g["remove_B"]["cost"]


def test_planted_fw_loop_order_is_caught(oracle_lib):
    # k innermost (a classic mistake) is not Floyd-Warshall
    caught = 0
    for seed in range(10):
        W = rand_graph(6, seed, lo=0, hi=20, p_missing=0.5)
        D = O.exact(W)
        n = D.shape[0]
        for i in range(n):
            for j in range(n):
                for k in range(n):
                    if D[i, k] < O.INF and D[k, j] < O.INF and D[i, k] + D[k, j] < D[i, j]:
                        D[i, j] = D[i, k] + D[k, j]
        caught += not np.array_equal(D, O.brute_force_apsp(W))
    assert caught > 0
