"""Pins for the oracle's path queries (Algorithm 7, Algorithm 8), Algorithm
10/11's key_node_list and the need_update_lists of Algorithms 11 and 12,
against things other than the oracle itself:

* every loop-free path enumerated by brute force (n <= 7): the shortest ones
  and their length;
* closed forms (a directed cycle has one path; a "diamond" of m equal
  two-edge routes has exactly m shortest paths, all found by Algorithm 8);
* the definition behind Theorem theo_algo12: the pairs whose distance grows
  when a node is removed, by brute force on the graph without that node;
* the essential nodes of a pair (on every shortest path), by brute force;
* planted mistakes in copies of the oracle's steps.
"""
import numpy as np
import pytest

import synth
from oracle import apsp as O


def rand_graph(n, seed, lo=0, hi=9, p_missing=0.0, undirected=False):
    W = synth.complete_digraph_i32(n, lo, hi, seed)
    if p_missing > 0:
        m = synth.uniform_f64(seed, 99, n * n).reshape(n, n) < p_missing
        np.fill_diagonal(m, False)
        W = W.copy()
        W[m] = synth.INF_I32
    if undirected:
        W = np.minimum(W, W.T)
    return W


def all_simple_paths(W, s, t):
    """Every loop-free path s -> t with its exact length (DFS)."""
    E = O.exact(W)
    n = E.shape[0]
    out = []
    stack = [(s, [s], 0)]
    while stack:
        u, path, L = stack.pop()
        if u == t:
            out.append((path, L))
            continue
        for v in range(n):
            if v in path or E[u, v] >= O.INF:
                continue
            stack.append((v, path + [v], L + E[u, v]))
    return out


def shortest_simple_paths(W, s, t):
    ps = all_simple_paths(W, s, t)
    if not ps:
        return [], O.INF
    best = min(L for _, L in ps)
    return [p for p, L in ps if L == best], best


CASES = [dict(n=n, seed=s, lo=lo, p_missing=pm, undirected=u)
         for n in (2, 4, 6, 7) for s in (1, 2, 3) for lo in (0, 1) for pm in (0.0, 0.4) for u in (False, True)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
def test_alg7_path_is_a_brute_force_shortest_path(case, oracle_lib):
    W = rand_graph(**case)
    n = W.shape[0]
    alive = np.ones(n, dtype=bool)
    M = O.fw(W)
    for i in range(n):
        for j in range(n):
            p = O.warm_shortest_path(M, W, alive, i, j)
            if i == j:
                assert p == [i]
                continue
            best, L = shortest_simple_paths(W, i, j)
            if not best:
                assert p == [] and M[i, j] == O.INF
                continue
            assert p in best, (i, j, p, best)
            assert O.path_length(W, p) == L == M[i, j]


@pytest.mark.parametrize("case", CASES[::3], ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
def test_alg8_paths_are_distinct_shortest_paths(case, oracle_lib):
    W = rand_graph(**case)
    n = W.shape[0]
    alive = np.ones(n, dtype=bool)
    M = O.fw(W)
    for i in range(n):
        for j in range(n):
            ps = O.all_shortest_paths_alg8(M, W, alive, i, j)
            if i == j:
                assert ps == [[i]]
                continue
            best, _ = shortest_simple_paths(W, i, j)
            assert len(ps) == len({tuple(p) for p in ps})
            for p in ps:
                assert p in best
            if best:
                assert ps[0] == O.warm_shortest_path(M, W, alive, i, j)


def test_alg8_diamond_closed_form(oracle_lib):
    # s = 0 -> t_k -> j = m + 1 with weights 3 and 4 for every k, plus a direct
    # edge of 8 and edges between the t's of 5: exactly m shortest paths of 7.
    m = 6
    n = m + 2
    W = np.full((n, n), synth.INF_I32, dtype=np.int32)
    np.fill_diagonal(W, 0)
    for k in range(1, m + 1):
        W[0, k], W[k, n - 1] = 3, 4
        for k2 in range(1, m + 1):
            if k2 != k:
                W[k, k2] = 5
    W[0, n - 1] = 8
    M = O.fw(W)
    alive = np.ones(n, dtype=bool)
    assert O.candidate_node_list(M, alive, 0, n - 1) == list(range(n))
    ps = O.all_shortest_paths_alg8(M, W, alive, 0, n - 1)
    assert sorted(ps) == [[0, k, n - 1] for k in range(1, m + 1)]
    assert O.warm_shortest_path(M, W, alive, 0, n - 1) == [0, 1, n - 1]   # lowest index on a tie


def test_alg7_directed_cycle_closed_form(oracle_lib):
    n = 40
    w = synth.uniform_int(7, 0, n, 1, 100)
    W = np.full((n, n), synth.INF_I32, dtype=np.int32)
    np.fill_diagonal(W, 0)
    for i in range(n):
        W[i, (i + 1) % n] = w[i]
    M = O.fw(W)
    alive = np.ones(n, dtype=bool)
    for i, j in [(0, 39), (5, 4), (17, 23), (39, 0)]:
        expect = [(i + s) % n for s in range((j - i) % n + 1)]
        assert O.warm_shortest_path(M, W, alive, i, j) == expect


def test_alg7_dead_slots_and_unreachable(oracle_lib):
    W = rand_graph(7, 4, lo=1, p_missing=0.5)
    alive = np.array([1, 1, 0, 1, 1, 0, 1], dtype=bool)
    M = O.fw(W, alive)
    live = np.flatnonzero(alive)
    sub = W[np.ix_(live, live)]
    for a, i in enumerate(live):
        for b, j in enumerate(live):
            p = O.warm_shortest_path(M, W, alive, int(i), int(j))
            assert not any(x in (2, 5) for x in p)
            best, _ = shortest_simple_paths(sub, a, b)
            if a != b:
                assert [int(np.flatnonzero(live == x)[0]) for x in p] in best or (not best and p == [])


@pytest.mark.parametrize("seed", range(10))
@pytest.mark.parametrize("lo", [0, 1])
def test_alg12_list_is_exactly_the_pairs_that_grow(seed, lo, oracle_lib):
    n = 7
    W = rand_graph(n, seed, lo=lo, hi=4, p_missing=0.2 if seed % 2 else 0.0)
    alive = np.ones(n, dtype=bool)
    M = O.fw(W)
    for k in range(n):
        a2 = alive.copy()
        a2[k] = False
        after = O.brute_force_apsp(W, a2)
        grow = {(i, j) for i in range(n) for j in range(n)
                if i != j and k not in (i, j) and after[i, j] > M[i, j]}
        lst = O.need_update_list_alg12(M, W, alive, k)
        got = {(i, j) for i, js in lst.items() for j in js}
        assert got == grow
        full = {(i, j) for i, js in O.need_update_list(M, alive, k).items() for j in js}
        assert got <= full


def test_alg12_prunes_ties_that_corollary3_lists(oracle_lib):
    # Two equal routes 0 -> 1 -> 3 and 0 -> 2 -> 3: removing 1 lists (0, 3)
    # under Corollary 3 but its distance does not grow.
    W = np.full((4, 4), synth.INF_I32, dtype=np.int32)
    np.fill_diagonal(W, 0)
    W[0, 1] = W[1, 3] = W[0, 2] = W[2, 3] = 2
    M = O.fw(W)
    alive = np.ones(4, dtype=bool)
    assert 3 in O.need_update_list(M, alive, 1)[0]
    assert O.need_update_list_alg12(M, W, alive, 1)[0] == []
    assert O.need_update_list_alg12(M, W, alive, 1) == {0: [], 2: [], 3: []}


def test_planted_strict_candidate_test_is_caught(oracle_lib):
    # Writing the candidate test as "keep t iff SPD(i,t)+SPD(t,j) < SPD(i,j)"
    # keeps no intermediate node, so only direct edges remain.
    caught = 0
    for seed in range(6):
        W = rand_graph(6, seed, lo=1)
        M = O.fw(W)
        n = 6
        for i in range(n):
            for j in range(n):
                if i == j:
                    continue
                cand = [i] + [t for t in range(n) if t not in (i, j) and M[i, t] + M[t, j] < M[i, j]] + [j]
                _, pred = O.small_dijkstra(O.exact(W)[np.ix_(cand, cand)], 0)
                p = [cand[a] for a in O._tree_path(pred, 0, len(cand) - 1)]
                caught += O.path_length(W, p) != M[i, j]
    assert caught > 0


def test_planted_alg12_without_removing_k_is_caught(oracle_lib):
    # Leaving k among the candidates makes every pair's small-graph distance
    # equal SPD(i, j), so nothing is listed.
    caught = 0
    for seed in range(6):
        W = rand_graph(6, seed, lo=1, hi=5)
        M = O.fw(W)
        alive = np.ones(6, dtype=bool)
        for k in range(6):
            E = O.exact(W)
            rem = [v for v in range(6) if v != k]
            bad = set()
            for i in rem:
                for j in rem:
                    if i == j or M[i, j] < M[i, k] + M[k, j]:
                        continue
                    cand = [i] + [t for t in range(6) if t not in (i, j) and M[i, t] + M[t, j] <= M[i, j]] + [j]
                    dist, _ = O.small_dijkstra(E[np.ix_(cand, cand)], 0)
                    if dist[-1] > M[i, j]:
                        bad.add((i, j))
            good = {(i, j) for i, js in O.need_update_list_alg12(M, W, alive, k).items() for j in js}
            caught += bad != good
    assert caught > 0


def essential_nodes(W, i, j):
    """Nodes on every shortest loop-free path i -> j, without i and j (brute force)."""
    best, _ = shortest_simple_paths(W, i, j)
    if not best:
        return None
    common = set(best[0])
    for p in best[1:]:
        common &= set(p)
    return common - {i, j}


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("lo", [0, 1])
def test_key_node_list_contains_the_essential_nodes(seed, lo, oracle_lib):
    n = 7
    W = rand_graph(n, seed, lo=lo, hi=4, p_missing=0.2 if seed % 2 else 0.0)
    M = O.fw(W)
    alive = np.ones(n, dtype=bool)
    for i in range(n):
        for j in range(n):
            key = O.key_node_list(M, W, alive, i, j)
            ess = essential_nodes(W, i, j) if i != j else None
            if i == j or M[i, j] >= O.INF:
                assert key is None
                continue
            assert ess <= set(key)                       # a path set can only miss paths
            # the listed nodes lie on the first path (Psi), which is a shortest path
            assert set(key) <= set(O.warm_shortest_path(M, W, alive, i, j)) - {i, j}


@pytest.mark.parametrize("seed", range(6))
def test_key_node_list_is_the_path_interior_when_paths_are_unique(seed, oracle_lib):
    # weights U[1, 10^6] on 7 nodes: shortest paths are unique, so the
    # intersection is the interior of the one path
    n = 7
    W = synth.complete_digraph_i32(n, 1, 10**6, 500 + seed)
    M = O.fw(W)
    alive = np.ones(n, dtype=bool)
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            best, _ = shortest_simple_paths(W, i, j)
            assert len(best) == 1
            assert O.key_node_list(M, W, alive, i, j) == sorted(best[0][1:-1])


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("lo", [0, 1])
def test_alg11_list_between_alg12_and_corollary3(seed, lo, oracle_lib):
    n = 7
    W = rand_graph(n, seed, lo=lo, hi=4, p_missing=0.2 if seed % 2 else 0.0)
    M = O.fw(W)
    alive = np.ones(n, dtype=bool)
    for k in range(n):
        a11 = {(i, j) for i, js in O.need_update_list_alg11(M, W, alive, k).items() for j in js}
        a12 = {(i, j) for i, js in O.need_update_list_alg12(M, W, alive, k).items() for j in js}
        c3 = {(i, j) for i, js in O.need_update_list(M, alive, k).items() for j in js}
        assert a12 <= a11 <= c3


def test_alg11_equals_alg12_when_paths_are_unique(oracle_lib):
    n = 7
    for seed in range(4):
        W = synth.complete_digraph_i32(n, 1, 10**6, 600 + seed)
        M = O.fw(W)
        alive = np.ones(n, dtype=bool)
        for k in range(n):
            assert O.need_update_list_alg11(M, W, alive, k) == O.need_update_list_alg12(M, W, alive, k)


def test_planted_key_node_list_without_intersection_is_caught(oracle_lib):
    # Taking Psi's interior alone (no intersection with the other paths) lists
    # nodes that some other shortest path avoids: the essential-node pin fails.
    caught = 0
    for seed in range(8):
        W = rand_graph(6, seed, lo=0, hi=3)
        M = O.fw(W)
        alive = np.ones(6, dtype=bool)
        for i in range(6):
            for j in range(6):
                if i == j or M[i, j] >= O.INF:
                    continue
                bad = set(O.warm_shortest_path(M, W, alive, i, j)) - {i, j}
                ess = essential_nodes(W, i, j)
                caught += bad != ess
    assert caught > 0


@pytest.mark.parametrize("seed", range(6))
def test_alg7_float_paths_are_shortest(seed, oracle_lib):
    # lognormal fp32 weights: the float candidate test (with its slack) keeps
    # every node of some shortest path, so the small graph reaches the optimum
    n = 7
    W = synth.lognormal_digraph_f32(n, 80 + seed)
    M = O.fw(W)
    alive = np.ones(n, dtype=bool)
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            p = O.warm_shortest_path(M, W, alive, i, j)
            best, L = shortest_simple_paths(W.astype(np.float64), i, j)
            assert abs(O.path_length(W, p) - L) <= 1e-12 * L
            assert p[0] == i and p[-1] == j and len(set(p)) == len(p)


@pytest.mark.parametrize("seed", range(4))
def test_alg12_undirected_list_is_the_pairs_that_grow(seed, oracle_lib):
    n = 7
    W = rand_graph(n, 120 + seed, lo=0, hi=3, undirected=True)
    alive = np.ones(n, dtype=bool)
    M = O.fw(W)
    for k in range(n):
        a2 = alive.copy()
        a2[k] = False
        after = O.brute_force_apsp(W, a2)
        grow = {(i, j) for i in range(n) for j in range(n) if i != j and k not in (i, j) and after[i, j] > M[i, j]}
        got = {(i, j) for i, js in O.need_update_list_alg12(M, W, alive, k).items() for j in js}
        assert got == grow
        assert all((j, i) in got for (i, j) in got)      # symmetric, like the graph
