"""Pins for the oracle's minimax (bottleneck path) variant, which the paper's
Discussion proposes: brute force over loop-free paths, the textbook minimum
spanning tree property, and the warm insertion and removal list against it."""
import numpy as np
import pytest

import synth
from oracle import apsp as O


def rand_graph(n, seed, lo=1, hi=20, p_missing=0.0, undirected=False):
    W = synth.complete_digraph_i32(n, lo, hi, seed)
    if p_missing > 0:
        m = synth.uniform_f64(seed, 99, n * n).reshape(n, n) < p_missing
        np.fill_diagonal(m, False)
        W = W.copy()
        W[m] = synth.INF_I32
    if undirected:
        W = np.minimum(W, W.T)
    return W


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("undirected", [False, True])
@pytest.mark.parametrize("pm", [0.0, 0.4])
def test_fw_minimax_matches_brute_force(seed, undirected, pm):
    W = rand_graph(7, seed, p_missing=pm, undirected=undirected)
    assert np.array_equal(O.fw_minimax(W), O.brute_force_minimax(W))


def _mst_bottleneck(W):
    """Prim's minimum spanning tree of a connected undirected graph, then the
    largest edge on the tree path between every pair."""
    E = O.exact(W)
    n = E.shape[0]
    in_tree = [0]
    adj = {v: [] for v in range(n)}
    best = {v: (E[0, v], 0) for v in range(1, n)}
    while best:
        v = min(best, key=lambda x: (best[x][0], x))
        w, u = best.pop(v)
        adj[u].append((v, w))
        adj[v].append((u, w))
        in_tree.append(v)
        for x in best:
            if E[v, x] < best[x][0]:
                best[x] = (E[v, x], v)
    B = np.zeros((n, n), dtype=np.int64)
    for s in range(n):
        stack = [(s, -1, 0)]
        while stack:
            u, parent, worst = stack.pop()
            B[s, u] = worst
            for v, w in adj[u]:
                if v != parent:
                    stack.append((v, u, max(worst, w)))
    return B


@pytest.mark.parametrize("seed", range(5))
def test_undirected_minimax_equals_mst_path_bottleneck(seed):
    # textbook: in a connected undirected graph the minimax distance is the
    # largest edge on the minimum spanning tree path
    W = rand_graph(40, 70 + seed, lo=1, hi=10**6, undirected=True)
    assert np.array_equal(O.fw_minimax(W), _mst_bottleneck(W))


@pytest.mark.parametrize("seed", range(6))
def test_minimax_insertion_matches_brute_force(seed):
    n = 7
    W = rand_graph(n, 20 + seed, p_missing=0.3)
    for p in (0, 3, 6):
        alive = np.ones(n, dtype=bool)
        alive[p] = False
        M = O.fw_minimax(W, alive)
        M2 = O.add_node_minimax(M, alive, p, W[:, p], W[p, :])
        assert np.array_equal(M2, O.brute_force_minimax(W))


@pytest.mark.parametrize("seed", range(6))
def test_minimax_removal_list_covers_every_change(seed):
    n = 7
    W = rand_graph(n, 40 + seed, hi=6, p_missing=0.2)
    M = O.fw_minimax(W)
    alive = np.ones(n, dtype=bool)
    for k in range(n):
        a2 = alive.copy()
        a2[k] = False
        after = O.brute_force_minimax(W, a2)
        listed = {(i, j) for i, js in O.need_update_list_minimax(M, alive, k).items() for j in js}
        for i in range(n):
            for j in range(n):
                if i != j and k not in (i, j) and after[i, j] != M[i, j]:
                    assert (i, j) in listed


def test_planted_sum_instead_of_max_is_caught():
    caught = 0
    for seed in range(5):
        W = rand_graph(6, 60 + seed)
        D = O.exact(W)
        for k in range(6):
            D = np.minimum(D, D[:, k:k + 1] + D[k:k + 1, :])   # min-plus, not min-max
        caught += not np.array_equal(D, O.brute_force_minimax(W))
    assert caught > 0
