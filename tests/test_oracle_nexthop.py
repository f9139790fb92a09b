"""Pins for the oracle's next hops (oracle.next_hop_row), against things other
than the oracle itself:

* brute force at n <= 7 with positive weights: the next hop is the lowest
  first node of the shortest loop-free paths enumerated by DFS;
* the invariant with zero weights and missing edges: w(i, t) + SPD(t, j) ==
  SPD(i, j) for the chosen t, and no lower t satisfies it;
* a closed form: on a directed cycle every next hop is the successor;
* following next hops reaches j with total weight SPD(i, j) (positive weights);
* planted mistakes (a strict comparison, the direct edge preferred) are caught.
"""
import numpy as np
import pytest

import synth
from oracle import apsp as O
from test_oracle_paths import all_simple_paths, rand_graph


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("n", [3, 5, 7])
def test_next_hop_is_lowest_first_hop_of_a_shortest_path(seed, n):
    W = rand_graph(n, 40 + seed, lo=1, hi=6, p_missing=0.2)
    M = O.brute_force_apsp(W)
    alive = np.ones(n, bool)
    for i in range(n):
        row = O.next_hop_row(O.fw(W), W, alive, i)
        for j in range(n):
            if i == j:
                assert row[j] == i
                continue
            paths = all_simple_paths(W, i, j)
            if not paths:
                assert row[j] == -1
                continue
            best = min(L for _, L in paths)
            assert best == M[i, j]
            assert row[j] == min(p[1] for p, L in paths if L == best), (i, j)


@pytest.mark.parametrize("seed", range(4))
def test_next_hop_invariant_with_zero_weights(seed):
    n = 30
    W = rand_graph(n, 70 + seed, lo=0, hi=3, p_missing=0.3)
    M = O.fw(W)
    E = O.exact(W)
    alive = np.ones(n, bool)
    alive[[4, 11]] = False
    M = O.fw(W, alive)
    E = O.exact(W, alive)
    for i in np.flatnonzero(alive):
        row = O.next_hop_row(M, W, alive, int(i))
        for j in range(n):
            if not alive[j] or M[i, j] == O.INF:
                assert row[j] == -1 or (j == i and row[j] == i)
                continue
            if j == i:
                assert row[j] == i
                continue
            t = row[j]
            assert alive[t] and t != i and E[i, t] + M[t, j] == M[i, j]
            lower = [s for s in range(t) if s != i and alive[s] and E[i, s] < O.INF and M[s, j] < O.INF
                     and E[i, s] + M[s, j] == M[i, j]]
            assert not lower


def test_next_hop_on_a_cycle_is_the_successor():
    n = 9
    W = np.full((n, n), synth.INF_I32, np.int32)
    np.fill_diagonal(W, 0)
    for v in range(n):
        W[v, (v + 1) % n] = 1 + v
    M = O.fw(W)
    alive = np.ones(n, bool)
    for i in range(n):
        row = O.next_hop_row(M, W, alive, i)
        for j in range(n):
            assert row[j] == (i if j == i else (i + 1) % n)


@pytest.mark.parametrize("seed", range(3))
def test_following_next_hops_gives_a_shortest_path(seed):
    n = 40
    W = rand_graph(n, 90 + seed, lo=1, hi=50, p_missing=0.5)
    M = O.fw(W)
    E = O.exact(W)
    alive = np.ones(n, bool)
    NH = np.array([O.next_hop_row(M, W, alive, i) for i in range(n)])
    for i in range(n):
        for j in range(n):
            if M[i, j] == O.INF or i == j:
                continue
            u, L, steps = i, 0, 0
            while u != j:
                t = int(NH[u, j])
                L += int(E[u, t])
                u = t
                steps += 1
                assert steps < n
            assert L == M[i, j]


def test_planted_mistakes_are_caught():
    W = rand_graph(7, 5, lo=1, hi=6, p_missing=0.2)
    M = O.fw(W)
    E = O.exact(W)
    alive = np.ones(7, bool)

    def strict(i):        # "<" instead of "==": never true for an exact D
        out = np.full(7, -1)
        out[i] = i
        for j in range(7):
            for t in range(7):
                if j != i and t != i and E[i, t] < O.INF and M[t, j] < O.INF and E[i, t] + M[t, j] < M[i, j]:
                    out[j] = t
                    break
        return out

    def direct_first(i):  # prefers the direct edge even when it is not shortest
        out = O.next_hop_row(M, W, alive, i).copy()
        for j in range(7):
            if j != i and E[i, j] < O.INF:
                out[j] = j
        return out

    ref = [O.next_hop_row(M, W, alive, i) for i in range(7)]
    assert any(not np.array_equal(strict(i), ref[i]) for i in range(7))
    assert any(not np.array_equal(direct_first(i), ref[i]) for i in range(7))
