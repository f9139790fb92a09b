"""CPU oracle for warm-start APSP after a minor graph update.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this module.  It shares no
code with the CUDA path and never imports the product package.

Everything is exact: integer weights are carried in int64 (a missing edge is
``INF``), float weights in fp64 (a missing edge is +inf).  Matrices are dense
row-major in *slot space*: a dead slot has an all-missing row and column, so
it takes part in no path (the paper removes a node by setting its distances to
and from every other node to infinity, Section 3.2).

What each function follows:

* ``fw``                      Floyd-Warshall, the cold solver the paper compares
                              against (Section 2, Algorithm 5 line "Floyd_Warshall").
* ``dijkstra_rows``           per-source Dijkstra (Algorithm 5).
* ``brute_force_apsp``        the definition of SPD itself (notation table:
                              minimum over loop-free paths), by enumeration.
* ``add_node``                Corollary 1, Corollary 2 and Theorem 3 (Section 3.1).
* ``need_update_list``        Section 3.2 via Theorem 4 / Corollary 3.
* ``cost_of_remove``          Definition (Cost), Eq. (equ:cost_defi).
* ``remove_node_alg5``        Algorithm 5.
* ``modify_edge_alg6``        Algorithm 6.
* ``apsp_after``              the plain definition: the APSP matrix of the
                              updated graph, by ``fw``.
* ``warm_shortest_path``      Algorithm 7 (candidate_node_list, small matrix,
                              Dijkstra on it; Theorem al_correct).
* ``all_shortest_paths_alg8`` Algorithm 8 on Algorithm 7's small graph.
* ``need_update_list_alg12``  Algorithm 12 (Theorem theo_algo12).
* ``key_node_list``,
  ``need_update_list_alg11``  Algorithm 10's key_node_list of one pair with
                              Algorithm 11's shortcut; Algorithm 11.
* ``fw_minimax``, ``add_node_minimax``, ``need_update_list_minimax``
                              the Discussion's minimax (bottleneck) variant.
"""
from __future__ import annotations

import ctypes
import itertools
import os
from typing import Dict, List, Optional, Sequence

import numpy as np

#: Missing edge / unreachable, int64 side.  Equal to ORACLE_INF_I64 in apsp_oracle.c.
INF = 1 << 60
#: Missing edge as stored by int32 callers (two of them fit in int32).
INF_I32 = 0x3FFFFFFF

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None


def _clib():
    """The compiled FW / Dijkstra (built on demand by oracle/build.py)."""
    global _lib
    if _lib is None:
        from . import build as _b
        path = _b.build()
        lib = ctypes.CDLL(path)
        i64, p = ctypes.c_int64, ctypes.c_void_p
        lib.oracle_fw_i64.argtypes = [i64, p]
        lib.oracle_fw_f64.argtypes = [i64, p]
        lib.oracle_dijkstra_rows_i64.argtypes = [i64, p, i64, p, p]
        lib.oracle_dijkstra_rows_f64.argtypes = [i64, p, i64, p, p]
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def num_threads() -> int:
    return int(_clib().oracle_num_threads())


# ---------------------------------------------------------------------------
# Representation helpers (int32 <-> exact int64, float32 <-> fp64)
# ---------------------------------------------------------------------------

def is_float(a: np.ndarray) -> bool:
    return np.issubdtype(a.dtype, np.floating)


def exact(W: np.ndarray, alive: Optional[np.ndarray] = None) -> np.ndarray:
    """Copy of an adjacency matrix in exact arithmetic (int64 or fp64).

    int32 INF_I32 entries (and anything larger) become INF.  Dead slots get
    an all-missing row and column; live diagonals are 0.
    """
    if is_float(W):
        E = np.array(W, dtype=np.float64, copy=True)
        miss = np.inf
    else:
        E = np.array(W, dtype=np.int64, copy=True)
        E[E >= INF_I32] = INF
        miss = INF
    n = E.shape[0]
    if alive is None:
        alive = np.ones(n, dtype=bool)
    alive = np.asarray(alive, dtype=bool)
    E[~alive, :] = miss
    E[:, ~alive] = miss
    idx = np.flatnonzero(alive)
    E[idx, idx] = 0
    return E


def to_i32(D: np.ndarray) -> np.ndarray:
    """Exact int64 distances as the int32 convention (unreachable -> INF_I32)."""
    out = np.minimum(D, INF_I32)
    return out.astype(np.int32)


def missing(D: np.ndarray):
    return np.inf if is_float(D) else INF


# ---------------------------------------------------------------------------
# Cold solvers
# ---------------------------------------------------------------------------

def fw(W: np.ndarray, alive: Optional[np.ndarray] = None) -> np.ndarray:
    """APSP matrix by Floyd-Warshall on the exact copy of W (C, OpenMP over rows)."""
    D = np.ascontiguousarray(exact(W, alive))
    n = D.shape[0]
    if is_float(D):
        _clib().oracle_fw_f64(n, D.ctypes.data)
    else:
        _clib().oracle_fw_i64(n, D.ctypes.data)
    return D


def fw_python(W: np.ndarray, alive: Optional[np.ndarray] = None) -> np.ndarray:
    """Floyd-Warshall with the k-loop in Python and the (i, j) update as one
    numpy expression per k.  Same recurrence as ``fw``; used to cross-check the
    compiled one on small inputs."""
    D = exact(W, alive)
    n = D.shape[0]
    for k in range(n):
        cand = D[:, k:k + 1] + D[k:k + 1, :]
        if not is_float(D):
            cand = np.where((D[:, k:k + 1] >= INF) | (D[k:k + 1, :] >= INF), INF, cand)
        np.minimum(D, cand, out=D)
    return D


def dijkstra_rows(W: np.ndarray, sources: Sequence[int], alive: Optional[np.ndarray] = None) -> np.ndarray:
    """Rows `sources` of the APSP matrix, one dense Dijkstra per source."""
    E = np.ascontiguousarray(exact(W, alive))
    n = E.shape[0]
    src = np.ascontiguousarray(np.asarray(sources, dtype=np.int64))
    out = np.empty((len(src), n), dtype=E.dtype)
    if is_float(E):
        _clib().oracle_dijkstra_rows_f64(n, E.ctypes.data, len(src), src.ctypes.data, out.ctypes.data)
    else:
        _clib().oracle_dijkstra_rows_i64(n, E.ctypes.data, len(src), src.ctypes.data, out.ctypes.data)
    return out


def brute_force_apsp(W: np.ndarray, alive: Optional[np.ndarray] = None) -> np.ndarray:
    """SPD by its definition: the least length over every loop-free path
    (notation table: a path may not repeat a node).  Exponential; n <= 8."""
    E = exact(W, alive)
    n = E.shape[0]
    assert n <= 9, "brute force is exponential"
    miss = missing(E)
    D = np.full((n, n), miss, dtype=E.dtype)
    live = [v for v in range(n) if E[v, v] == 0]
    for s in live:
        D[s, s] = 0
        # depth-first enumeration of every loop-free path starting at s
        stack = [(s, 0, 1 << s)]
        while stack:
            u, length, seen = stack.pop()
            for v in live:
                if seen >> v & 1:
                    continue
                w = E[u, v]
                if w == miss:
                    continue
                L = length + w
                if L < D[s, v]:
                    D[s, v] = L
                stack.append((v, L, seen | (1 << v)))
    return D


# ---------------------------------------------------------------------------
# Adding a node: Corollary 1, Corollary 2, Theorem 3 (Section 3.1)
# ---------------------------------------------------------------------------

def add_node(M: np.ndarray, alive: np.ndarray, p: int, in_w: np.ndarray, out_w: np.ndarray) -> np.ndarray:
    """APSP matrix of G + p from the APSP matrix M of G (slot p dead in M).

    in_w[t] = d(t, p), out_w[t] = d(p, t) for every slot t (dead t ignored).
      Corollary 1: SPD(p, r | G+p) = min_t d(p, t) + SPD(t, r | G)
      Corollary 2: SPD(r, p | G+p) = min_t SPD(r, t | G) + d(t, p)
      Theorem 3:   SPD(i, j | G+p) = min(SPD(i, j | G), SPD(i, p | G+p) + SPD(p, j | G+p))
    """
    alive = np.asarray(alive, dtype=bool)
    assert not alive[p]
    miss = missing(M)
    live = np.flatnonzero(alive)
    wi = np.array(np.asarray(in_w), dtype=M.dtype)
    wo = np.array(np.asarray(out_w), dtype=M.dtype)
    if not is_float(M):
        wi[wi >= INF_I32] = INF
        wo[wo >= INF_I32] = INF
    n = M.shape[0]
    out_row = np.full(n, miss, dtype=M.dtype)   # SPD(p, r | G + p)
    in_col = np.full(n, miss, dtype=M.dtype)    # SPD(r, p | G + p)
    for r in live:
        out_row[r] = _min_sum(wo[live], M[live, r], miss)       # Corollary 1
        in_col[r] = _min_sum(M[r, live], wi[live], miss)        # Corollary 2
    M2 = M.copy()
    for i in live:                                              # Theorem 3
        x2 = _add(in_col[i], out_row[live], miss)
        M2[i, live] = np.minimum(M[i, live], x2)
    M2[p, :] = out_row
    M2[:, p] = in_col
    M2[p, p] = 0
    return M2


def _add(a, b, miss):
    s = a + b
    if miss is not np.inf:
        s = np.where((np.asarray(a) >= INF) | (np.asarray(b) >= INF), INF, s)
    return s


def _min_sum(a: np.ndarray, b: np.ndarray, miss):
    if len(a) == 0:
        return miss
    return np.min(_add(a, b, miss))


# ---------------------------------------------------------------------------
# Removing a node: need_update_list, Cost, Algorithm 5 (Section 3.2)
# ---------------------------------------------------------------------------

def need_update_list(M: np.ndarray, alive: np.ndarray, k: int) -> Dict[int, List[int]]:
    """need_update_list for removing node k (Section 3.2, Theorem 4 / Corollary 3).

    Pair (i, j), i != j, both live and different from k, is listed under node i
    unless SPD(i, j) < SPD(i, k) + SPD(k, j) (strictly less: k is then not needed).
    Unreachable pairs stay unreachable after a removal and are not listed.
    """
    alive = np.asarray(alive, dtype=bool)
    miss = missing(M)
    lst: Dict[int, List[int]] = {}
    rem = [v for v in np.flatnonzero(alive) if v != k]
    for i in rem:
        row = []
        for j in rem:
            if j == i or M[i, j] == miss:
                continue
            t = _add(M[i, k], M[k, j], miss)
            if not (M[i, j] < t):
                row.append(int(j))
        lst[int(i)] = row
    return lst


def cost_of_remove(lst: Dict[int, List[int]], N: int) -> float:
    """Cost C = (number of non-empty items of need_update_list) / (N - 1),
    N the number of nodes of G (Definition, Eq. (equ:cost_defi))."""
    if N <= 1:
        return 0.0
    return sum(1 for v in lst.values() if len(v) > 0) / (N - 1)


def remove_node_alg5(W: np.ndarray, M: np.ndarray, alive: np.ndarray, k: int, delta: float):
    """Algorithm 5, APSP_remove_node(G, M_G, G_k, delta).

    Returns (M', alive', info).  Steps in the algorithm's order: the remaining
    node list, need_update_list, Cost; if Cost > delta the whole matrix of
    G - G_k is recomputed by Floyd-Warshall, else M is copied and, for every
    remaining node i with a non-empty list, one Dijkstra from i on G - G_k
    overwrites the listed entries.
    """
    alive = np.asarray(alive, dtype=bool)
    alive2 = alive.copy()
    alive2[k] = False                                       # remaining_node_list
    lst = need_update_list(M, alive, k)
    N = int(alive.sum())
    cost = cost_of_remove(lst, N)
    if cost > delta:
        return fw(W, alive2), alive2, {"cost": cost, "path": "cold", "list": lst}
    M2 = M.copy()
    miss = missing(M)
    M2[k, :] = miss
    M2[:, k] = miss
    for i in np.flatnonzero(alive2):
        if len(lst[int(i)]) > 0:
            temp = dijkstra_rows(W, [int(i)], alive2)[0]
            for j in lst[int(i)]:
                M2[i, j] = temp[j]
    return M2, alive2, {"cost": cost, "path": "warm", "list": lst}


def modify_edge_alg6(W: np.ndarray, M: np.ndarray, alive: np.ndarray, e: Sequence[int], w, delta: float,
                     undirected: bool = False):
    """Algorithm 6, APSP_modify_edge(G, M_G, e_n, e_w, delta).

    Cost of removing each end node; remove the cheaper one (on a tie, node j,
    as the algorithm's else-branch does) with Algorithm 5; then set the edge
    weight and add the node back by the warm start of Section 3.1.  Returns
    (M', W').
    """
    i, j = int(e[0]), int(e[1])
    cost_i = cost_of_remove(need_update_list(M, alive, i), int(np.sum(alive)))
    cost_j = cost_of_remove(need_update_list(M, alive, j), int(np.sum(alive)))
    k = i if cost_i < cost_j else j
    Mk, alive_k, _ = remove_node_alg5(W, M, alive, k, delta)
    W2 = np.array(W, copy=True)                              # cal_updated_graph
    W2[i, j] = w
    if undirected:
        W2[j, i] = w
    in_w = W2[:, k].copy()
    out_w = W2[k, :].copy()
    M2 = add_node(Mk, alive_k, k, in_w, out_w)
    return M2, W2


# ---------------------------------------------------------------------------
# Plain definitions used as parity targets
# ---------------------------------------------------------------------------

def apsp_after(W: np.ndarray, alive: np.ndarray) -> np.ndarray:
    """The APSP matrix of the (updated) graph: Floyd-Warshall from scratch."""
    return fw(W, alive)


def edge_affected_pairs(M: np.ndarray, alive: np.ndarray, u: int, v: int, w_old, undirected: bool = False):
    """Pairs (i, j), i != j, whose distance may grow when edge (u, v) of weight
    w_old becomes heavier: those with SPD(i, j) = SPD(i, u) + w_old + SPD(v, j)
    (for an undirected graph, also through (v, u)).

    This is Corollary 3's test with the removed node replaced by the edge: a
    pair whose distance is strictly below every path through the edge keeps
    its distance.
    """
    miss = missing(M)
    live = np.flatnonzero(np.asarray(alive, dtype=bool))
    out = set()
    orient = [(u, v)] + ([(v, u)] if undirected else [])
    for (a, b) in orient:
        for i in live:
            for j in live:
                if i == j or M[i, j] == miss:
                    continue
                t = _add(_add(M[i, a], w_old, miss), M[b, j], miss)
                if not (M[i, j] < t):
                    out.add((int(i), int(j)))
    return out


def lowest_free_slot(alive: np.ndarray) -> int:
    """Slot rule for a new node (the paper's G_{n+1}): the lowest dead slot."""
    dead = np.flatnonzero(~np.asarray(alive, dtype=bool))
    return int(dead[0]) if len(dead) else -1


def check_invariants(W: np.ndarray, D: np.ndarray, alive: np.ndarray) -> List[str]:
    """Properties every APSP matrix has; returns the list of violations.

    D[i][i] = 0; D <= W; triangle inequality D[i][j] <= D[i][t] + D[t][j];
    and every finite D[i][j] (i != j) is tight through some first edge:
    exists t != i with W[i][t] + D[t][j] = D[i][j].  (With positive weights
    these equations have only one solution, the APSP matrix.)
    """
    E = exact(W, alive)
    miss = missing(E)
    live = np.flatnonzero(np.asarray(alive, dtype=bool))
    bad = []
    Dl = D[np.ix_(live, live)]
    El = E[np.ix_(live, live)]
    if np.any(np.diag(Dl) != 0):
        bad.append("diagonal")
    if np.any(Dl > El):
        bad.append("D > W")
    for t in range(len(live)):
        s = _add(Dl[:, t:t + 1], Dl[t:t + 1, :], miss)
        if np.any(Dl > s):
            bad.append(f"triangle via {live[t]}")
            break
    for a in range(len(live)):
        for b in range(len(live)):
            if a == b or Dl[a, b] == miss:
                continue
            first = _add(El[a, :], Dl[:, b], miss)
            first[a] = miss
            if not np.any(first == Dl[a, b]):
                bad.append(f"not tight ({live[a]},{live[b]})")
                return bad
    return bad


def itertools_paths_min(W: np.ndarray) -> np.ndarray:
    """Second brute force by permutations (independent of the DFS above): for
    every ordered pair, the minimum over every ordered choice of intermediate
    nodes.  n <= 7."""
    E = exact(W)
    n = E.shape[0]
    miss = missing(E)
    D = np.full((n, n), miss, dtype=E.dtype)
    for s in range(n):
        D[s, s] = 0
        for t in range(n):
            if t == s:
                continue
            others = [v for v in range(n) if v not in (s, t)]
            for r in range(len(others) + 1):
                for mid in itertools.permutations(others, r):
                    path = (s,) + mid + (t,)
                    L = 0
                    ok = True
                    for a, b in zip(path, path[1:]):
                        if E[a, b] == miss:
                            ok = False
                            break
                        L = L + E[a, b]
                    if ok and L < D[s, t]:
                        D[s, t] = L
    return D


# ---------------------------------------------------------------------------
# Warm-start path queries: Algorithm 7, Algorithm 8, Theorem al_correct
# (Section 4); exact removal list: Algorithm 12, Theorem theo_algo12
# ---------------------------------------------------------------------------

#: Relative slack of the float candidate test (the same reading as the float
#: tightness test): extra candidates only enlarge the small graph; a missed
#: one could drop every shortest path from it.
FLOAT_SLACK = 2.0 ** -8


def _on_some_shortest_path(M: np.ndarray, i: int, j: int, t: int) -> bool:
    """Algorithm 7's candidate test: t is kept unless SPD(i, j) < SPD(i, t) + SPD(t, j)."""
    miss = missing(M)
    via = _add(M[i, t], M[t, j], miss)
    if via == miss:
        return False
    if is_float(M):
        return bool(via <= M[i, j] * (1.0 + FLOAT_SLACK))
    return not (M[i, j] < via)


def candidate_node_list(M: np.ndarray, alive: np.ndarray, i: int, j: int) -> List[int]:
    """Algorithm 7's candidate_node_list: i, then every other live node t
    (in increasing slot order) that is on some shortest i -> j path, then j."""
    live = [int(t) for t in np.flatnonzero(np.asarray(alive, dtype=bool))]
    cand = [i]
    for t in live:
        if t == i or t == j:
            continue
        if _on_some_shortest_path(M, i, j, t):
            cand.append(t)
    cand.append(j)
    return cand


def small_dijkstra(A: np.ndarray, s: int):
    """Dense Dijkstra on a small matrix A (A[a][b] = weight a -> b, missing =
    INF / inf) from node s.  Returns (dist, pred); pred[s] = -1 and -1 for
    unreachable nodes.  The next node is the unvisited one of least distance,
    the lowest index on a tie; a node's predecessor changes only on a strict
    improvement."""
    K = A.shape[0]
    miss = missing(A)
    dist = np.full(K, miss, dtype=A.dtype)
    pred = np.full(K, -1, dtype=np.int64)
    done = np.zeros(K, dtype=bool)
    dist[s] = 0
    for _ in range(K):
        best, a = miss, -1
        for b in range(K):
            if not done[b] and dist[b] < best:
                best, a = dist[b], b
        if a < 0:
            break
        done[a] = True
        for b in range(K):
            if done[b] or A[a, b] == miss:
                continue
            nd = dist[a] + A[a, b]
            if nd < dist[b]:
                dist[b] = nd
                pred[b] = a
    return dist, pred


def _tree_path(pred: np.ndarray, s: int, t: int) -> List[int]:
    out = [t]
    while out[-1] != s:
        p = int(pred[out[-1]])
        if p < 0:
            return []
        out.append(p)
    return out[::-1]


def warm_shortest_path(M: np.ndarray, W: np.ndarray, alive: np.ndarray, i: int, j: int) -> List[int]:
    """Algorithm 7, warm_cal_shortest_path(M_G, A_G, i, j).

    In the algorithm's order: [i] when i == j; the candidate_node_list (i, the
    nodes t with not SPD(i, j) < SPD(i, t) + SPD(t, j), then j); the small
    matrix of the adjacency among the candidates; Dijkstra from small node 0
    to small node K - 1; the path translated back to slot ids.  Theorem
    al_correct: the small graph holds every shortest i -> j path.  An
    unreachable pair (the paper is silent) gives the empty list.
    """
    if i == j:
        return [i]
    if M[i, j] == missing(M):
        return []
    cand = candidate_node_list(M, alive, i, j)
    small = exact(np.asarray(W)[np.ix_(cand, cand)])     # small_matrix[a][b] = A_G[cand[a]][cand[b]]
    _, pred = small_dijkstra(small, 0)
    return [cand[a] for a in _tree_path(pred, 0, len(cand) - 1)]


def all_shortest_paths_alg8(M: np.ndarray, W: np.ndarray, alive: np.ndarray, i: int, j: int) -> List[List[int]]:
    """Algorithm 8, warm_cal_all_shortest_paths, on Algorithm 7's small graph.

    One shortest path Psi(i, j) first; then for every candidate t other than
    i and j, a shortest i -> t path joined to a shortest t -> j path (both on
    the small graph), appended unless already listed.  A join that visits a
    node twice (possible only through zero-weight cycles; the paper is
    silent) is a walk, not a path, and is skipped.  Every listed path is a
    shortest i -> j path; the list need not hold every one of them.
    """
    if i == j:
        return [[i]]
    if M[i, j] == missing(M):
        return []
    cand = candidate_node_list(M, alive, i, j)
    small = exact(np.asarray(W)[np.ix_(cand, cand)])
    K = len(cand)
    _, pred_i = small_dijkstra(small, 0)
    _, pred_j = small_dijkstra(np.ascontiguousarray(small.T), K - 1)   # reverse graph: t -> j
    out = [[cand[a] for a in _tree_path(pred_i, 0, K - 1)]]
    for t in range(1, K - 1):
        first = _tree_path(pred_i, 0, t)
        second = _tree_path(pred_j, K - 1, t)[::-1]
        if not first or not second:
            continue
        p = [cand[a] for a in first + second[1:]]
        if len(set(p)) != len(p):      # zero-weight cycles can make the join a walk, not a path
            continue
        if p not in out:
            out.append(p)
    return out


def path_length(W: np.ndarray, path: Sequence[int]):
    """Sum of the edge weights along `path` in exact arithmetic (missing if an edge is missing)."""
    E = exact(W)
    miss = missing(E)
    L = E.dtype.type(0)
    for a, b in zip(path, path[1:]):
        if E[a, b] == miss:
            return miss
        L = L + E[a, b]
    return L


def need_update_list_alg12(M: np.ndarray, W: np.ndarray, alive: np.ndarray, k: int) -> Dict[int, List[int]]:
    """Algorithm 12's need_update_list for removing node k.

    For every ordered pair (i, j) of remaining nodes with SPD(i, j) >= SPD(i, k)
    + SPD(k, j) (Corollary 3's list): the candidate list of Algorithm 7 without
    k, its small matrix, and Dijkstra from i to j on it (Phi_ij); the pair is
    listed iff Phi_ij > SPD(i, j).  By Theorem theo_algo12 these are exactly
    the pairs whose distance grows when k is removed.
    """
    alive = np.asarray(alive, dtype=bool)
    miss = missing(M)
    E = exact(W, alive)
    rem = [int(v) for v in np.flatnonzero(alive) if v != k]
    lst: Dict[int, List[int]] = {}
    for i in rem:
        row = []
        for j in rem:
            if j == i or M[i, j] == miss:
                continue
            if M[i, j] < _add(M[i, k], M[k, j], miss):
                continue
            cand = [i] + [t for t in rem if t not in (i, j) and _on_some_shortest_path(M, i, j, t)] + [j]
            dist, _ = small_dijkstra(E[np.ix_(cand, cand)], 0)
            if dist[len(cand) - 1] > M[i, j]:
                row.append(j)
        lst[i] = row
    return lst


def key_node_list(M: np.ndarray, W: np.ndarray, alive: np.ndarray, i: int, j: int) -> Optional[List[int]]:
    """key_node_list of pair (i, j) (Algorithm 10, steps for one pair, with
    Algorithm 11's shortcut): the nodes common to every path in Algorithm 8's
    path set, without i and j.  Algorithm 11 takes the joins through the
    candidates off Psi(i, j) only (it replaces {i, j} by Psi's nodes in
    Algorithm 8's split), since a join through a node of Psi adds nothing to
    the intersection that Psi does not.  None when j is unreachable.  The path
    set may miss shortest paths, so the list can only be larger than the set
    of truly essential nodes."""
    if i == j or M[i, j] == missing(M):
        return None
    cand = candidate_node_list(M, alive, i, j)
    small = exact(np.asarray(W)[np.ix_(cand, cand)])
    K = len(cand)
    _, pred_i = small_dijkstra(small, 0)
    _, pred_j = small_dijkstra(np.ascontiguousarray(small.T), K - 1)
    psi = _tree_path(pred_i, 0, K - 1)
    on_psi = set(psi)
    common = set(psi)
    for t in range(1, K - 1):
        if t in on_psi:
            continue
        first = _tree_path(pred_i, 0, t)
        second = _tree_path(pred_j, K - 1, t)[::-1]
        if not first or not second:
            continue
        p = first + second[1:]
        if len(set(p)) != len(p):
            continue
        common &= set(p)
    common -= {0, K - 1}
    return sorted(cand[a] for a in common)


def need_update_list_alg11(M: np.ndarray, W: np.ndarray, alive: np.ndarray, k: int) -> Dict[int, List[int]]:
    """Algorithm 11's need_update_list for removing node k: among the pairs
    with SPD(i, j) >= SPD(i, k) + SPD(k, j) (Corollary 3), those whose
    key_node_list holds k."""
    alive = np.asarray(alive, dtype=bool)
    miss = missing(M)
    rem = [int(v) for v in np.flatnonzero(alive) if v != k]
    lst: Dict[int, List[int]] = {}
    for i in rem:
        row = []
        for j in rem:
            if j == i or M[i, j] == miss or M[i, j] < _add(M[i, k], M[k, j], miss):
                continue
            key = key_node_list(M, W, alive, i, j)
            if key is not None and k in key:
                row.append(j)
        lst[i] = row
    return lst


# ---------------------------------------------------------------------------
# Next hops (the optional next-hop output of the hot-path plan)
# ---------------------------------------------------------------------------

def next_hop_row(M: np.ndarray, W: np.ndarray, alive: np.ndarray, i: int) -> np.ndarray:
    """Row i of the next-hop matrix: for every live j != i with SPD(i, j)
    finite, the lowest live t != i such that the edge i -> t followed by a
    shortest t -> j path is a shortest i -> j walk, w(i, t) + SPD(t, j) ==
    SPD(i, j) (fp: within the tightness slack); i for j == i; -1 where j is
    dead or unreachable.  With positive weights this is the lowest first hop
    of a shortest i -> j path."""
    alive = np.asarray(alive, dtype=bool)
    E = exact(W, alive)
    miss = missing(M)
    n = M.shape[0]
    out = np.full(n, -1, dtype=np.int64)
    if not alive[i]:
        return out
    out[i] = i
    for j in np.flatnonzero(alive):
        if j == i or M[i, j] == miss:
            continue
        for t in np.flatnonzero(alive):
            if t == i or E[i, t] == miss or M[t, j] == miss:
                continue
            via = E[i, t] + M[t, j]
            ok = via <= M[i, j] * (1.0 + FLOAT_SLACK) if is_float(M) else via == M[i, j]
            if ok:
                out[j] = t
                break
    return out


# ---------------------------------------------------------------------------
# Minimax (bottleneck) paths: the Discussion's variant.  The value of a path
# is its largest edge weight; SPD becomes the least such value over paths.
# ---------------------------------------------------------------------------

def fw_minimax(W: np.ndarray, alive: Optional[np.ndarray] = None) -> np.ndarray:
    """Minimax distance matrix by Floyd-Warshall in the (min, max) semiring:
    D[i][j] = min(D[i][j], max(D[i][k], D[k][j])) for k in order."""
    D = exact(W, alive)
    n = D.shape[0]
    for k in range(n):
        D = np.minimum(D, np.maximum(D[:, k:k + 1], D[k:k + 1, :]))
    return D


def brute_force_minimax(W: np.ndarray, alive: Optional[np.ndarray] = None) -> np.ndarray:
    """Minimax distances by their definition: the least largest edge over every
    loop-free path (n <= 8)."""
    E = exact(W, alive)
    n = E.shape[0]
    assert n <= 9, "brute force is exponential"
    miss = missing(E)
    D = np.full((n, n), miss, dtype=E.dtype)
    live = [v for v in range(n) if E[v, v] == 0]
    for s in live:
        D[s, s] = 0
        stack = [(s, E.dtype.type(0), 1 << s)]
        while stack:
            u, worst, seen = stack.pop()
            for v in live:
                if seen >> v & 1 or E[u, v] == miss:
                    continue
                b = max(worst, E[u, v])
                if b < D[s, v]:
                    D[s, v] = b
                stack.append((v, b, seen | (1 << v)))
    return D


def add_node_minimax(M: np.ndarray, alive: np.ndarray, p: int, in_w: np.ndarray, out_w: np.ndarray) -> np.ndarray:
    """Section 3.1 in the (min, max) semiring: Corollaries 1 and 2 with max in
    place of +, then Theorem 3's min(M[i][j], max(in[i], out[j]))."""
    alive = np.asarray(alive, dtype=bool)
    assert not alive[p]
    miss = missing(M)
    live = np.flatnonzero(alive)
    wi = np.array(np.asarray(in_w), dtype=M.dtype)
    wo = np.array(np.asarray(out_w), dtype=M.dtype)
    if not is_float(M):
        wi[wi >= INF_I32] = INF
        wo[wo >= INF_I32] = INF
    n = M.shape[0]
    out_row = np.full(n, miss, dtype=M.dtype)
    in_col = np.full(n, miss, dtype=M.dtype)
    for r in live:
        if len(live):
            out_row[r] = np.min(np.maximum(wo[live], M[live, r]))
            in_col[r] = np.min(np.maximum(M[r, live], wi[live]))
    M2 = M.copy()
    for i in live:
        M2[i, live] = np.minimum(M[i, live], np.maximum(in_col[i], out_row[live]))
    M2[p, :] = out_row
    M2[:, p] = in_col
    M2[p, p] = 0
    return M2


def need_update_list_minimax(M: np.ndarray, alive: np.ndarray, k: int) -> Dict[int, List[int]]:
    """Corollary 3's test for removing k in the (min, max) semiring: (i, j) is
    listed unless SPD(i, j) < max(SPD(i, k), SPD(k, j))."""
    alive = np.asarray(alive, dtype=bool)
    miss = missing(M)
    rem = [int(v) for v in np.flatnonzero(alive) if v != k]
    lst: Dict[int, List[int]] = {}
    for i in rem:
        lst[i] = [j for j in rem if j != i and M[i, j] != miss and not (M[i, j] < max(M[i, k], M[k, j]))]
    return lst
