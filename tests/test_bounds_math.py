"""The two pruning tests the device applies, checked against the oracle.

1. Node insertion reads only the rows t with w(p, t) <= w(p, t0) + E0
   (t0 the lightest out-edge of p, E0 = max over live j of D[t0][j]), and
   likewise only the columns r with w(r, p) <= w(r1, p) + E1 (Section 3.1,
   Corollaries 1 and 2).  The minima over those rows and columns must equal
   the oracle's insertion exactly, including the case where a live node is
   unreachable (the bound is then infinite and every row stays).
2. The later re-relaxation passes skip y for pair j when
   dy - ly[y] >= cur - ly[j] or dy + lx[y] >= cur + lx[j], with ly, lx the old
   row and column of the removed node (D[v][.] and D[.][u] for an increase of
   u -> v).  A skipped y must give no candidate below cur: dy + D[y][j] >= cur
   for every value D[y][j] can hold during the repair, which is at least the
   old distance.

These run on the CPU and use only the oracle and numpy.
"""
import numpy as np
import pytest

import synth
from oracle import apsp as O


def _graph(n, seed, kind):
    if kind == "float":
        return synth.lognormal_digraph_f32(n, seed)
    W = synth.complete_digraph_i32(n, 1, 1000, seed)
    if kind == "missing":
        m = synth.uniform_f64(seed, 77, n * n).reshape(n, n) < 0.6
        np.fill_diagonal(m, False)
        W = W.copy()
        W[m] = synth.INF_I32
    if kind == "unreachable":
        W = W.copy()
        W[:, 5] = synth.INF_I32   # nothing reaches node 5
        W[5, 5] = 0
    if kind == "undirected":
        W = np.minimum(W, W.T)
    return W


def _restricted_insertion(M, alive, w_in, w_out):
    """Corollaries 1 and 2 over the candidate rows / columns only; returns
    (out over live columns, in over live rows, number of candidates)."""
    miss = O.missing(M)
    live = np.flatnonzero(alive)
    res = []
    count = 0
    for w, rows_of in ((w_out, lambda t: M[t, live]), (w_in, lambda t: M[live, t])):
        wl = w[live]
        fin = wl < miss
        best = np.full(len(live), miss, dtype=M.dtype)
        if fin.any():
            t0 = live[np.argmin(np.where(fin, wl, miss))]
            e = rows_of(t0).max()
            keep = fin & (wl <= (miss if e >= miss else w[t0] + e))
            for t in live[keep]:
                best = np.minimum(best, O._add(w[t], rows_of(t), miss))
            count += int(keep.sum())
        res.append(best)
    return res[0], res[1], count


@pytest.mark.parametrize("kind", ["int", "missing", "unreachable", "undirected", "float"])
@pytest.mark.parametrize("wide", [True, False])
def test_insertion_candidates_give_the_exact_new_row_and_column(kind, wide):
    n, cap = 90, 96
    W = _graph(n, 11, kind)
    alive = np.zeros(cap, bool)
    alive[:n] = True
    Wc = np.full((cap, cap), np.inf if kind == "float" else synth.INF_I32, dtype=W.dtype)
    Wc[:n, :n] = W
    M = O.fw(Wc, alive)
    hi = 10 ** 6 if wide else 30
    for t in range(3):
        w_out = synth.uniform_int(12, 2 * t, cap, 1, hi).astype(np.int64)
        w_in = w_out.copy() if kind == "undirected" else synth.uniform_int(12, 2 * t + 1, cap, 1, hi).astype(np.int64)
        if kind == "float":
            w_out, w_in = w_out.astype(np.float64) * 0.37, w_in.astype(np.float64) * 0.37
        p = n + t
        ref = O.add_node(M, alive, p, w_in, w_out)
        live = np.flatnonzero(alive)
        out_c, in_c, count = _restricted_insertion(M, alive, w_in, w_out)
        assert np.array_equal(ref[p, live], out_c), (kind, wide, t)
        assert np.array_equal(ref[live, p], in_c), (kind, wide, t)
        if kind == "unreachable" and t == 0:
            # nothing reaches node 5 yet (the first new node gives it an
            # in-edge), so max_j D[t0][j] is infinite and Corollary 1 keeps
            # every row (Corollary 2's bound stays finite)
            assert count >= len(live)
        elif wide and kind not in ("float", "unreachable"):
            assert count <= len(live) // 4, count   # the bound is selective
        M = ref
        alive[p] = True


@pytest.mark.parametrize("update", ["removal", "increase", "undirected_removal"])
def test_skipped_gathers_cannot_lower_a_pair(update):
    n = 70
    W = synth.complete_digraph_i32(n, 1, 60, 23).astype(np.int64)
    if update == "undirected_removal":
        W = np.minimum(W, W.T)
    D = O.fw(W)
    rng = np.random.default_rng(5)
    checked = skipped = 0
    for case in range(6):
        if update == "increase":
            u = int(rng.integers(n))
            v = int(np.argmin(np.where(np.arange(n) == u, 10 ** 9, W[u])))   # a tight edge
            ly, lx = D[v, :], D[:, u]
            W2 = W.copy()
            W2[u, v] = W[u, v] * 4
            D2 = O.fw(W2)
            listed = D[:, u][:, None] + W[u, v] + D[v, :][None, :] == D
            listed &= D2 > D - 1   # pairs through the edge (all of them may change)
            rows = range(n)
        else:
            k = int(rng.integers(n))
            ly, lx = D[k, :], D[:, k]
            alive = np.ones(n, bool)
            alive[k] = False
            D2 = O.fw(W, alive)
            lst = O.need_update_list(D, np.ones(n, bool), k)
            listed = np.zeros((n, n), bool)
            for i, js in lst.items():
                listed[i, js] = True
            rows = lst.keys()
        for i in rows:
            J = np.flatnonzero(listed[i])
            if len(J) < 2:
                continue
            for j in J:
                # cur: any value pair (i, j) can hold (at least its new distance)
                for cur in (D2[i, j], D2[i, j] + rng.integers(0, 40)):
                    for y in J:
                        if y == j:
                            continue
                        dy = D2[i, y] + rng.integers(0, 40)
                        keep = dy - ly[y] < cur - ly[j] and dy + lx[y] < cur + lx[j]
                        checked += 1
                        if not keep:
                            skipped += 1
                            # the smallest value D[y][j] can hold during the repair
                            assert dy + D[y, j] >= cur, (update, case, i, j, y)
    assert checked > 0 and skipped > 0
