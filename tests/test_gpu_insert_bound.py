"""Node insertion with the candidate bound of the reductions (Section 3.1,
Corollaries 1 and 2).

Only rows t with w(p, t) <= w(p, t0) + max_j D[t0][j] (t0 the lightest out-edge
of p) can attain a minimum of Corollary 1, and likewise the columns of
Corollary 2.  The device reads only those rows when the bound leaves few of
them (stats "reduce_rows" >= 0) and every row otherwise (-1).  Either way
every entry must equal the oracle's Floyd-Warshall of the mirrored weights:
bit-exact for int32, within 1e-5 relative for fp32.
"""
import numpy as np
import pytest

import synth
from oracle import apsp as O

pytestmark = pytest.mark.gpu

F32_RTOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2412_15122_gb300 import build
    build.build()


class _Mirror:
    def __init__(self, W, cap):
        n = W.shape[0]
        self.fp = W.dtype == np.float32
        self.inf = np.float32(np.inf) if self.fp else np.int32(synth.INF_I32)
        self.W = np.full((cap, cap), self.inf, dtype=W.dtype)
        self.W[:n, :n] = W
        self.alive = np.zeros(cap, bool)
        self.alive[:n] = True

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


def _check(g, mir, tag):
    D = g.D()
    m = D.shape[0]
    ref = O.fw(mir.W[:m, :m], mir.alive[:m])
    if mir.fp:
        Df = D.astype(np.float64)
        assert np.array_equal(np.isinf(Df), np.isinf(ref)), tag
        fin = np.isfinite(ref)
        assert (np.abs(Df[fin] - ref[fin]) <= F32_RTOL * np.abs(ref[fin]) + 1e-30).all(), tag
    else:
        exp = O.to_i32(ref)
        bad = np.argwhere(D != exp)
        assert len(bad) == 0, f"{tag}: {len(bad)} entries differ, first {bad[0]}"


def _vec(seed, stream, cap, lo, hi, fp=False):
    if fp:
        return (synth.uniform_f64(seed, stream, cap) * (hi - lo) + lo).astype(np.float32)
    return synth.uniform_int(seed, stream, cap, lo, hi).astype(np.int32)


def _insert(g, mir, iw, ow):
    p = g.add_node(iw, ow)
    assert p == mir.add(iw, ow)
    return g.stats()["reduce_rows"]


@pytest.mark.parametrize("fp", [False, True])
def test_wide_new_weights_read_only_candidates(fp):
    # Graph weights in [1, 1000] (distances far below 1e6), new node weights
    # in [1, 1e6]: a handful of candidates.  Several insertions with a removal
    # in between (slot reuse), each checked in full.
    from paper_2412_15122_gb300 import Graph
    n, cap = 600, 640
    W = synth.complete_digraph_i32(n, 1, 1000, 31)
    if fp:
        W = W.astype(np.float32) * np.float32(0.37)
    g, mir = Graph(W, cap), _Mirror(W, cap)
    seen = []
    for t in range(6):
        if t == 3:
            g.remove_node(17)
            mir.remove(17)
        iw = _vec(31, 100 + 2 * t, cap, 1, 10**6, fp)
        ow = _vec(31, 101 + 2 * t, cap, 1, 10**6, fp)
        rr = _insert(g, mir, iw, ow)
        seen.append(rr)
        _check(g, mir, f"insert {t}")
    assert all(0 < r <= cap // 8 for r in seen), seen
    g.close()


def test_narrow_weights_fall_back_to_the_full_pass():
    # New node weights as light as the graph's own: the bound keeps more than
    # an eighth of the rows, so the full pass runs.
    from paper_2412_15122_gb300 import Graph
    n, cap = 400, 416
    W = synth.complete_digraph_i32(n, 1, 1000, 5)
    g, mir = Graph(W, cap), _Mirror(W, cap)
    rr = _insert(g, mir, _vec(5, 1, cap, 1, 20), _vec(5, 2, cap, 1, 20))
    assert rr == -1
    _check(g, mir, "full pass")
    g.close()


def test_unreachable_node_makes_the_bound_infinite():
    # A live node with no in-edges is unreachable from every other node, so
    # max_j D[t0][j] is infinite and no row may be dropped.
    from paper_2412_15122_gb300 import Graph
    n, cap = 300, 320
    W = synth.complete_digraph_i32(n, 1, 1000, 8)
    W[:, 42] = synth.INF_I32
    W[42, 42] = 0
    g, mir = Graph(W, cap), _Mirror(W, cap)
    iw, ow = _vec(8, 1, cap, 1, 10**6), _vec(8, 2, cap, 1, 10**6)
    rr = _insert(g, mir, iw, ow)
    assert rr == -1
    _check(g, mir, "unreachable node")
    g.close()


def test_undirected_and_one_sided_insertions():
    from paper_2412_15122_gb300 import Graph
    n, cap = 500, 520
    W = synth.complete_digraph_i32(n, 1, 1000, 12)
    W = np.minimum(W, W.T)
    g, mir = Graph(W, cap, undirected=True), _Mirror(W, cap)
    w = _vec(12, 1, cap, 1, 10**6)
    rr = _insert(g, mir, w, w)
    assert 0 < rr <= cap // 8
    _check(g, mir, "undirected")
    g.close()
    # directed: out-edges only, in-edges only, no edges at all
    W = synth.complete_digraph_i32(n, 1, 1000, 13)
    g, mir = Graph(W, cap), _Mirror(W, cap)
    none = np.full(cap, synth.INF_I32, np.int32)
    for t, (iw, ow) in enumerate([(none, _vec(13, 1, cap, 1, 10**6)), (_vec(13, 2, cap, 1, 10**6), none),
                                  (none, none)]):
        rr = _insert(g, mir, iw, ow)
        assert 0 <= rr <= cap // 8
        _check(g, mir, f"one-sided {t}")
    g.close()


def test_weights_exactly_at_the_bound_are_kept():
    # Several out-edges (in-edges) weigh exactly w(p, t0) + max_j D[t0][j]:
    # they can tie the minimum and must stay candidates (the result is checked
    # in full; ties change no value either way, so this pins the comparison).
    from paper_2412_15122_gb300 import Graph
    n, cap = 300, 320
    W = synth.complete_digraph_i32(n, 1, 1000, 21)
    D = O.to_i32(O.fw(W))
    ow = _vec(21, 1, cap, 5000, 10**6)
    iw = _vec(21, 2, cap, 5000, 10**6)
    ow[7], iw[9] = 3, 4
    e0 = int(D[7].max())
    e1 = int(D[:, 9].max())
    ow[[11, 50, 299]] = 3 + e0
    iw[[12, 60, 298]] = 4 + e1
    g, mir = Graph(W, cap), _Mirror(W, cap)
    rr = _insert(g, mir, iw, ow)
    assert rr >= 8
    _check(g, mir, "ties at the bound")
    g.close()
