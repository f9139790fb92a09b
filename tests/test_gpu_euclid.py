"""Parity on the learned-dispatch workload's graphs: undirected complete
Euclidean graphs (points uniform in the unit square, weight = round(1e4 *
distance), int32).  Rounded distances make ties between multi-hop routes
common, which is where Corollary 3's list, the tightness tests and the
re-relaxation are stressed hardest (Section 3.2).

The update mix is 10 % node additions (a new uniform point), 40 % removals,
10 % halved and 40 % x4 edges, each edge the lightest out-edge of a node (a
tight edge, so increases are never trivial).
"""
import numpy as np
import pytest

import synth
from oracle import apsp as O

pytestmark = pytest.mark.gpu

MIX = (0.1, 0.4, 0.1, 0.4)   # add, remove, decrease, increase


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2412_15122_gb300 import build
    build.build()


class _Euclid:
    """The graph on the device and the test's own copy of weights and points."""

    def __init__(self, n, cap, seed):
        from paper_2412_15122_gb300 import Graph
        W, pts = synth.euclidean_undirected_i32(n, seed)
        self.g = Graph(W, cap, undirected=True)
        self.W = np.full((cap, cap), synth.INF_I32, np.int32)
        self.W[:n, :n] = W
        self.alive = np.zeros(cap, bool)
        self.alive[:n] = True
        self.pts = np.zeros((cap, 2))
        self.pts[:n] = pts
        self.touched = set()

    def apply(self, up, seed, t):
        live = np.flatnonzero(self.alive)
        if up.kind == synth.ADD:
            cap = len(self.alive)
            w, pnt = synth.new_point_weights_i32(self.pts[live], seed, 5000 + t)
            vec = np.full(cap, synth.INF_I32, np.int32)
            vec[live] = w
            p = self.g.add_node(vec, vec)
            assert p == O.lowest_free_slot(self.alive)
            self.pts[p] = pnt
            self.W[:, p] = vec
            self.W[p, :] = vec
            self.W[p, p] = 0
            self.alive[p] = True
            self.touched.add(p)
            return f"add {p}"
        if up.kind == synth.REMOVE:
            k = int(live[up.a])
            self.g.remove_node(k)
            self.alive[k] = False
            self.W[k, :] = self.W[:, k] = synth.INF_I32
            return f"remove {k}"
        u = int(live[up.a])
        row = np.where(self.alive, self.W[u].astype(np.int64), synth.INF_I32)
        row[u] = synth.INF_I32
        v = int(np.argmin(row))                    # lightest out-edge: always tight
        w0 = int(self.W[u, v])
        w = w0 // 2 if up.kind == synth.DECREASE else max(1, w0) * 4
        self.g.update_edge(u, v, w)
        self.W[u, v] = self.W[v, u] = w
        self.touched.update((u, v))
        return f"{up.kind} ({u},{v}) {w0}->{w}"

    def check_full(self, tag):
        D = self.g.D()
        m = D.shape[0]
        live = np.flatnonzero(self.alive[:m])
        ref = O.to_i32(O.fw(self.W[:m, :m], self.alive[:m]))
        got = D[np.ix_(live, live)]
        exp = ref[np.ix_(live, live)]
        if not np.array_equal(got, exp):
            i, j = np.argwhere(got != exp)[0]
            raise AssertionError(f"{tag}: {int((got != exp).sum())} entries differ, first ({live[i]},{live[j]}) "
                                 f"got {got[i, j]} expected {exp[i, j]}")

    def check_rows(self, rows, tag):
        D = self.g.D()
        m = D.shape[0]
        live = np.flatnonzero(self.alive[:m])
        ref = O.to_i32(O.dijkstra_rows(self.W[:m, :m], rows, self.alive[:m]))
        np.testing.assert_array_equal(D[np.ix_(rows, live)], ref[:, live], err_msg=tag)


@pytest.mark.parametrize("dispatch", ["warm", "cold"])
def test_euclidean_n1024_mixed_updates_full_matrix(dispatch):
    n, cap, seed = 1024, 1024 + 32, 3
    e = _Euclid(n, cap, seed)
    e.g.set_dispatch(dispatch)
    ups = synth.mixed_updates(n, 40 if dispatch == "warm" else 12, seed, fractions=MIX, tight=True,
                              capacity=cap, stream=90)
    kinds = set()
    for t, up in enumerate(ups):
        tag = e.apply(up, seed, t)
        st = e.g.stats()
        kinds.add(st["op"])
        if st["op"] in ("remove", "increase") and dispatch == "warm":
            assert st["path"] in ("warm", "trivial")
        e.check_full(f"step {t}: {tag}")
    assert {"remove", "increase"} <= kinds
    e.g.close()


def test_euclidean_n16384_sampled_rows():
    # The learned-dispatch workload's graph at full size: 20 updates, then 64
    # sampled source rows plus every row an update touched, by Dijkstra.
    n, cap, seed = 16384, 16384 + 64, 3
    e = _Euclid(n, cap, seed)
    ups = synth.mixed_updates(n, 20, seed, fractions=MIX, tight=True, capacity=cap, stream=91)
    warm = 0
    for t, up in enumerate(ups):
        e.apply(up, seed, t)
        st = e.g.stats()
        warm += st["path"] == "warm"
    assert warm >= 5
    live = np.flatnonzero(e.alive)
    pick = live[synth.uniform_int(seed, 11, 64, 0, len(live) - 1)]
    rows = np.unique(np.concatenate([pick, [r for r in e.touched if e.alive[r]]])).astype(np.int64)
    e.check_rows(rows, "n=16384 Euclidean")
    e.g.close()
