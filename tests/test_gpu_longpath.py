"""Parity on graphs whose shortest paths have hundreds of edges.

A directed cycle with lognormal(0, 1) weights plus one heavy chord per 20
nodes: shortest paths follow the cycle for 100-800 edges before a chord pays.
Removing a node or raising a tight cycle edge in the middle of such paths
affects pairs whose fp32 distances are sums of hundreds of rounded terms, the
case where the fp32 tightness slack (2^-8 relative) must still catch every
affected pair.  fp32 results are compared with the fp64 oracle at 1e-5
relative; the same graphs with integer weights are compared bit for bit.

fp32 error bound: a distance over h edges is a sum of h non-negative terms,
so it is within (h - 1) * 2^-24 relative of the exact value; that is <= 1e-5
for h <= 168 edges, the range over which the 1e-5 contract is guaranteed.
`test_path_of_168_edges` checks a graph at that boundary.
"""
import numpy as np
import pytest

import synth
from oracle import apsp as O

pytestmark = pytest.mark.gpu

RTOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2412_15122_gb300 import build
    build.build()


def cycle_with_chords(n, seed, fp, every=20, factor=300.0):
    w = np.exp(synth.normal_f64(seed, 1, n))
    m = n // every
    a = synth.uniform_int(seed, 2, m, 0, n - 1)
    b = synth.uniform_int(seed, 3, m, 0, n - 1)
    cw = np.exp(synth.normal_f64(seed, 4, m)) * factor
    if fp:
        W = np.full((n, n), np.inf, np.float32)
        w, cw = w.astype(np.float32), cw.astype(np.float32)
    else:
        W = np.full((n, n), synth.INF_I32, np.int32)
        w, cw = np.rint(w * 100).astype(np.int32), np.rint(cw * 100).astype(np.int32)
    np.fill_diagonal(W, 0)
    W[np.arange(n), (np.arange(n) + 1) % n] = w
    for x, y, c in zip(a, b, cw):
        if x != y and (x + 1) % n != y:
            W[x, y] = min(W[x, y], c)
    return W


def hop_counts(W, D, s):
    """Edges on a shortest path from s to every node (fewest among ties)."""
    E = O.exact(W)
    d = D[s]
    h = np.full(len(d), -1)
    h[s] = 0
    for v in np.argsort(d, kind="stable"):
        if v == s or not np.isfinite(d[v]):
            continue
        ok = np.isfinite(E[:, v]) & (np.arange(len(d)) != v) & (h >= 0)
        tight = ok & (np.abs(d + E[:, v] - d[v]) <= 1e-9 * max(1.0, d[v]))
        h[v] = int(h[tight].min()) + 1
    return h


def check(g, Wm, alive, fp, tag):
    D = g.D()
    m = D.shape[0]
    live = np.flatnonzero(alive[:m])
    ref = O.fw(Wm[:m, :m], alive[:m])[np.ix_(live, live)]
    got = D[np.ix_(live, live)]
    if fp:
        fin = np.isfinite(ref)
        assert np.array_equal(np.isfinite(got), fin), tag
        rel = np.abs(got[fin].astype(np.float64) - ref[fin]) / np.maximum(ref[fin], 1e-30)
        assert rel.max() <= RTOL, f"{tag}: max rel err {rel.max():.3g}"
    else:
        np.testing.assert_array_equal(got, O.to_i32(ref), err_msg=tag)


@pytest.mark.parametrize("fp", [True, False])
def test_long_paths_removals_and_tight_increases(fp):
    from paper_2412_15122_gb300 import Graph
    n, cap = 1500, 1536
    W = cycle_with_chords(n, 5, fp)
    h = hop_counts(W, O.fw(W), 0)
    assert h.max() >= 300 and np.median(h) >= 100, (h.max(), np.median(h))
    g = Graph(W, cap)
    g.set_dispatch("warm")
    inf = np.float32(np.inf) if fp else np.int32(synth.INF_I32)
    Wm = np.full((cap, cap), inf, W.dtype)
    Wm[:n, :n] = W
    alive = np.zeros(cap, bool)
    alive[:n] = True
    picks = synth.uniform_int(5, 9, 12, 0, n - 1)
    for t, x in enumerate(picks):
        x = int(x)
        while not alive[x]:
            x = (x + 1) % n
        if t % 2 == 0:
            g.remove_node(x)
            alive[x] = False
            Wm[x, :] = Wm[:, x] = inf
            tag = f"remove {x}"
        else:
            y = (x + 1) % n                        # the cycle edge out of x
            while not alive[y]:
                y = (y + 1) % n
            if Wm[x, y] == inf:
                continue
            w = Wm[x, y] * 4
            g.update_edge(x, y, w)
            Wm[x, y] = w
            tag = f"increase ({x},{y})"
        st = g.stats()
        assert st["path"] in ("warm", "trivial"), tag
        check(g, Wm, alive, fp, tag)
    g.close()


def test_path_of_168_edges():
    # A directed path of 168 edges (the longest for which (h - 1) * 2^-24 <=
    # 1e-5) plus heavy back edges, fp32: removals and increases along it stay
    # within 1e-5 of the fp64 oracle.
    from paper_2412_15122_gb300 import Graph
    n, cap = 169, 176
    w = np.exp(synth.normal_f64(17, 1, n)).astype(np.float32)
    W = np.full((n, n), np.inf, np.float32)
    np.fill_diagonal(W, 0)
    W[np.arange(n - 1), np.arange(1, n)] = w[:-1]
    W[np.arange(1, n), np.arange(n - 1)] = (w[1:] * 50).astype(np.float32)
    D0 = O.fw(W)
    assert hop_counts(W, D0, 0)[n - 1] == 168
    g = Graph(W, cap)
    Wm = np.full((cap, cap), np.inf, np.float32)
    Wm[:n, :n] = W
    alive = np.zeros(cap, bool)
    alive[:n] = True
    check(g, Wm, alive, True, "init")
    for x in (40, 120):
        g.update_edge(x, x + 1, Wm[x, x + 1] * 4)
        Wm[x, x + 1] *= 4
        check(g, Wm, alive, True, f"increase ({x},{x + 1})")
    g.remove_node(84)
    alive[84] = False
    Wm[84, :] = Wm[:, 84] = np.inf
    check(g, Wm, alive, True, "remove 84")
    g.close()
