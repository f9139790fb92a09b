"""The host's copy of the weights behind edge updates.

An edge update reads the old weight W[u][v] on the host to choose the
increase or the decrease path.  The library keeps that copy without column
writes and fills in device-input adds lazily (a ring of 8 pending adds), so a
stream of device-input adds, removals that free and reuse their slots, and
edge updates on the added nodes must still see the right weights.  Every
update's effect is checked through D against the oracle's Floyd-Warshall of
the test's own weight mirror.
"""
import numpy as np
import pytest

import synth
from oracle import apsp as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2412_15122_gb300 import build
    build.build()


@pytest.mark.parametrize("undirected", [False, True])
def test_device_adds_removals_and_edges_interleaved(undirected):
    import torch
    from paper_2412_15122_gb300 import Graph
    n, cap = 96, 128
    W = synth.complete_digraph_i32(n, 1, 200, 40)
    if undirected:
        W = np.minimum(W, W.T)
    g = Graph(W, cap, undirected=undirected)
    M = np.full((cap, cap), synth.INF_I32, np.int32)
    M[:n, :n] = W
    alive = np.zeros(cap, bool)
    alive[:n] = True
    added = []
    for t in range(30):
        # a device-input add (the ring holds 8 pending ones)
        iw = synth.uniform_int(40, 100 + 2 * t, cap, 1, 200).astype(np.int32)
        ow = iw.copy() if undirected else synth.uniform_int(40, 101 + 2 * t, cap, 1, 200).astype(np.int32)
        p = g.add_node(torch.from_numpy(iw).cuda(), torch.from_numpy(ow).cuda())
        assert p == O.lowest_free_slot(alive)
        live = alive.copy()
        M[:, p] = np.where(live, iw, synth.INF_I32)
        M[p, :] = np.where(live, ow, synth.INF_I32)
        M[p, p] = 0
        alive[p] = True
        added.append(p)
        if t % 3 == 1:
            # remove a node added a few steps ago: its slot is reused by a later add
            k = added.pop(0)
            g.remove_node(k)
            alive[k] = False
            M[k, :] = synth.INF_I32
            M[:, k] = synth.INF_I32
        if t % 2 == 0 and added:
            # an increase and a decrease touching the newest node
            u = added[-1]
            v = int(np.flatnonzero(alive & (np.arange(cap) != u))[t % 7])
            for (a, b), f in (((u, v), 4), ((v, u), 0.5)):
                w = max(1, int(M[a, b] * f))
                g.update_edge(a, b, w)
                M[a, b] = w
                if undirected:
                    M[b, a] = w
        D = g.D()
        m = D.shape[0]
        ref = O.to_i32(O.fw(M[:m, :m], alive[:m]))
        assert np.array_equal(D, ref), f"step {t}"
    g.close()
