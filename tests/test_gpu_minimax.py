"""Minimax (bottleneck) distances on the device (APSP_MINIMAX), the variant of
the paper's Discussion: a path's value is its largest edge weight.

Every result is compared with the oracle's plain definition,
oracle.fw_minimax on the test's own copy of the weights (itself pinned by
brute force and the minimum-spanning-tree bottleneck property); insertions
also with oracle.add_node_minimax and removal lists pair by pair with
oracle.need_update_list_minimax.  max and min are exact, so int32 and fp32
results are both compared for equality.
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


def make(n, seed, fp=False, undirected=False, hi=20, p_missing=0.0):
    if fp:
        W = synth.lognormal_digraph_f32(n, seed)
    else:
        W = synth.complete_digraph_i32(n, 0, hi, seed)
    if p_missing > 0:
        m = synth.uniform_f64(seed, 77, n * n).reshape(n, n) < p_missing
        np.fill_diagonal(m, False)
        W = W.copy()
        W[m] = np.inf if fp else synth.INF_I32
    if undirected:
        W = np.minimum(W, W.T)
    return W


class Mirror:
    def __init__(self, W, cap, und):
        n = W.shape[0]
        self.fp = W.dtype == np.float32
        self.inf = np.float32(np.inf) if self.fp else np.int32(synth.INF_I32)
        self.W = np.full((cap, cap), self.inf, W.dtype)
        self.W[:n, :n] = W
        self.alive = np.zeros(cap, bool)
        self.alive[:n] = True
        self.und = und

    def expected(self, m):
        return O.fw_minimax(self.W[:m, :m], self.alive[:m])


def check(g, mir, tag):
    D = g.D()
    m = D.shape[0]
    ref = mir.expected(m)
    live = np.flatnonzero(mir.alive[:m])
    got = D[np.ix_(live, live)]
    exp = ref[np.ix_(live, live)]
    exp = exp.astype(np.float32) if mir.fp else O.to_i32(exp)
    if not np.array_equal(got, exp):
        bad = np.argwhere(got != exp)
        i, j = bad[0]
        raise AssertionError(f"{tag}: {len(bad)} entries differ, first ({live[i]},{live[j]}) got {got[i, j]} "
                             f"expected {exp[i, j]}")


def G(W, cap, und):
    from paper_2412_15122_gb300 import Graph
    return Graph(W, cap, undirected=und, minimax=True)


@pytest.mark.parametrize("n", [1, 2, 31, 130, 257])
@pytest.mark.parametrize("fp", [False, True])
@pytest.mark.parametrize("und", [False, True])
def test_minimax_floyd_warshall_matches_oracle(n, fp, und):
    W = make(n, 500 + n, fp=fp, undirected=und, p_missing=0.3)
    g = G(W, n + 3, und)
    check(g, Mirror(W, n + 3, und), "init")
    g.close()


@pytest.mark.parametrize("fp", [False, True])
def test_minimax_insertion_matches_oracle(fp):
    n, cap = 90, 96
    W = make(n, 7, fp=fp, p_missing=0.2)
    g = G(W, cap, False)
    mir = Mirror(W, cap, False)
    for t in range(3):
        live = mir.alive.copy()
        M = mir.expected(cap)
        if fp:
            iw = np.exp(synth.normal_f64(7, 10 + t, cap)).astype(np.float32)
            ow = np.exp(synth.normal_f64(7, 20 + t, cap)).astype(np.float32)
        else:
            iw = synth.uniform_int(7, 10 + t, cap, 0, 20).astype(np.int32)
            ow = synth.uniform_int(7, 20 + t, cap, 0, 20).astype(np.int32)
        p = g.add_node(iw, ow)
        assert p == O.lowest_free_slot(mir.alive)
        want = O.add_node_minimax(M, live, p, np.where(live, iw, mir.inf), np.where(live, ow, mir.inf))
        mir.W[:, p] = np.where(live, iw, mir.inf)
        mir.W[p, :] = np.where(live, ow, mir.inf)
        mir.W[p, p] = 0
        mir.alive[p] = True
        D = g.D()
        m = D.shape[0]
        lv = np.flatnonzero(mir.alive[:m])
        w = want[:m, :m][np.ix_(lv, lv)]
        w = w.astype(np.float32) if fp else O.to_i32(w)
        assert np.array_equal(D[np.ix_(lv, lv)], w), f"insert {t}"
        check(g, mir, f"insert {t}")
        if t == 0:   # make room for the next insertions
            k = int(np.flatnonzero(mir.alive)[5])
            g.remove_node(k)
            mir.alive[k] = False
            mir.W[k, :] = mir.W[:, k] = mir.inf
    g.close()


@pytest.mark.parametrize("und", [False, True])
@pytest.mark.parametrize("dispatch", ["warm", "cold"])
def test_minimax_removal_list_and_result(und, dispatch):
    n, cap = 120, 128
    W = make(n, 11, undirected=und, p_missing=0.1)
    g = G(W, cap, und)
    g.set_dispatch(dispatch)
    mir = Mirror(W, cap, und)
    for t in range(5):
        live = np.flatnonzero(mir.alive)
        k = int(live[synth.uniform_int(11, 30 + t, 1, 0, len(live) - 1)[0]])
        M = mir.expected(cap)
        want = {(i, j) for i, js in O.need_update_list_minimax(M, mir.alive, k).items() for j in js}
        g.remove_node(k)
        mir.alive[k] = False
        mir.W[k, :] = mir.W[:, k] = mir.inf
        st = g.stats()
        got = {(int(a), int(b)) for a, b in g.last_list()}
        assert got == want, f"remove {k}: list differs"
        assert st["affected_pairs"] == len(want)
        if want:
            assert st["path"] == dispatch
        check(g, mir, f"remove {k}")
    g.close()


@pytest.mark.parametrize("fp", [False, True])
@pytest.mark.parametrize("und", [False, True])
def test_minimax_mixed_updates(fp, und):
    n, cap = 150, 176
    W = make(n, 13, fp=fp, undirected=und, p_missing=0.2)
    g = G(W, cap, und)
    mir = Mirror(W, cap, und)
    ups = synth.mixed_updates(n, 30, 13, tight=True, capacity=cap, w_lo=0, w_hi=20,
                              weights="lognormal" if fp else "int")
    for t, up in enumerate(ups):
        live = np.flatnonzero(mir.alive)
        if up.kind == synth.ADD:
            iw = np.full(cap, mir.inf, W.dtype)
            iw[live] = up.in_w[:len(live)]
            ow = iw.copy() if und else np.full(cap, mir.inf, W.dtype)
            if not und:
                ow[live] = up.out_w[:len(live)]
            p = g.add_node(iw, ow)
            assert p == O.lowest_free_slot(mir.alive)
            mir.W[:, p] = iw
            mir.W[p, :] = ow
            mir.W[p, p] = 0
            mir.alive[p] = True
            tag = f"add {p}"
        elif up.kind == synth.REMOVE:
            k = int(live[up.a])
            g.remove_node(k)
            mir.alive[k] = False
            mir.W[k, :] = mir.W[:, k] = mir.inf
            tag = f"remove {k}"
        else:
            u = int(live[up.a])
            row = np.where(mir.alive, mir.W[u].astype(np.float64), np.inf)
            row[u] = np.inf
            v = int(np.argmin(row))
            w0 = mir.W[u, v]
            if up.kind == synth.DECREASE:
                w = np.float32(w0 / 2) if fp else np.int32(w0 // 2)
            else:
                w = np.float32(w0 * 4 + 1) if fp else np.int32(int(w0) * 4 + 1)
            g.update_edge(u, v, w)
            mir.W[u, v] = w
            if und:
                mir.W[v, u] = w
            tag = f"{up.kind} ({u},{v}) {w0}->{w}"
        check(g, mir, f"step {t}: {tag}")
    g.close()


def test_minimax_unsupported_calls():
    from paper_2412_15122_gb300 import ApspError
    W = make(40, 3)
    g = G(W, 40, False)
    with pytest.raises(ApspError) as e:
        g.query_path(0, 5)
    assert e.value.status == 9
    with pytest.raises(ApspError):
        g.set_list_mode("algorithm12")
    g.close()
