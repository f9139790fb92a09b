"""The allocation-free insertion entry point (apsp_add_node_noalloc) gives the
same matrix as the regular apsp_add_node path.

Callers that cannot allocate device memory when they add a node (a request
handler that must not block on cudaMalloc, a framework that owns all device
memory through its own pool) use apsp_add_node_noalloc on a matrix they own;
its scratch is a fixed library array shared by every call.  Two calls in a row
check that the second call is not disturbed by what the first left in it.

The entry point reads only entries whose row and column are live and not the
new node, so the test fills row and column p, a second dead slot's row and
column, and the padding beyond n_slots with values that would corrupt a sum
(INT32_MAX, negative values, NaN) and still expects the regular result.
Collected last (file name) so that a failure here does not hide other tests.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

JUNK_I32 = [0x7FFFFFFF, -1, -(2 ** 31) + 7, 0]
JUNK_F32 = [-np.inf, np.nan, -1.0, 0.0]


def _weights(fp, call, cap):
    if fp:
        iw = np.exp(synth.normal_f64(8, 50 + call, cap)).astype(np.float32)
        ow = np.exp(synth.normal_f64(8, 60 + call, cap)).astype(np.float32)
    else:
        iw = synth.uniform_int(8, 50 + call, cap, 1, 1000).astype(np.int32)
        ow = synth.uniform_int(8, 60 + call, cap, 1, 1000).astype(np.int32)
    return iw, ow


@pytest.mark.parametrize("fp", [False, True])
@pytest.mark.parametrize("pad", [0, 4])
def test_noalloc_insertion_matches_add_node_twice(fp, pad):
    import torch
    from paper_2412_15122_gb300 import Graph, build
    from paper_2412_15122_gb300 import apsp as A

    build.build()
    n, cap = 200, 200            # n_slots stays 200 (a multiple of 4)
    ld = n + pad
    W = synth.lognormal_digraph_f32(n, 8) if fp else synth.complete_digraph_i32(n, 1, 1000, 8)
    g = Graph(W, cap)
    dt = A.APSP_F32 if fp else A.APSP_I32
    junk = JUNK_F32 if fp else JUNK_I32
    npdt = np.float32 if fp else np.int32
    stream = torch.cuda.current_stream()
    # call 0: slots 90 and 17 removed, the new node takes 17 (90 stays dead);
    # call 1: slot 150 removed, the new node takes 90 (150 stays dead)
    for call, removed in enumerate(((90, 17), (150,))):
        for k in removed:
            g.remove_node(k)
        D0 = g.D()                                       # APSP matrix before the insertion
        alive_np = g.alive().astype(np.int32)
        iw, ow = _weights(fp, call, cap)
        p = g.add_node(iw, ow)                           # regular path
        assert alive_np[p] == 0
        expect = g.D()
        live = g.alive().astype(bool)
        dead = np.flatnonzero(~live)
        assert dead.size >= 1
        # caller-owned matrix: the live block of D0, junk everywhere else
        Dh = np.empty((n, ld), dtype=npdt)
        Dh[:, :n] = D0
        for j, idx in enumerate(dead):
            Dh[idx, :] = junk[(call + j) % 4]
            Dh[:, idx] = junk[(call + j + 1) % 4]
        Dh[p, :] = junk[(call + 2) % 4]
        Dh[:, p] = junk[(call + 3) % 4]
        if pad:
            Dh[:, n:] = junk[call % 4]
        before = Dh.copy()
        Dn = torch.from_numpy(Dh).cuda()
        A.apsp_add_node_noalloc(Dn, ld, n, torch.from_numpy(alive_np).cuda(), dt, torch.from_numpy(iw).cuda(),
                                torch.from_numpy(ow).cuda(), p, stream)
        torch.cuda.synchronize()
        got = Dn.cpu().numpy()
        block = np.ix_(live, live)                       # live slots, p included
        e, o = expect[block], got[:, :n][block]
        if fp:
            fin = np.isfinite(e)
            assert np.array_equal(np.isfinite(o), fin), f"call {call}"
            assert np.all(np.abs(o[fin] - e[fin]) <= 1e-5 * np.abs(e[fin])), f"call {call}"
        else:
            assert np.array_equal(o, e), f"call {call}"
        inf = np.inf if fp else synth.INF_I32
        assert np.all(got[p, dead] == inf), "row p at dead slots reads missing"
        others = ~live
        others[p] = False
        rows_dead = np.ix_(others, np.ones(n, bool))
        np.testing.assert_array_equal(got[:, :n][rows_dead], before[:, :n][rows_dead])
        live_not_p = live.copy()
        live_not_p[p] = False                            # row p is written in full (above)
        np.testing.assert_array_equal(got[np.ix_(live_not_p, others)], before[np.ix_(live_not_p, others)])
        if pad:
            np.testing.assert_array_equal(got[:, n:], before[:, n:])
    g.close()


def test_noalloc_rejects_sizes_beyond_the_maximum():
    import torch
    from paper_2412_15122_gb300 import ApspError, build
    from paper_2412_15122_gb300 import apsp as A

    build.build()
    m = A.lib()  # noqa: F841
    d = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(ApspError) as e:
        A.apsp_add_node_noalloc(d, 16388, 16388, d, A.APSP_I32, d, d, 0)
    assert e.value.status == 4
    with pytest.raises(ApspError) as e:
        A.apsp_add_node_noalloc(d, 6, 6, d, A.APSP_I32, d, d, 0)   # not a multiple of 4
    assert e.value.status == 1
