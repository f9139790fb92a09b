"""The allocation-free insertion entry point (apsp_add_node_noalloc) gives the
same matrix as the regular apsp_add_node path.

Callers that cannot allocate device memory when they add a node (a request
handler that must not block on cudaMalloc, a framework that owns all device
memory through its own pool) use apsp_add_node_noalloc on a matrix they own;
its scratch is a fixed library array shared by every call.  Two calls in a row
check that the second call is not disturbed by what the first left in it.
Collected last (file name) so that a failure here does not hide other tests.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fp", [False, True])
def test_noalloc_insertion_matches_add_node_twice(fp):
    import torch
    from paper_2412_15122_gb300 import Graph, build
    from paper_2412_15122_gb300 import apsp as A

    build.build()
    n, cap = 200, 200            # n_slots stays 200 (a multiple of 4)
    W = synth.lognormal_digraph_f32(n, 8) if fp else synth.complete_digraph_i32(n, 1, 1000, 8)
    g = Graph(W, cap)
    dt = A.APSP_F32 if fp else A.APSP_I32
    stream = torch.cuda.current_stream()
    for call, k in enumerate((17, 150)):
        g.remove_node(k)
        D0 = torch.from_numpy(g.D()).cuda()              # APSP matrix with slot k dead
        alive = torch.from_numpy(g.alive().astype(np.int32)).cuda()
        if fp:
            iw = np.exp(synth.normal_f64(8, 50 + call, cap)).astype(np.float32)
            ow = np.exp(synth.normal_f64(8, 60 + call, cap)).astype(np.float32)
        else:
            iw = synth.uniform_int(8, 50 + call, cap, 1, 1000).astype(np.int32)
            ow = synth.uniform_int(8, 60 + call, cap, 1, 1000).astype(np.int32)
        p = g.add_node(iw, ow)                           # regular path
        assert p == k
        expect = g.D()
        Dn = D0.clone()
        A.apsp_add_node_noalloc(Dn, n, n, alive, dt, torch.from_numpy(iw).cuda(), torch.from_numpy(ow).cuda(),
                                k, stream)
        torch.cuda.synchronize()
        got = Dn.cpu().numpy()
        if fp:
            fin = np.isfinite(expect)
            assert np.array_equal(np.isfinite(got), fin)
            assert np.all(np.abs(got[fin] - expect[fin]) <= 1e-5 * np.abs(expect[fin])), f"call {call}"
        else:
            assert np.array_equal(got, expect), f"call {call}"
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
