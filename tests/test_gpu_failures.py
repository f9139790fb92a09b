"""Failure detection without a GPU fault: a bounded device wait that runs out
reports APSP_E_TIMEOUT and leaves the device usable; allocation failures come
back as APSP_E_NOMEM; the caller's allocator is honoured."""
import time

import numpy as np
import pytest

import synth
from oracle import apsp as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    import torch
    assert torch.cuda.is_available()
    from paper_2412_15122_gb300 import apsp, build
    build.build()
    return apsp


def _small_check(A):
    from paper_2412_15122_gb300 import Graph
    W = synth.complete_digraph_i32(40, 1, 100, 17)
    g = Graph(W, 48)
    g.remove_node(3)
    alive = np.ones(40, dtype=bool)
    alive[3] = False
    ref = O.to_i32(O.fw(W, alive))
    D = g.D()
    live = np.flatnonzero(alive)
    assert np.array_equal(D[np.ix_(live, live)], ref[np.ix_(live, live)])
    g.close()


def test_barrier_wait_runs_out_and_reports_timeout(A):
    assert A.apsp_selftest_barrier_timeout(False) == 0
    t0 = time.perf_counter()
    assert A.apsp_selftest_barrier_timeout(True) == 7          # APSP_E_TIMEOUT
    waited = time.perf_counter() - t0
    assert 1.5 < waited < 30.0
    _small_check(A)                                             # the device is still usable


def test_failing_allocator_gives_nomem_and_recovers(A):
    lib = A.lib()
    calls = []

    def refuse(nbytes, stream, ctx):
        calls.append(nbytes)
        return None

    def ignore(ptr, nbytes, stream, ctx):
        pass

    alloc, free = A.ALLOC_FN(refuse), A.FREE_FN(ignore)
    assert lib.apsp_set_allocator(alloc, free, None) == 0
    try:
        W = synth.complete_digraph_i32(30, 1, 100, 5)
        with pytest.raises(A.ApspError) as e:
            A.apsp_init(W, 30, 32, A.APSP_I32)
        assert e.value.status == 5                              # APSP_E_NOMEM
        assert calls
    finally:
        A.apsp_set_allocator_default()
    _small_check(A)


def test_torch_caching_allocator_path(A):
    A.apsp_set_allocator_torch()
    try:
        _small_check(A)
    finally:
        A.apsp_set_allocator_default()
