"""The seeded input generators against their published definitions:
SplitMix64 (Steele, Lea & Flood 2014) in counter mode, the multiply-shift
bounded-integer reduction and the 53-bit doubles."""
import numpy as np

import synth


def test_splitmix64_reference_outputs():
    # the first outputs of SplitMix64 started from state 0
    expect = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    state, got = 0, []
    for _ in expect:
        state = (state + synth.GAMMA) & synth.MASK64
        got.append(synth._mix64_scalar(state))
    assert got == expect
    # the vectorised mix agrees with the scalar one
    z = np.array([synth.GAMMA * k & synth.MASK64 for k in range(1, 5)], dtype=np.uint64)
    assert [int(x) for x in synth._mix64(z)] == expect


def test_counter_mode_draws():
    seed, stream = 7, 3
    base = synth.stream_base(seed, stream)
    manual = [synth._mix64_scalar(base + (i + 1) * synth.GAMMA) for i in range(2, 7)]
    assert [int(x) for x in synth.u64(seed, stream, 5, offset=2)] == manual
    assert synth.stream_base(seed, 3) != synth.stream_base(seed, 4) != synth.stream_base(seed + 1, 4)


def test_bounded_integers_and_doubles():
    lo, hi = 5, 17
    r = synth.uniform_int(1, 2, 20000, lo, hi)
    assert r.min() == lo and r.max() == hi
    raw = synth.u64(1, 2, 20000)
    assert np.array_equal(r, ((raw >> np.uint64(32)) * np.uint64(hi - lo + 1) >> np.uint64(32)).astype(np.int64) + lo)
    f = synth.uniform_f64(1, 2, 20000)
    assert (f >= 0).all() and (f < 1).all()
    assert np.array_equal(f, (raw >> np.uint64(11)).astype(np.float64) / 2.0 ** 53)


def test_complete_graph_shape():
    W = synth.complete_digraph_i32(9, 1, 100, 4)
    assert W.dtype == np.int32 and W.shape == (9, 9)
    assert (np.diag(W) == 0).all()
    off = W[~np.eye(9, dtype=bool)]
    assert off.min() >= 1 and off.max() <= 100
