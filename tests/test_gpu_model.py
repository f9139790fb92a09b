"""Cost model on the GPU: the hand-written training kernels and the device
inference used by APSP_DISPATCH_MODEL, against the fp64 oracle."""
import numpy as np
import pytest

from oracle import apsp as OA
from oracle import mlp as OM

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    from paper_2412_15122_gb300 import apsp, build
    build.build()
    return apsp


def _data(n, seed, nan_frac=0.1):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, 6)) * [0.3, 2.0, 0.5, 0.01, 0.2, 0.3] + [0.5, 12, 0, 0.01, 0.2, 0.3]
    Y = np.stack([X[:, 1] * 0.8 + 20 * X[:, 3] + rng.normal(scale=0.1, size=n), 0.3 * X[:, 1] ** 2], 1)
    Y[rng.random(size=Y.shape) < nan_frac] = np.nan
    return X, Y


@pytest.mark.parametrize("n", [1, 37, 1000, 5003])
def test_loss_and_gradient_match_oracle(A, n):
    P = OM.random_params(n, scale=1.0)
    X, Y = _data(n, n + 1)
    L_ref, g_ref = OM.loss_grad(P, X, Y)
    L, g = A.apsp_model_loss_grad(P.astype(np.float32), X.astype(np.float32), Y.astype(np.float32))
    assert abs(L - L_ref) <= 1e-4 * max(1.0, abs(L_ref))
    scale = max(1e-6, np.abs(g_ref).max())
    np.testing.assert_allclose(g, g_ref, rtol=1e-3, atol=1e-4 * scale)
    assert np.linalg.norm(g - g_ref) <= 1e-4 * max(1e-12, np.linalg.norm(g_ref)) * 10


def test_predict_matches_oracle(A):
    P = OM.random_params(3, scale=1.0)
    X, _ = _data(777, 4)
    out = A.apsp_model_predict(P.astype(np.float32), X.astype(np.float32))
    ref = OM.forward(P, X)
    np.testing.assert_allclose(out, ref, rtol=1e-4, atol=1e-4 * np.abs(ref).max())


def test_training_fits_a_smooth_target(A):
    X, Y = _data(4000, 5, nan_frac=0.0)
    P, L = A.apsp_model_train(X, Y, epochs=60, batch=128, lr=3e-3, seed=7)
    base = float(np.nanmean((Y - np.nanmean(Y, 0)) ** 2) * 2)
    assert L < 0.05 * base, (L, base)
    # the reported loss is the oracle's loss of the returned parameters
    assert abs(L - OM.loss(P, X, Y)) <= 1e-3 * max(1.0, L)


def test_training_is_reproducible_for_a_seed(A):
    X, Y = _data(500, 6)
    P1, _ = A.apsp_model_train(X, Y, epochs=3, batch=64, lr=1e-3, seed=11)
    P2, _ = A.apsp_model_train(X, Y, epochs=3, batch=64, lr=1e-3, seed=11)
    # same initialisation and shuffles; fp32 atomics may reorder sums
    np.testing.assert_allclose(P1, P2, rtol=1e-3, atol=1e-5)


def test_set_model_rejects_bad_standardisation(A):
    from paper_2412_15122_gb300 import Graph
    import synth
    W = synth.complete_digraph_i32(16, 1, 100, 1)
    g = Graph(W, 32)
    P = OM.random_params(1).astype(np.float32)
    P[6] = 0.0   # sd[0]
    with pytest.raises(A.ApspError):
        g.set_model(P)
    g.close()


def _forced_model(warm, cold):
    d = {k: v.copy() for k, v in OM.unpack(OM.random_params(2)).items()}
    d["W3"][:] = 0.0
    d["b3"][:] = [warm, cold]
    return OM.pack(d).astype(np.float32)


@pytest.mark.parametrize("prefer", ["warm", "cold"])
def test_model_dispatch_picks_cheaper_path_and_stays_exact(A, prefer):
    from paper_2412_15122_gb300 import Graph
    import synth
    n = 96
    W = synth.complete_digraph_i32(n, 1, 1000, 21)
    g = Graph(W, n + 32)
    g.set_dispatch("model")
    g.set_model(_forced_model(5.0, 20.0) if prefer == "warm" else _forced_model(20.0, 5.0))
    M = OA.fw(W)
    alive = np.ones(n, bool)
    for k in (3, 50, 77):
        g.remove_node(k)
        st = g.stats()
        if st["affected_pairs"] > 0:
            assert st["path"] == prefer, st
            assert st["model_warm"] == pytest.approx(5.0 if prefer == "warm" else 20.0)
        alive[k] = False
    Wl = W.astype(np.int64).copy()
    Wl[~alive, :] = OA.INF_I32
    Wl[:, ~alive] = OA.INF_I32
    ref = OA.to_i32(OA.fw(Wl, alive))
    D = g.D()[:n, :n]
    np.testing.assert_array_equal(D[np.ix_(alive, alive)], ref[np.ix_(alive, alive)])
    g.close()
