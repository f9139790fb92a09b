"""Pins of the cost-model oracle (oracle/mlp.py) against mathematics that does
not depend on its own formulas: central finite differences of the loss,
closed forms of degenerate networks, and missing labels."""
import numpy as np
import pytest

from oracle import mlp as O


def _data(n, seed, nan_frac=0.0):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, O.N_IN)) * 3 + 1
    Y = rng.normal(size=(n, O.N_OUT)) * 2 + 5
    if nan_frac:
        Y[rng.random(size=Y.shape) < nan_frac] = np.nan
    return X, Y


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_gradient_matches_central_differences(seed):
    P = O.random_params(seed, scale=1.0)
    X, Y = _data(37, seed + 10, nan_frac=0.2)
    L, g = O.loss_grad(P, X, Y)
    assert abs(L - O.loss(P, X, Y)) <= 1e-12 * max(1.0, L)
    rng = np.random.default_rng(seed + 20)
    coords = rng.choice(O.N_TRAIN, size=60, replace=False)
    h = 1e-6
    for c in coords:
        Pp, Pm = P.copy(), P.copy()
        Pp[2 * O.N_IN + c] += h
        Pm[2 * O.N_IN + c] -= h
        fd = (O.loss(Pp, X, Y) - O.loss(Pm, X, Y)) / (2 * h)
        assert abs(fd - g[c]) <= 1e-5 * max(1.0, abs(fd)), (c, fd, g[c])


def test_zero_output_weights_give_the_bias():
    d = O.unpack(O.random_params(4))
    d = {k: v.copy() for k, v in d.items()}
    d["W3"][:] = 0.0
    d["b3"][:] = [3.25, -1.5]
    X, _ = _data(11, 5)
    np.testing.assert_array_equal(O.forward(O.pack(d), X), np.tile([3.25, -1.5], (11, 1)))


def test_linear_regime_is_a_matrix_product():
    # with every hidden pre-activation positive the network is affine:
    # o = W3 (W2 (W1 x^ + b1) + b2) + b3
    d = {k: v.copy() for k, v in O.unpack(O.random_params(6)).items()}
    d["b1"][:] = 100.0
    d["W2"] = np.abs(d["W2"])
    d["b2"][:] = 100.0
    X, _ = _data(9, 7)
    Xh = (X - d["mu"]) / d["sd"]
    assert (Xh @ d["W1"].T + d["b1"] > 0).all()
    expect = ((Xh @ d["W1"].T + d["b1"]) @ d["W2"].T + d["b2"]) @ d["W3"].T + d["b3"]
    np.testing.assert_allclose(O.forward(O.pack(d), X), expect, rtol=1e-12)


def test_perfect_fit_has_zero_loss_and_gradient():
    P = O.random_params(8)
    X, _ = _data(20, 9)
    Y = O.forward(P, X)
    L, g = O.loss_grad(P, X, Y)
    assert L == 0.0
    assert np.abs(g).max() == 0.0


def test_missing_labels_count_as_absent_terms():
    P = O.random_params(10)
    X, Y = _data(25, 11)
    Yn = Y.copy()
    Yn[3, 0] = np.nan
    Yn[7, :] = np.nan
    # the loss with NaN labels equals the loss with those outputs predicted exactly
    Yfill = Yn.copy()
    Ofw = O.forward(P, X)
    Yfill[np.isnan(Yn)] = Ofw[np.isnan(Yn)]
    assert abs(O.loss(P, X, Yn) - O.loss(P, X, Yfill)) <= 1e-12
    np.testing.assert_allclose(O.loss_grad(P, X, Yn)[1], O.loss_grad(P, X, Yfill)[1], atol=1e-12)


def test_planted_relu_mistake_is_caught(monkeypatch):
    """A backward pass that forgets the ReLU mask of the first layer must fail
    the finite-difference pin."""
    P = O.random_params(12, scale=1.5)
    X, Y = _data(30, 13)
    real = O.loss_grad

    def wrong(params, X_, Y_):
        d = O.unpack(params)
        Xh = (X_ - d["mu"]) / d["sd"]
        z1 = Xh @ d["W1"].T + d["b1"]
        h1 = np.maximum(z1, 0)
        z2 = h1 @ d["W2"].T + d["b2"]
        h2 = np.maximum(z2, 0)
        Ov = h2 @ d["W3"].T + d["b3"]
        D = Ov - Y_
        dO = 2 * D / X_.shape[0]
        dh2 = (dO @ d["W3"]) * (z2 > 0)
        dh1 = dh2 @ d["W2"]                 # mask dropped
        g = np.concatenate([(dh1.T @ Xh).ravel(), dh1.sum(0), (dh2.T @ h1).ravel(), dh2.sum(0),
                            (dO.T @ h2).ravel(), dO.sum(0)])
        return float((D * D).sum() / X_.shape[0]), g

    _, g_wrong = wrong(P, X, Y)
    _, g_real = real(P, X, Y)
    # central differences agree with the real gradient and not with the planted one
    worst = 0.0
    for c in range(0, O.N_IN * O.N_H + O.N_H, 7):
        Pp, Pm = P.copy(), P.copy()
        Pp[2 * O.N_IN + c] += 1e-6
        Pm[2 * O.N_IN + c] -= 1e-6
        fd = (O.loss(Pp, X, Y) - O.loss(Pm, X, Y)) / 2e-6
        assert abs(fd - g_real[c]) <= 1e-5 * max(1.0, abs(fd))
        worst = max(worst, abs(fd - g_wrong[c]))
    assert worst > 1e-3
