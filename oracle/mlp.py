"""CPU oracle of the warm/cold cost model (fp64, numpy).

TEST INFRASTRUCTURE ONLY: imported by the tests and nothing else.  Shares no
code with the CUDA path.

The model is a multilayer perceptron with two ReLU hidden layers of 64 units
that maps the 6 features of an update to 2 outputs (predicted log2
microseconds of the warm and of the cold path).  The paper has no such model:
it decides with a threshold delta on Cost (Algorithm 5, Definition of Cost);
the model replaces that threshold.  Written from the definition:

    x^ = (x - mu) / sd
    z1 = W1 x^ + b1,  h1 = max(z1, 0)
    z2 = W2 h1 + b2,  h2 = max(z2, 0)
    o  = W3 h2 + b3
    loss = (1/n) * sum over samples and outputs of (o - y)^2   (NaN y: absent)

and its gradient by the chain rule.  Parameter block (floats, this order):
mu[6], sd[6], W1[64][6], b1[64], W2[64][64], b2[64], W3[2][64], b3[2]; the
gradient covers the block from W1 on.
"""
from __future__ import annotations

from typing import Dict, Tuple

import numpy as np

N_IN, N_H, N_OUT = 6, 64, 2
_SHAPES = [("mu", (N_IN,)), ("sd", (N_IN,)), ("W1", (N_H, N_IN)), ("b1", (N_H,)),
           ("W2", (N_H, N_H)), ("b2", (N_H,)), ("W3", (N_OUT, N_H)), ("b3", (N_OUT,))]
N_PARAM = sum(int(np.prod(s)) for _, s in _SHAPES)
N_TRAIN = N_PARAM - 2 * N_IN


def unpack(params) -> Dict[str, np.ndarray]:
    p = np.asarray(params, dtype=np.float64).ravel()
    if p.size != N_PARAM:
        raise ValueError(f"expected {N_PARAM} parameters, got {p.size}")
    out, o = {}, 0
    for name, shape in _SHAPES:
        k = int(np.prod(shape))
        out[name] = p[o:o + k].reshape(shape)
        o += k
    return out


def pack(d: Dict[str, np.ndarray]) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in _SHAPES])


def forward(params, X) -> np.ndarray:
    """Outputs (n x 2) for raw features X (n x 6)."""
    P = unpack(params)
    Xh = (np.asarray(X, np.float64) - P["mu"]) / P["sd"]
    h1 = np.maximum(Xh @ P["W1"].T + P["b1"], 0.0)
    h2 = np.maximum(h1 @ P["W2"].T + P["b2"], 0.0)
    return h2 @ P["W3"].T + P["b3"]


def loss(params, X, Y) -> float:
    O = forward(params, X)
    Y = np.asarray(Y, np.float64)
    m = ~np.isnan(Y)
    D = np.where(m, O - np.where(m, Y, 0.0), 0.0)
    return float((D * D).sum() / X.shape[0])


def loss_grad(params, X, Y) -> Tuple[float, np.ndarray]:
    """Loss and its gradient with respect to W1, b1, W2, b2, W3, b3 (in the
    parameter block's order), by backpropagation."""
    P = unpack(params)
    X = np.asarray(X, np.float64)
    Y = np.asarray(Y, np.float64)
    n = X.shape[0]
    Xh = (X - P["mu"]) / P["sd"]
    z1 = Xh @ P["W1"].T + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(z2, 0.0)
    O = h2 @ P["W3"].T + P["b3"]
    m = ~np.isnan(Y)
    D = np.where(m, O - np.where(m, Y, 0.0), 0.0)
    L = float((D * D).sum() / n)
    dO = 2.0 * D / n                      # dL/dO
    gW3 = dO.T @ h2
    gb3 = dO.sum(0)
    dh2 = (dO @ P["W3"]) * (z2 > 0)       # through the ReLU
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(0)
    dh1 = (dh2 @ P["W2"]) * (z1 > 0)
    gW1 = dh1.T @ Xh
    gb1 = dh1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return L, g


def random_params(seed: int, scale: float = 0.5) -> np.ndarray:
    """A parameter block with non-degenerate standardisation, for tests."""
    rng = np.random.default_rng(seed)
    d = {"mu": rng.normal(size=N_IN), "sd": rng.uniform(0.5, 2.0, size=N_IN)}
    for name, shape in _SHAPES[2:]:
        d[name] = rng.normal(scale=scale / np.sqrt(shape[-1] if len(shape) > 1 else N_H), size=shape)
    return pack(d)
