"""Seeded synthetic inputs for warm-start APSP workloads.

This module is shared by the CPU oracle's tests and by the CUDA path's tests
and benchmark.  It holds no shortest-path arithmetic: it only draws random
numbers and builds weight matrices and update streams from them.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used in counter mode: draw i of
stream s is mix(base(seed, s) + (i + 1) * GAMMA).  Bounded integers use the
multiply-shift reduction of the top 32 bits (Lemire, "Fast random integer
generation in an interval", 2019, without the rejection step), uniform doubles
use the top 53 bits, and normal deviates use the Box-Muller transform.

Workload shapes follow the paper's experiments (Section 5: random complete
graphs of N nodes, random node removal, random edge modification); the weight
distributions are fixed here because the paper does not state them.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB

#: "no edge" for int32 weights; chosen so that two of them still fit in int32.
INF_I32 = 0x3FFFFFFF


def _mix64_scalar(z: int) -> int:
    z &= MASK64
    z = ((z ^ (z >> 30)) * _M1) & MASK64
    z = ((z ^ (z >> 27)) * _M2) & MASK64
    return z ^ (z >> 31)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(_M1)
        z ^= z >> np.uint64(27)
        z *= np.uint64(_M2)
        z ^= z >> np.uint64(31)
    return z


def stream_base(seed: int, stream: int) -> int:
    """64-bit starting state of sub-stream `stream` of `seed`."""
    return _mix64_scalar(_mix64_scalar(seed * GAMMA + 0x5EED) ^ (stream * 0xD1B54A32D192ED03))


def u64(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """`count` raw 64-bit draws of (seed, stream), starting at draw `offset`."""
    base = np.uint64(stream_base(seed, stream))
    idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        states = base + idx * np.uint64(GAMMA)
    return _mix64(states)


def uniform_int(seed: int, stream: int, count: int, lo: int, hi: int, offset: int = 0) -> np.ndarray:
    """Integers uniform in [lo, hi] (inclusive), int64."""
    span = hi - lo + 1
    assert 0 < span < (1 << 32)
    top = u64(seed, stream, count, offset) >> np.uint64(32)
    with np.errstate(over="ignore"):
        r = (top * np.uint64(span)) >> np.uint64(32)
    return r.astype(np.int64) + lo


def uniform_f64(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles uniform in [0, 1) from the top 53 bits."""
    return (u64(seed, stream, count, offset) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def normal_f64(seed: int, stream: int, count: int) -> np.ndarray:
    """Standard normal deviates by Box-Muller (one deviate per pair of draws)."""
    u = uniform_f64(seed, stream, 2 * count)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


# ---------------------------------------------------------------------------
# Weight matrices (row-major, W[i][j] = weight of edge i -> j, diagonal 0)
# ---------------------------------------------------------------------------

def complete_digraph_i32(n: int, lo: int, hi: int, seed: int, stream: int = 0) -> np.ndarray:
    """Directed complete graph, int32 weights uniform in [lo, hi]."""
    w = uniform_int(seed, stream, n * n, lo, hi).reshape(n, n).astype(np.int32)
    np.fill_diagonal(w, 0)
    return w


def lognormal_digraph_f32(n: int, seed: int, stream: int = 0) -> np.ndarray:
    """Directed complete graph, fp32 weights exp(N(0, 1))."""
    w = np.exp(normal_f64(seed, stream, n * n)).reshape(n, n).astype(np.float32)
    np.fill_diagonal(w, 0.0)
    return w


def unit_square_points(n: int, seed: int, stream: int = 0) -> np.ndarray:
    """n points uniform in the unit square, float64 (n, 2)."""
    return uniform_f64(seed, stream, 2 * n).reshape(n, 2)


def euclidean_weights_i32(p: np.ndarray, q: np.ndarray, scale: float = 1e4) -> np.ndarray:
    """round(scale * |p_a - q_b|) for all a, b, as int32 (round half up)."""
    d = np.hypot(p[:, None, 0] - q[None, :, 0], p[:, None, 1] - q[None, :, 1])
    return np.floor(d * scale + 0.5).astype(np.int32)


def euclidean_undirected_i32(n: int, seed: int, stream: int = 0, scale: float = 1e4):
    """Undirected complete Euclidean graph; returns (W, points)."""
    pts = unit_square_points(n, seed, stream)
    w = euclidean_weights_i32(pts, pts, scale)
    np.fill_diagonal(w, 0)
    return w, pts


# ---------------------------------------------------------------------------
# Update streams
# ---------------------------------------------------------------------------

ADD, REMOVE, DECREASE, INCREASE = "add", "remove", "decrease", "increase"
KINDS = (ADD, REMOVE, DECREASE, INCREASE)


@dataclasses.dataclass
class Update:
    """One graph update.

    Node references are ranks among the live nodes in ascending slot order
    (``a`` / ``b``), so the stream does not depend on how a consumer assigns
    slot ids.  For ``add`` the consumer uses ``in_w`` / ``out_w``: draw r is the
    weight to / from the r-th live node.  For edge updates the consumer derives
    the new weight from the current one: ``decrease`` halves it (floor),
    ``increase`` multiplies it by 4 (capped at ``cap``).  When ``tight`` is set,
    ``b`` is to be replaced by the lightest out-edge of ``a`` (that edge is
    always a shortest path in a complete graph with non-negative weights).
    """

    kind: str
    a: int = -1
    b: int = -1
    tight: bool = False
    in_w: Optional[np.ndarray] = None
    out_w: Optional[np.ndarray] = None
    cap: int = 1 << 26


def mixed_updates(n0: int, count: int, seed: int, *, fractions=(0.25, 0.25, 0.25, 0.25),
                  w_lo: int = 1, w_hi: int = 1000, tight: bool = False,
                  capacity: Optional[int] = None, min_live: int = 4,
                  stream: int = 7, weights: str = "int",
                  cap: int = 1 << 26) -> List[Update]:
    """A seeded stream of `count` mixed updates on a graph that starts with n0 live nodes.

    `fractions` = (add, remove, decrease, increase).  Kinds are drawn i.i.d.;
    adds are skipped when `capacity` live nodes exist and removals when only
    `min_live` remain.  New-node weights are int uniform in [w_lo, w_hi] or, for
    weights="lognormal", exp(N(0,1)) as float32.
    """
    kinds_u = uniform_f64(seed, stream, count)
    picks = u64(seed, stream + 1, 2 * count)
    cum = np.cumsum(np.asarray(fractions, dtype=np.float64))
    cum /= cum[-1]
    live = n0
    out: List[Update] = []
    for t in range(count):
        kind = KINDS[int(np.searchsorted(cum, kinds_u[t], side="right"))]
        if kind == ADD and capacity is not None and live >= capacity:
            kind = REMOVE
        if kind == REMOVE and live <= min_live:
            kind = ADD
        r0 = int(picks[2 * t] % np.uint64(live))
        r1 = int(picks[2 * t + 1] % np.uint64(live - 1))
        if r1 >= r0:
            r1 += 1
        if kind == ADD:
            m = live
            if weights == "lognormal":
                iw = np.exp(normal_f64(seed, 1000 + 2 * t, m)).astype(np.float32)
                ow = np.exp(normal_f64(seed, 1001 + 2 * t, m)).astype(np.float32)
            else:
                iw = uniform_int(seed, 1000 + 2 * t, m, w_lo, w_hi).astype(np.int32)
                ow = uniform_int(seed, 1001 + 2 * t, m, w_lo, w_hi).astype(np.int32)
            out.append(Update(ADD, in_w=iw, out_w=ow))
            live += 1
        elif kind == REMOVE:
            out.append(Update(REMOVE, a=r0))
            live -= 1
        else:
            out.append(Update(kind, a=r0, b=r1, tight=tight, cap=cap))
    return out


def new_point_weights_i32(pts_live: np.ndarray, seed: int, stream: int, scale: float = 1e4):
    """A new uniform point and its rounded Euclidean weights to the live points."""
    p = unit_square_points(1, seed, stream)
    return euclidean_weights_i32(p, pts_live, scale)[0], p[0]
