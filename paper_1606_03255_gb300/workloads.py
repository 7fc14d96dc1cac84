"""Seeded synthetic inputs shaped like the paper's experiments.

This module holds random-number recipes only -- none of the transform's
arithmetic -- so that the CUDA path, the tests, the benchmark and the oracle
can all be fed identical bits.  Every generator takes a seed and returns
numpy arrays (float64 / complex128 unless a dtype is asked for).

Node convention: a node is w = x + i*v with v >= 0, z = exp(2 pi i w), so
|z| = exp(-2 pi v).  Nodes are returned as an (M, 2) float64 array of
(Re w, Im w), which is the layout the C ABI takes.
"""
from __future__ import annotations

import numpy as np

TWO_PI = 2.0 * np.pi


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(int(seed))


def coefficients(N: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """c_k with Re and Im i.i.d. N(0, 1)."""
    g = _rng(seed)
    c = g.standard_normal(N) + 1j * g.standard_normal(N)
    return c.astype(dtype)


def nodes_from_polar(r: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """z = r exp(2 pi i theta) -> w = theta + i (-ln r) / (2 pi) as (M, 2)."""
    return np.stack([np.asarray(theta, np.float64),
                     -np.log(np.asarray(r, np.float64)) / TWO_PI], axis=-1)


def nodes_disk_uniform(M: int, seed: int) -> np.ndarray:
    """Nodes uniform in the unit disk: r = sqrt(U), U in (0, 1]; theta ~ U[0, 1)."""
    g = _rng(seed)
    u = 1.0 - g.random(M)              # (0, 1]: r > 0
    theta = g.random(M)
    return nodes_from_polar(np.sqrt(u), theta)


def nodes_circle_clustered(M: int, seed: int) -> np.ndarray:
    """Half the nodes exactly on |z| = 1, half with 1 - |z| = 10^(-6U), U ~ U[0, 1].

    The clustered half has Im w = -log1p(-delta) / (2 pi), delta = 10^(-6U); the
    order of the two halves is interleaved at random.
    """
    g = _rng(seed)
    theta = g.random(M)
    v = np.zeros(M)
    half = M // 2
    delta = 10.0 ** (-6.0 * g.random(M - half))
    v_cl = -np.log1p(-delta) / TWO_PI
    v_cl[~np.isfinite(v_cl)] = 40.0    # delta == 1 -> z = 0 (Z^0)
    idx = g.permutation(M)[half:]
    v[idx] = v_cl
    return np.stack([theta, v], axis=-1)


def nodes_paper_section5(M: int, q: int, seed: int) -> np.ndarray:
    """Section 5: x_j ~ U[0, 1), y_j ~ U[0, (2q-1) ln 2], y the paper's radial variable."""
    g = _rng(seed)
    x = g.random(M)
    y = g.random(M) * (2 * q - 1) * np.log(2.0)
    return np.stack([x, y / TWO_PI], axis=-1)


def nodes_equispaced_circle(M: int, radius: float = 1.0) -> np.ndarray:
    """x_j = j / M on the circle |z| = radius."""
    x = np.arange(M, dtype=np.float64) / M
    v = np.full(M, -np.log(radius) / TWO_PI if radius < 1.0 else 0.0)
    return np.stack([x, v], axis=-1)


def laplace_inputs(N: int, M: int, seed: int):
    """Real Laplace data: t_k ~ U[0, 1], s_j ~ U[0, 2N], c_k real N(0, 1)."""
    g = _rng(seed)
    t = g.random(N)
    s = g.random(M) * 2.0 * N
    c = g.standard_normal(N)
    return c, t, s


def batched_degrees(B: int, seed: int, lo: float = 8.0, hi: float = 16.0) -> np.ndarray:
    """N_i = floor(2^U), U ~ U[lo, hi] (log-uniform integer degrees)."""
    g = _rng(seed)
    return np.floor(2.0 ** (lo + (hi - lo) * g.random(B))).astype(np.int64)


def targets(M: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """g_j with Re and Im i.i.d. N(0, 1) (loss targets)."""
    return coefficients(M, seed, dtype)
