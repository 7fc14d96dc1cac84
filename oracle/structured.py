"""Structured reference: the matrices that Algorithms 1 and 2 of Kunis & Melzer apply (numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Tiny N only.  Nothing
here follows the listings of the paper: each function assembles, block by
block, the dense matrix that the paper proves its algorithm applies and
multiplies it with the coefficient vector.

* Algorithm 1 applies K~ of eq. (A.1): for a node in Y_m and a frequency in
  Omega_l the entry is 1 (l > L_m), the rank-q interpolant
  L^{Y_m} K^{Y_m,Omega_l} (L^{Omega_l})^T of Definition 3.2 (l_m <= l <= L_m)
  or 0 (l < l_m); rows of Y_M are all ones.
* Algorithm 2 applies the Hadamard product A o K~ (Lemma 4.1, Lemma 4.2,
  Theorem 4.3): A = (exp(2 pi i xi_k x_j)) the Fourier matrix, here formed
  exactly (a dense NDFT), and K~ the matrix above for the kernel exp(-y xi)
  with y = 2 pi Im w.  So what remains is the error of the hierarchical
  Laplace factorisation alone.

Readings of the paper taken here (each is restated where it is used):

* Index shift: the paper sums k = 1..N, this code k = 0..N-1, so xi_k = k and
  xi_1 = N - 1.  The k = 0 term has kernel value 1 for every node.
* Z^0 nodes (|z| < eps, i.e. y > ln(1/eps)) return c_0, not 0: the paper's
  bound |f(z)| < eps ||c||_1 there assumes k >= 1 (proof of Theorem 4.3).
* Alg. 2 uses y_1 = ln(1/eps) (after Z^0 is removed every y lies in
  [0, ln(1/eps)], proof of Theorem 4.3) and xi_1 = N - 1.
* Lemma 4.1 needs both factors at eps/3: the Laplace partition (Definition 3.2:
  q, the number of levels, l_m, L_m) is built with eps_K = eps / 3.
* The inner logarithm in l_m is the natural one: Lemma A.2(ii) needs
  y_1 xi_1 / 2^(m+l) >= ln(1/eps).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


# --------------------------------------------------------------------------
# Section 2: Chebyshev nodes, barycentric Lagrange polynomials.

def chebyshev_points(q: int) -> np.ndarray:
    """t_j = cos((2j+1) pi / (2q)), j = 0..q-1: zeros of T_q (Section 2)."""
    j = np.arange(q, dtype=np.float64)
    return np.cos((2.0 * j + 1.0) * np.pi / (2.0 * q))


def barycentric_weights(q: int) -> np.ndarray:
    """lambda_r = (-1)^r sin((2r+1) pi / (2q)) (Section 2)."""
    r = np.arange(q, dtype=np.float64)
    return (-1.0) ** r * np.sin((2.0 * r + 1.0) * np.pi / (2.0 * q))


def interval_points(a: float, b: float, q: int) -> np.ndarray:
    """Chebyshev nodes of [a, b]: c^A + (diam A / 2) t_j (Section 2)."""
    return 0.5 * (a + b) + 0.5 * (b - a) * chebyshev_points(q)


def lagrange_barycentric(y, a: float, b: float, q: int) -> np.ndarray:
    """Matrix (len(y), q) of L_r^A(y) by the barycentric formula (Section 2).

    At a Chebyshev node y = y_s the formula divides by zero; there L_r = delta_rs.
    """
    y = np.atleast_1d(np.asarray(y, dtype=np.float64))
    nodes = interval_points(a, b, q)
    lam = barycentric_weights(q)
    diff = y[:, None] - nodes[None, :]
    hit = diff == 0.0
    with np.errstate(divide="ignore", invalid="ignore"):
        terms = lam[None, :] / diff
        out = terms / terms.sum(axis=1, keepdims=True)
    rows = hit.any(axis=1)
    if rows.any():
        out[rows] = hit[rows].astype(np.float64)
    return out


def lagrange_product(y, a: float, b: float, q: int) -> np.ndarray:
    """L_r^A(y) by the product formula of Section 2 (used to pin the barycentric one)."""
    y = np.atleast_1d(np.asarray(y, dtype=np.float64))
    nodes = interval_points(a, b, q)
    out = np.ones((y.size, q))
    for r in range(q):
        for j in range(q):
            if j != r:
                out[:, r] *= (y - nodes[j]) / (nodes[r] - nodes[j])
    return out


# --------------------------------------------------------------------------
# Definition 3.2: rank, number of levels, block ranges, dyadic partition.

@dataclass
class LaplaceParams:
    eps: float
    y1: float
    xi1: float
    q: int
    M: int                       # number of levels (the paper's M)
    ell: dict = field(default_factory=dict)   # l_m, m = 1..M-1
    L: dict = field(default_factory=dict)     # L_m = M - m


def rank_q(eps: float) -> int:
    """q = ceil(1/2 + log_4(1/eps)) (Definition 3.2)."""
    return int(math.ceil(0.5 + math.log(1.0 / eps, 4.0)))


def laplace_params(eps: float, y1: float, xi1: float, q: int | None = None) -> LaplaceParams:
    """Definition 3.2 with the natural inner logarithm in l_m."""
    qq = rank_q(eps) if q is None else int(q)
    if y1 <= 0.0 or xi1 <= 0.0:
        return LaplaceParams(eps, y1, xi1, qq, 1)
    M = int(math.ceil(math.log2(y1 * xi1 / eps))) + 1
    M = max(M, 1)
    p = LaplaceParams(eps, y1, xi1, qq, M)
    for m in range(1, M):
        p.ell[m] = max(1, int(math.floor(math.log2(y1 * xi1) - m
                                         - math.log2(math.log(1.0 / eps)))) + 1)
        p.L[m] = M - m
    return p


def band_of(v, v1: float, M: int) -> np.ndarray:
    """Dyadic band index: v in (v1/2^b, v1/2^(b-1)] -> b (b < M); v <= v1/2^(M-1) -> M."""
    v = np.atleast_1d(np.asarray(v, dtype=np.float64))
    out = np.full(v.shape, M, dtype=np.int64)
    undecided = np.ones(v.shape, dtype=bool)
    for b in range(1, M):
        edge = math.ldexp(v1, -b)
        sel = undecided & (v > edge)
        out[sel] = b
        undecided &= ~sel
    return out


def band_interval(v1: float, b: int) -> tuple[float, float]:
    """(v1/2^b, v1/2^(b-1)) for b < M (Definition 3.2)."""
    b = int(b)
    return math.ldexp(v1, -b), math.ldexp(v1, -(b - 1))


def kernel_block(params: LaplaceParams, m: int, l: int) -> np.ndarray:
    """K^{Y_m, Omega_l}_{s r} = exp(-y_s^{Y_m} xi_r^{Omega_l}) (Definition 3.2)."""
    ya, yb = band_interval(params.y1, m)
    xa, xb = band_interval(params.xi1, l)
    ys = interval_points(ya, yb, params.q)
    xr = interval_points(xa, xb, params.q)
    return np.exp(-np.outer(ys, xr))


# --------------------------------------------------------------------------
# Algorithm 1 (Section 3): the matrix K~ of eq. (A.1), assembled block by block.

def tilde_kernel(yv, xv, p: LaplaceParams, y1: float, xi1: float) -> np.ndarray:
    """Dense K~ (len(yv), len(xv)) of eq. (A.1) for the kernel exp(-y xi).

    Node y in Y_m (m < M) and frequency xi in Omega_l (Definition 3.2):
      l > L_m:          1                                     (Lemma A.2 (iv))
      l_m <= l <= L_m:  L^{Y_m}(y) K^{Y_m,Omega_l} L^{Omega_l}(xi)^T  (Lemma A.1)
      l < l_m:          0                                     (Lemma A.2 (ii))
    and every row of Y_M is 1 (Lemma A.2 (i)); with a single level (M = 1)
    every entry is 1.  Each block is one product of the three factors.
    """
    yv = np.atleast_1d(np.asarray(yv, dtype=np.float64))
    xv = np.atleast_1d(np.asarray(xv, dtype=np.float64))
    K = np.zeros((yv.size, xv.size))
    if p.M == 1:
        K[:] = 1.0
        return K
    by = band_of(yv, y1, p.M)
    bx = band_of(xv, xi1, p.M)
    K[by == p.M, :] = 1.0
    cols = {l: np.nonzero(bx == l)[0] for l in range(1, p.M + 1)}
    Lx = {}
    for l in range(1, p.M):
        if cols[l].size:
            Lx[l] = lagrange_barycentric(xv[cols[l]], *band_interval(xi1, l), p.q)
    for m in range(1, p.M):
        rows = np.nonzero(by == m)[0]
        if not rows.size:
            continue
        Ly = lagrange_barycentric(yv[rows], *band_interval(y1, m), p.q)
        for l in range(1, p.M + 1):
            if not cols[l].size:
                continue
            if l > p.L[m]:
                K[np.ix_(rows, cols[l])] = 1.0
            elif l >= p.ell[m]:
                K[np.ix_(rows, cols[l])] = Ly @ kernel_block(p, m, l) @ Lx[l].T
    return K


def laplace_tilde_matrix(t, s, eps: float, q: int | None = None,
                         y1: float | None = None, xi1: float | None = None):
    """Dense K~ of eq. (A.1) for nodes s and frequencies t; returns (K~, params).

    Entry (j, k) approximates exp(-s_j t_k); y_1 = max s_j and xi_1 = max t_k
    unless given (Algorithm 1 takes the largest node and frequency).
    """
    t = np.asarray(t, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    xi1 = (float(t.max()) if t.size else 0.0) if xi1 is None else float(xi1)
    y1 = (float(s.max()) if s.size else 0.0) if y1 is None else float(y1)
    p = laplace_params(eps, y1, xi1, q)
    return tilde_kernel(s, t, p, y1, xi1), p


def laplace_alg1(c, t, s, eps: float, q: int | None = None):
    """What Algorithm 1 returns, f~ = K~ c (eq. (A.1), Theorem A.3); (f~, params).

    Real or complex c.  K~ is formed densely (tiny N only).
    """
    c = np.asarray(c)
    K, p = laplace_tilde_matrix(t, s, eps, q)
    return K @ c, p


# --------------------------------------------------------------------------
# Algorithm 2 with the exact NDFT in place of A~.

def _frac_phase(x: np.ndarray, k: np.ndarray) -> np.ndarray:
    """frac(outer(x, k)) with ~1 ulp error: x = xh + xl, xh holding 26 bits."""
    x = np.asarray(x, dtype=np.float64)
    xh = np.round(x * 2.0 ** 26) / 2.0 ** 26          # exact split
    xl = x - xh                                        # exact
    kk = k.astype(np.float64)
    ph = np.outer(xh, kk)                              # exact for k < 2^27
    ph = ph - np.floor(ph)
    ph = ph + np.outer(xl, kk)
    return ph - np.floor(ph)


def ndft(coef, k, x) -> np.ndarray:
    """Exact (dense) nonequispaced DFT: sum_k coef_k exp(2 pi i k x_j); coef may be 2-D."""
    k = np.asarray(k, dtype=np.int64)
    E = np.exp(2j * np.pi * _frac_phase(x, k))
    return E @ np.asarray(coef)


@dataclass
class XFLTParams:
    eps: float
    eps_K: float
    y1: float
    xi1: float
    lap: LaplaceParams


def xflt_params(N: int, eps: float, q: int | None = None) -> XFLTParams:
    """Alg. 2 parameters: y_1 = ln(1/eps), xi_1 = N - 1, Laplace part at eps/3."""
    eps_K = eps / 3.0
    y1 = math.log(1.0 / eps)
    xi1 = float(max(N - 1, 0))
    return XFLTParams(eps, eps_K, y1, xi1, laplace_params(eps_K, y1, xi1, q))


def _split_nodes(w):
    """(x, Im w) of complex nodes or of an (M, 2) array of (Re w, Im w)."""
    w = np.asarray(w)
    if not np.iscomplexobj(w):
        w = np.asarray(w, dtype=np.float64).reshape(-1, 2)
        return w[:, 0], w[:, 1]
    return w.real, w.imag


def fourier_matrix(k, x) -> np.ndarray:
    """A = (exp(2 pi i k x_j)) for integer k, formed exactly (phases reduced mod 1)."""
    return np.exp(2j * np.pi * _frac_phase(x, np.asarray(k, dtype=np.int64)))


def xflt_matrix(N: int, w, eps: float, q: int | None = None):
    """The matrix Algorithm 2 applies to c, with the NFFT replaced by A itself.

    Row j: Z^0 node (y_j > ln(1/eps), |z_j| < eps) -> e_0 (f~ = c_0, the index
    shift reading); else A_j o K~_j with A_jk = exp(2 pi i k x_j) and K~ of
    eq. (A.1) for exp(-y xi) at y = 2 pi Im w_j, xi = k, y_1 = ln(1/eps),
    xi_1 = N - 1, built at eps/3 (Lemma 4.1: C ~ A o K~, Theorem 4.3).
    Returns (matrix, XFLTParams).
    """
    x, yim = _split_nodes(w)
    P = xflt_params(N, eps, q)
    y = 2.0 * np.pi * yim                 # the paper's y: |z| = exp(-y)
    kall = np.arange(N)
    z0 = y > P.y1
    C = np.zeros((x.size, N), dtype=np.complex128)
    C[z0, 0] = 1.0
    keep = ~z0
    if keep.any():
        C[keep] = fourier_matrix(kall, x[keep]) * tilde_kernel(y[keep], kall, P.lap, P.y1, P.xi1)
    return C, P


def xflt_alg2(c, w, eps: float, q: int | None = None):
    """What Algorithm 2 returns with exact NDFTs, f~ = (A o K~) c; (f~, params).

    w: complex nodes in the closed upper half plane (z = exp(2 pi i w)) or an
    (M, 2) array of (Re w, Im w).  The matrix is formed densely (tiny N only).
    """
    c = np.asarray(c, dtype=np.complex128)
    C, P = xflt_matrix(c.size, w, eps, q)
    return C @ c, P


# --------------------------------------------------------------------------
# One-sided variant of Algorithm 2: interpolation in y only.
#
# For fixed frequency k, g(y) = exp(-y k) on A = Y_m = (a, 2a] is replaced by
# its Chebyshev interpolant sum_s L_s^A(y) exp(-y_s^A k) -- the first of the
# two interpolations in the proof of Theorem 3.1 (asymptotically smooth
# kernels).  The error formula of Section 2 with diam A = a and
# max_A |g^(q)| = k^q exp(-a k) bounds one entry by
#     2 (k a / 4)^q exp(-k a) / q!  <=  2 q^q exp(-q) / (4^q q!)
# (the maximum over k a >= 0 is at k a = q).  Frequencies with k a >
# ln(1/eps_K) are dropped exactly as region (ii) of Algorithm 2 (l < l_m).

def onesided_entry_bound(ka, q: int) -> np.ndarray:
    """2 (ka/4)^q exp(-ka) / q!: per-entry bound of the one-sided interpolation."""
    ka = np.asarray(ka, dtype=np.float64)
    return np.exp(math.log(2.0) + q * np.log(np.maximum(ka, 1e-300) / 4.0) - ka
                  - math.lgamma(q + 1.0)) * (ka > 0)


def rank_q_onesided(eps: float, qmax: int = 64) -> int:
    """Smallest q with 2 q^q e^-q / (4^q q!) <= eps (the bound maximised over k a)."""
    for q in range(1, qmax + 1):
        if float(onesided_entry_bound(float(q), q)) <= eps:
            return q
    raise ValueError("eps too small")


def xflt_alg2_onesided(c, w, eps: float, q: int | None = None):
    """The one-sided variant with exact NDFTs, f~ = (A o K~1) c; returns (f~, q).

    Z^0 rows and the Y_M band as in xflt_matrix.  For a node in Y_m, m < M,
    K~1(y, k) = sum_s L_s^{Y_m}(y) exp(-y_s k) (y_s the Chebyshev points of Y_m)
    for frequencies in Omega_l with l >= l_m, and 0 for l < l_m.
    """
    c = np.asarray(c, dtype=np.complex128)
    x, yim = _split_nodes(w)
    N = c.size
    P = xflt_params(N, eps)
    p = P.lap
    qq = rank_q_onesided(P.eps_K) if q is None else int(q)
    y = 2.0 * np.pi * yim
    kall = np.arange(N)
    z0 = y > P.y1
    K1 = np.zeros((x.size, N))
    if p.M == 1:
        K1[:] = 1.0
    else:
        by = band_of(y, P.y1, p.M)
        bk = band_of(kall.astype(np.float64), P.xi1, p.M)
        K1[by == p.M, :] = 1.0
        for m in range(1, p.M):
            rows = np.nonzero((by == m) & ~z0)[0]
            if not rows.size:
                continue
            ya, yb = band_interval(P.y1, m)
            ys = interval_points(ya, yb, qq)
            kk = np.nonzero(bk >= p.ell[m])[0]
            Ly = lagrange_barycentric(y[rows], ya, yb, qq)
            K1[np.ix_(rows, kk)] = Ly @ np.exp(-np.outer(ys, kk.astype(np.float64)))
    Cm = fourier_matrix(kall, x) * K1
    Cm[z0] = 0.0
    Cm[z0, 0] = 1.0
    return Cm @ c, qq


# --------------------------------------------------------------------------
# Generalised Algorithm 1 (Section 3, the theorem after Algorithm 1):
# asymptotically smooth kernels kappa(y, xi), all blocks Y_m x Omega_l with
# 1 <= m, l <= M - 1 interpolated (no blocks are replaced by 0 or 1), the near
# fields Y_M (every frequency) and Omega_M (every node) summed directly, and
# M = ceil(log2(y_1 xi_1 N / eps)) + 1.
#
# Asymptotic smoothness |d^q/dy^q kappa| <= C q! mu^q q^nu y^-q (y xi)^-s with
#   exp(-y xi):       C = 1,            mu = 1, nu = 0, s = 0
#                     (xi^q e^(-y xi) = y^-q (y xi)^q e^(-y xi) <= y^-q q^q e^-q <= y^-q q!);
#   K_1/2(y xi) = sqrt(pi / (2 y xi)) e^(-y xi):
#                     C = sqrt(pi/2),   mu = 1, nu = 0, s = 1/2   (the example there).
# The proof of Theorem 3.1 bounds one block by
#   C mu^q q^nu 2^(1-2q) (2 + (2/pi) ln q) (dist(A,0) dist(B,0))^-s,
# and dist(A,0) dist(B,0) >= (y_1 / 2^(M-1)) (xi_1 / 2^(M-1)) on the far field;
# q is the smallest value whose bound is <= eps.

SMOOTH_CONSTANTS = {"exp": (1.0, 1.0, 0.0, 0.0),
                    "bessel_half": (math.sqrt(math.pi / 2.0), 1.0, 0.0, 0.5)}


def smooth_kernel(kind: str, y, xi):
    """kappa(y, xi) of the generalised Algorithm 1."""
    x = np.multiply.outer(np.asarray(y, dtype=np.float64), np.asarray(xi, dtype=np.float64))
    if kind == "bessel_half":
        return np.sqrt(math.pi / (2.0 * x)) * np.exp(-x)
    if kind == "exp":
        return np.exp(-x)
    raise ValueError(kind)


def general_block_bound(kind: str, q: int, dist_product: float) -> float:
    C, mu, nu, s = SMOOTH_CONSTANTS[kind]
    return C * mu ** q * q ** nu * 2.0 ** (1 - 2 * q) * (2.0 + 2.0 / math.pi * math.log(q)) \
        * dist_product ** (-s)


@dataclass
class GeneralParams:
    kind: str
    eps: float
    y1: float
    xi1: float
    q: int
    M: int


def general_params(kind: str, eps: float, y1: float, xi1: float, N: int,
                   q: int | None = None) -> GeneralParams:
    if y1 <= 0.0 or xi1 <= 0.0 or N < 1:
        return GeneralParams(kind, eps, y1, xi1, q or 1, 1)
    M = max(1, int(math.ceil(math.log2(y1 * xi1 * N / eps))) + 1)
    if q is None:
        dmin = (y1 / 2.0 ** (M - 1)) * (xi1 / 2.0 ** (M - 1))
        q = 1
        while general_block_bound(kind, q, dmin) > eps:
            q += 1
    return GeneralParams(kind, eps, y1, xi1, int(q), M)


def general_tilde_kernel(kind: str, p: GeneralParams, t, s) -> np.ndarray:
    """Dense matrix of the generalised Algorithm 1 for kappa(s_j, t_k).

    Rows of Y_M (the near field in y) and columns of Omega_M (the near field
    in xi) hold kappa itself; every other block Y_m x Omega_l, 1 <= m, l <= M-1,
    holds its interpolant L^{Y_m} kappa(y_s, xi_r) L^{Omega_l}(xi)^T.
    """
    t = np.asarray(t, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    K = smooth_kernel(kind, s, t) if t.size and s.size else np.zeros((s.size, t.size))
    if p.M == 1 or t.size == 0:
        return K
    bt = band_of(t, p.xi1, p.M)
    bs = band_of(s, p.y1, p.M)
    cols = {l: np.nonzero(bt == l)[0] for l in range(1, p.M)}
    Lx = {l: lagrange_barycentric(t[cols[l]], *band_interval(p.xi1, l), p.q)
          for l in cols if cols[l].size}
    for m in range(1, p.M):
        rows = np.nonzero(bs == m)[0]
        if not rows.size:
            continue
        ya, yb = band_interval(p.y1, m)
        ys = interval_points(ya, yb, p.q)
        Ly = lagrange_barycentric(s[rows], ya, yb, p.q)
        for l in Lx:
            xr = interval_points(*band_interval(p.xi1, l), p.q)
            K[np.ix_(rows, cols[l])] = Ly @ smooth_kernel(kind, ys, xr) @ Lx[l].T
    return K


def laplace_alg1_general(kind: str, c, t, s, eps: float, q: int | None = None):
    """What the generalised Algorithm 1 returns, f~ = K~ c; returns (f~, params)."""
    c = np.asarray(c)
    t = np.asarray(t, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    xi1 = float(t.max()) if t.size else 0.0
    y1 = float(s.max()) if s.size else 0.0
    p = general_params(kind, eps, y1, xi1, t.size, q)
    if t.size == 0:
        return np.zeros(s.shape, dtype=np.result_type(c.dtype, np.float64)), p
    return general_tilde_kernel(kind, p, t, s) @ c, p


# --------------------------------------------------------------------------
# Real exponents (eq. 4.1 with xi_k in [1, N]): Algorithm 2 with the Fourier
# factor A = (exp(2 pi i xi_k x_j)) applied exactly (a dense NNDFT; the fast
# path uses an NNFFT).  Readings: x = Re w is taken as given (principal branch
# of z^xi: nodes with |Re w| <= 1/2, the negative real axis Re w = +-1/2 kept as
# the limit from either side), so no reduction mod 1; Z^0 nodes give 0
# (every term is below eps |c_k| there because xi_k >= 1); the frequency bands
# Omega_l and the weights W_{k,s} are those of Algorithm 2 evaluated at the
# values xi_k, with xi_1 = max xi_k.

def nndft(coef, xi, x) -> np.ndarray:
    """sum_k coef_k exp(2 pi i xi_k x_j) (dense); coef may be 2-D (k, s)."""
    xi = np.asarray(xi, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    E = np.exp(2j * np.pi * np.outer(x, xi))
    return E @ coef


def xflt_alg2_xi(c, xi, w, eps: float, q: int | None = None):
    """Algorithm 2 for real exponents xi_k >= 1 with exact NNDFTs; returns (f~, params).

    f~ = (A o K~) c with A_jk = exp(2 pi i xi_k x_j) and K~ of eq. (A.1) at
    y = 2 pi Im w_j and the values xi_k (xi_1 = max xi_k); Z^0 rows are 0.
    """
    c = np.asarray(c, dtype=np.complex128)
    xi = np.asarray(xi, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64).reshape(-1, 2)
    x, yim = w[:, 0], w[:, 1]
    eps_K = eps / 3.0
    y1 = math.log(1.0 / eps)
    xi1 = float(xi.max())
    p = laplace_params(eps_K, y1, xi1, q)
    P = XFLTParams(eps, eps_K, y1, xi1, p)
    y = 2.0 * np.pi * yim
    z0 = y > y1
    Cm = np.zeros((x.size, xi.size), dtype=np.complex128)
    keep = ~z0
    if keep.any():
        Cm[keep] = np.exp(2j * np.pi * np.outer(x[keep], xi)) * tilde_kernel(y[keep], xi, p, y1, xi1)
    return Cm @ c, P
