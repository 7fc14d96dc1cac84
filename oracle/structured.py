"""Structured reference: Algorithms 1 and 2 of Kunis & Melzer step by step (numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Tiny N only: every
block is formed as a dense matrix and the nonequispaced Fourier matrix A is
applied exactly (a dense NDFT), so what remains is the error of the
hierarchical Laplace factorisation alone.

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
# Algorithm 1: the fast discrete Laplace transform, and the dense K~ of (A.1).

def laplace_alg1(c, t, s, eps: float, q: int | None = None):
    """Algorithm 1 step by step: returns (f~, params).  Real or complex c."""
    c = np.asarray(c)
    t = np.asarray(t, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    xi1 = float(t.max()) if t.size else 0.0
    y1 = float(s.max()) if s.size else 0.0
    p = laplace_params(eps, y1, xi1, q)
    f = np.zeros(s.shape, dtype=np.result_type(c.dtype, np.float64))
    if p.M == 1:
        f[:] = c.sum()
        return f, p
    bt = band_of(t, xi1, p.M)
    bs = band_of(s, y1, p.M)
    # cumulative sums g_M .. g_1 over the frequency bands
    g = {p.M: c[bt == p.M].sum()}
    for m in range(p.M - 1, 0, -1):
        g[m] = g[m + 1] + c[bt == m].sum()
    f[bs == p.M] = g[1]
    # moments v^{Omega_l} = (L^{Omega_l})^T c^{Omega_l}
    v = {}
    for l in range(1, p.M):
        sel = bt == l
        a, b = band_interval(xi1, l)
        v[l] = lagrange_barycentric(t[sel], a, b, p.q).T @ c[sel]
    for m in range(1, p.M):
        sel = bs == m
        if not sel.any():
            continue
        h = np.zeros(p.q, dtype=f.dtype)
        for l in range(p.ell[m], p.L[m] + 1):
            h = h + kernel_block(p, m, l) @ v[l]
        a, b = band_interval(y1, m)
        f[sel] = lagrange_barycentric(s[sel], a, b, p.q) @ h + g[p.L[m] + 1]
    return f, p


def laplace_tilde_matrix(t, s, eps: float, q: int | None = None,
                         y1: float | None = None, xi1: float | None = None):
    """Dense K~ with entries defined by eq. (A.1): 1, interpolated, or 0 per block.

    Entry (j, k) approximates exp(-s_j t_k).  Rows with s_j in Y_M are all ones;
    for s_j in Y_m: columns with t_k in Omega_l, l_m <= l <= L_m, hold
    I_q^{Y_m x Omega_l} kappa; l > L_m hold 1; l < l_m hold 0.
    """
    t = np.asarray(t, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    xi1 = float(t.max()) if xi1 is None else float(xi1)
    y1 = float(s.max()) if y1 is None else float(y1)
    p = laplace_params(eps, y1, xi1, q)
    K = np.zeros((s.size, t.size))
    if p.M == 1:
        K[:] = 1.0
        return K, p
    bt = band_of(t, xi1, p.M)
    bs = band_of(s, y1, p.M)
    for j in range(s.size):
        m = bs[j]
        if m == p.M:
            K[j, :] = 1.0
            continue
        ya, yb = band_interval(y1, m)
        Ly = lagrange_barycentric(s[j], ya, yb, p.q)[0]
        for k in range(t.size):
            l = bt[k]
            if l > p.L[m]:
                K[j, k] = 1.0
            elif l >= p.ell[m]:
                xa, xb = band_interval(xi1, l)
                Lx = lagrange_barycentric(t[k], xa, xb, p.q)[0]
                K[j, k] = Ly @ kernel_block(p, m, l) @ Lx
    return K, p


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


def xflt_alg2(c, w, eps: float, q: int | None = None):
    """Algorithm 2 step by step with exact NDFTs; returns (f~, params).

    w: complex nodes in the closed upper half plane (z = exp(2 pi i w)) or an
    (M, 2) array of (Re w, Im w).
    """
    c = np.asarray(c, dtype=np.complex128)
    w = np.asarray(w)
    if not np.iscomplexobj(w):
        w = np.asarray(w, dtype=np.float64).reshape(-1, 2)
        x, yim = w[:, 0], w[:, 1]
    else:
        x, yim = w.real, w.imag
    N = c.size
    P = xflt_params(N, eps, q)
    p = P.lap
    y = 2.0 * np.pi * yim                 # the paper's y: |z| = exp(-y)
    f = np.zeros(x.shape, dtype=np.complex128)
    kall = np.arange(N)
    if N == 1:
        f[:] = c[0]
        return f, P
    z0 = y > P.y1                         # Z^0: |z| < eps  -> c_0 (index-shift reading)
    f[z0] = c[0]
    bx = np.where(z0, 0, band_of(y, P.y1, p.M))
    bk = band_of(kall.astype(np.float64), P.xi1, p.M)
    sel = bx == p.M                       # Z_M: kernel ~ 1 -> plain Fourier sum
    if sel.any():
        f[sel] = ndft(c, kall, x[sel])
    # F^_l = diag(c^l) L^{Omega_l}
    Fhat = {}
    for l in range(1, p.M):
        kl = kall[bk == l]
        a, b = band_interval(P.xi1, l)
        Fhat[l] = (c[kl][:, None] * lagrange_barycentric(kl.astype(np.float64), a, b, p.q), kl)
    for m in range(1, p.M):
        sel = bx == m
        if not sel.any():
            continue
        xm = x[sel]
        # region (iv): Omega = union of l > L_m, kernel ~ 1
        kiv = kall[bk > p.L[m]]
        fm = ndft(c[kiv], kiv, xm) if kiv.size else np.zeros(xm.size, complex)
        # interpolated blocks l_m..L_m stacked: one NDFT with q right-hand sides
        rows, ks = [], []
        for l in range(p.ell[m], p.L[m] + 1):
            Fl, kl = Fhat[l]
            if kl.size:
                rows.append(Fl @ kernel_block(p, m, l).T)
                ks.append(kl)
        if rows:
            F = ndft(np.concatenate(rows, axis=0), np.concatenate(ks), xm)
            ya, yb = band_interval(P.y1, m)
            Ly = lagrange_barycentric(y[sel], ya, yb, p.q)
            fm = fm + (Ly * F).sum(axis=1)
        f[sel] = fm
    return f, P


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
    """The one-sided variant step by step with exact NDFTs; returns (f~, q).

    Bands, Z^0 and the Y_M band as in xflt_alg2; band m < M keeps the
    frequencies of Omega_l, l >= l_m, and weights frequency k of right-hand
    side s by exp(-y_s k) at the Chebyshev points y_s of Y_m.
    """
    c = np.asarray(c, dtype=np.complex128)
    w = np.asarray(w)
    if not np.iscomplexobj(w):
        w = np.asarray(w, dtype=np.float64).reshape(-1, 2)
        x, yim = w[:, 0], w[:, 1]
    else:
        x, yim = w.real, w.imag
    N = c.size
    P = xflt_params(N, eps)
    p = P.lap
    qq = rank_q_onesided(P.eps_K) if q is None else int(q)
    y = 2.0 * np.pi * yim
    f = np.zeros(x.shape, dtype=np.complex128)
    kall = np.arange(N)
    if N == 1:
        f[:] = c[0]
        return f, qq
    z0 = y > P.y1
    f[z0] = c[0]
    bx = np.where(z0, 0, band_of(y, P.y1, p.M))
    bk = band_of(kall.astype(np.float64), P.xi1, p.M)
    sel = bx == p.M
    if sel.any():
        f[sel] = ndft(c, kall, x[sel])
    for m in range(1, p.M):
        sel = bx == m
        if not sel.any():
            continue
        ya, yb = band_interval(P.y1, m)
        ys = interval_points(ya, yb, qq)
        kk = kall[bk >= p.ell[m]]
        W = np.exp(-np.outer(kk.astype(np.float64), ys))          # (K, q)
        F = ndft(c[kk][:, None] * W, kk, x[sel])                   # (M_m, q)
        Ly = lagrange_barycentric(y[sel], ya, yb, qq)
        f[sel] = (Ly * F).sum(axis=1)
    return f, qq


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


def laplace_alg1_general(kind: str, c, t, s, eps: float, q: int | None = None):
    """The generalised Algorithm 1 step by step; returns (f~, params)."""
    c = np.asarray(c)
    t = np.asarray(t, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    xi1 = float(t.max()) if t.size else 0.0
    y1 = float(s.max()) if s.size else 0.0
    p = general_params(kind, eps, y1, xi1, t.size, q)
    f = np.zeros(s.shape, dtype=np.result_type(c.dtype, np.float64))
    if p.M == 1 or t.size == 0:
        if t.size:
            f[:] = smooth_kernel(kind, s, t) @ c
        return f, p
    bt = band_of(t, xi1, p.M)
    bs = band_of(s, y1, p.M)
    # near field in y: every frequency directly
    near_y = bs == p.M
    if near_y.any():
        f[near_y] = smooth_kernel(kind, s[near_y], t) @ c
    # moments v^{Omega_l} = (L^{Omega_l})^T c^{Omega_l}, l = 1 .. M-1
    v = {}
    for l in range(1, p.M):
        sel = bt == l
        a, b = band_interval(xi1, l)
        v[l] = lagrange_barycentric(t[sel], a, b, p.q).T @ c[sel]
    near_t = bt == p.M
    for m in range(1, p.M):
        sel = bs == m
        if not sel.any():
            continue
        ya, yb = band_interval(y1, m)
        ys = interval_points(ya, yb, p.q)
        h = np.zeros(p.q, dtype=f.dtype)
        for l in range(1, p.M):
            xa, xb = band_interval(xi1, l)
            h = h + smooth_kernel(kind, ys, interval_points(xa, xb, p.q)) @ v[l]
        fm = lagrange_barycentric(s[sel], ya, yb, p.q) @ h
        if near_t.any():   # near field in xi: directly for every node
            fm = fm + smooth_kernel(kind, s[sel], t[near_t]) @ c[near_t]
        f[sel] = fm
    return f, p


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
    """Algorithm 2 for real exponents xi_k >= 1 with exact NNDFTs; returns (f~, params)."""
    c = np.asarray(c, dtype=np.complex128)
    xi = np.asarray(xi, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64).reshape(-1, 2)
    x, yim = w[:, 0], w[:, 1]
    N = c.size
    eps_K = eps / 3.0
    y1 = math.log(1.0 / eps)
    xi1 = float(xi.max())
    p = laplace_params(eps_K, y1, xi1, q)
    P = XFLTParams(eps, eps_K, y1, xi1, p)
    y = 2.0 * np.pi * yim
    f = np.zeros(x.shape, dtype=np.complex128)
    z0 = y > y1
    bx = np.where(z0, 0, band_of(y, y1, p.M))
    bk = band_of(xi, xi1, p.M)
    sel = bx == p.M
    if sel.any():
        f[sel] = nndft(c, xi, x[sel])
    Fhat = {}
    for l in range(1, p.M):
        kl = np.nonzero(bk == l)[0]
        a, b = band_interval(xi1, l)
        Fhat[l] = (c[kl][:, None] * lagrange_barycentric(xi[kl], a, b, p.q), kl)
    for m in range(1, p.M):
        sel = bx == m
        if not sel.any():
            continue
        xm = x[sel]
        kiv = np.nonzero(bk > p.L[m])[0]
        fm = nndft(c[kiv], xi[kiv], xm) if kiv.size else np.zeros(xm.size, complex)
        rows, ks = [], []
        for l in range(p.ell[m], p.L[m] + 1):
            Fl, kl = Fhat[l]
            if kl.size:
                rows.append(Fl @ kernel_block(p, m, l).T)
                ks.append(kl)
        if rows:
            F = nndft(np.concatenate(rows, axis=0), xi[np.concatenate(ks)], xm)
            ya, yb = band_interval(y1, m)
            fm = fm + (lagrange_barycentric(y[sel], ya, yb, p.q) * F).sum(axis=1)
        f[sel] = fm
    return f, P
