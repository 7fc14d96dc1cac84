"""Pins of the structured reference (oracle/structured.py): Algorithms 1 and 2.

What the paper fixes and is checked here:

* Section 2: the barycentric formula equals the product form; partition of
  unity; L_r(y_s) = delta_rs; exact interpolation of polynomials of degree < q.
* Lemma A.1: every interpolated kernel entry is within 2^(1-2q) of exp(-y xi);
  Lemma A.2 (i), (ii), (iv): the entries set to 1 or 0 are within eps.
* K~ of eq. (A.1) reproduces exp(-y xi) exactly where both y and xi are
  Chebyshev points of their bands (the Kronecker property through
  Definition 3.2's blocks; a transposed coupling block fails it), and
  Theorem A.3: ||f - f~||_inf <= eps ||c||_1 against the plain oracle.
* Section 5 experiment shape: E(q) decays faster than 4^(-q).
* Lemma 4.2 (Hadamard identity) on random dense matrices, to roundoff.
* Theorem 4.3 / Algorithm 2 (exact NDFT): E <= eps against the plain oracle;
  Z^0 nodes return c_0; nodes on |z| = 1 reduce to the DFT.
* One-sided variant (interpolation in y only, first term of the proof of
  Theorem 3.1): every entry within the bound 2 (ka/4)^q e^-ka / q! of the
  error formula of Section 2 (checked on a dense y grid); the rank rule is the
  smallest q whose bound, maximised over ka by brute force, is <= eps/3;
  E <= eps on three node distributions; E decreases with q.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import structured as S
from paper_1606_03255_gb300 import workloads as W


@pytest.mark.parametrize("q", [1, 2, 5, 12, 22])
def test_barycentric_matches_product_form_and_unity(q):
    rng = np.random.default_rng(q)
    a, b = 0.37, 0.74
    y = a + (b - a) * rng.random(200)
    Lb = S.lagrange_barycentric(y, a, b, q)
    Lp = S.lagrange_product(y, a, b, q)
    assert np.max(np.abs(Lb - Lp)) < 1e-12 * max(1, q)
    assert np.max(np.abs(Lb.sum(axis=1) - 1.0)) < 1e-13
    nodes = S.interval_points(a, b, q)
    assert np.array_equal(S.lagrange_barycentric(nodes, a, b, q), np.eye(q))


def test_interpolation_is_exact_on_low_degree_polynomials():
    q = 9
    a, b = 2.0, 4.0
    rng = np.random.default_rng(0)
    coef = rng.standard_normal(q)            # degree q-1
    y = a + (b - a) * rng.random(100)
    nodes = S.interval_points(a, b, q)
    vals = np.polyval(coef, nodes)
    interp = S.lagrange_barycentric(y, a, b, q) @ vals
    assert np.max(np.abs(interp - np.polyval(coef, y))) < 1e-11 * np.max(np.abs(vals))
    # degree q is not reproduced
    coef2 = np.concatenate([[1.0], np.zeros(q)])
    interp2 = S.lagrange_barycentric(y, a, b, q) @ np.polyval(coef2, nodes)
    assert np.max(np.abs(interp2 - np.polyval(coef2, y))) > 1e-6


def test_definition_parameters_hand_computed():
    # q = ceil(1/2 + log_4(1/eps))
    assert S.rank_q(1e-6) == 11 and S.rank_q(1e-6 / 3) == 12
    assert S.rank_q(1e-12 / 3) == 22 and S.rank_q(1e-10 / 3) == 18
    assert S.rank_q(2.0 ** (1 - 2 * 7)) == 7
    # y1 * xi1 = 2^10, eps = 2^-10: M = ceil(log2(2^20)) + 1 = 21
    p = S.laplace_params(2.0 ** -10, 32.0, 32.0)
    assert p.M == 21
    # l_m = max(1, floor(10 - m - log2(ln 2^10)) + 1); log2(6.931...) = 2.79...
    for m in range(1, p.M):
        assert p.ell[m] == max(1, math.floor(10 - m - math.log2(10 * math.log(2))) + 1)
        assert p.L[m] == 21 - m
    assert p.ell[1] == 7 and p.ell[6] == 2 and p.ell[7] == 1


def test_band_assignment_edges():
    M = 6
    v1 = 10.0
    v = np.array([10.0, 5.0000001, 5.0, 2.5, 1e-9, 0.0, 10.0 / 32, 10.0 / 32 * 1.0000001])
    b = S.band_of(v, v1, M)
    # (5, 10] -> 1 ; (2.5, 5] -> 2 ; (1.25, 2.5] -> 3 ; ... [0, 10/32] -> 6
    assert list(b) == [1, 1, 2, 3, 6, 6, 6, 5]


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-9])
def test_kernel_entries_meet_lemma_bounds(eps):
    rng = np.random.default_rng(7)
    t = np.sort(rng.random(300))[::-1] * 3.0
    s = np.sort(rng.random(200))[::-1] * 500.0
    K, p = S.laplace_tilde_matrix(t, s, eps)
    exact = np.exp(-np.outer(s, t))
    bt = S.band_of(t, p.xi1, p.M)
    bs = S.band_of(s, p.y1, p.M)
    err = np.abs(K - exact)
    for j in range(s.size):
        m = bs[j]
        for k in range(t.size):
            l = bt[k]
            if m < p.M and p.ell[m] <= l <= p.L[m]:
                assert err[j, k] <= 2.0 ** (1 - 2 * p.q) + 1e-15      # Lemma A.1
            else:
                assert err[j, k] <= eps                                # Lemma A.2
    assert err.max() <= eps


@pytest.mark.parametrize("eps", [1e-4, 1e-6, 1e-10])
def test_algorithm1_meets_theorem(eps):
    c, t, s = W.laplace_inputs(400, 300, seed=4)
    f_alg, p = S.laplace_alg1(c, t, s, eps)
    f = oracle.laplace_direct(c, t, s)
    assert oracle.error_E(f, f_alg, c) <= eps                          # Theorem A.3


def test_tilde_blocks_interpolate_at_chebyshev_points():
    # nodes and frequencies placed on the Chebyshev points of their bands: every
    # interpolated entry of K~ is then exp(-y_s xi_r) itself (L_r(y_s) = delta_rs)
    eps, y1, xi1 = 1e-6, 400.0, 3.0
    p = S.laplace_params(eps, y1, xi1)
    ys, xs = [y1], [xi1]
    for m in (2, 5, 9):
        ys += list(S.interval_points(*S.band_interval(y1, m), p.q)[[0, 3, p.q - 1]])
    for l in range(1, p.M):
        xs += list(S.interval_points(*S.band_interval(xi1, l), p.q)[[1, p.q - 2]])
    ys, xs = np.array(ys), np.array(xs)
    K, _ = S.laplace_tilde_matrix(xs, ys, eps, y1=y1, xi1=xi1)
    by, bx = S.band_of(ys, y1, p.M), S.band_of(xs, xi1, p.M)
    exact = np.exp(-np.outer(ys, xs))
    n = 0
    for j in range(ys.size):
        for k in range(xs.size):
            m, l = by[j], bx[k]
            if m < p.M and p.ell[m] <= l <= p.L[m] and j > 0 and k > 0:
                assert abs(K[j, k] - exact[j, k]) <= 1e-15 * exact[j, k] + 1e-300, (m, l)
                n += 1
    assert n >= 20


def test_algorithm1_error_decays_faster_than_4_to_minus_q():
    # Section 5 workload shape (smaller N): y in [0, (2q-1) ln 2] is the paper's
    # choice; here nodes fill [0, 2N] and [0, 1] as in the Laplace config.
    c, t, s = W.laplace_inputs(2048, 512, seed=8)
    f = oracle.laplace_direct(c, t, s)
    qs = np.arange(2, 11)
    Es = []
    for q in qs:
        eps = 2.0 ** (1 - 2 * q)                 # so that rank_q(eps) == q
        assert S.rank_q(eps) == q
        fa, _ = S.laplace_alg1(c, t, s, eps)
        Es.append(oracle.error_E(f, fa, c))
        assert Es[-1] <= eps
    slope = np.polyfit(qs, np.log(np.maximum(Es, 1e-300)), 1)[0]
    assert -slope > math.log(4.0), (Es, slope)


def test_hadamard_identity_lemma_4_2():
    rng = np.random.default_rng(1)
    p_, n_, q = 17, 23, 5
    LY = rng.standard_normal((p_, q))
    KYO = rng.standard_normal((q, q))
    LO = rng.standard_normal((n_, q))
    A = rng.standard_normal((p_, n_)) + 1j * rng.standard_normal((p_, n_))
    f = rng.standard_normal(n_) + 1j * rng.standard_normal(n_)
    lhs = (A * (LY @ KYO @ LO.T)) @ f
    rhs = (LY * (A @ np.diag(f) @ LO @ KYO.T)) @ np.ones(q)
    assert np.max(np.abs(lhs - rhs)) < 1e-12 * np.max(np.abs(lhs))
    # the transposed coupling block is not the same thing
    bad = (LY * (A @ np.diag(f) @ LO @ KYO)) @ np.ones(q)
    assert np.max(np.abs(lhs - bad)) > 1e-3


@pytest.mark.parametrize("eps", [1e-4, 1e-6, 1e-10])
@pytest.mark.parametrize("kind", ["disk", "clustered", "paper"])
def test_algorithm2_meets_theorem(eps, kind):
    N, M = 512, 256
    c = W.coefficients(N, seed=12)
    if kind == "disk":
        w = W.nodes_disk_uniform(M, seed=13)
    elif kind == "clustered":
        w = W.nodes_circle_clustered(M, seed=14)
    else:
        w = W.nodes_paper_section5(M, S.rank_q(eps), seed=15)
    f = oracle.flt_direct(c, w)
    fa, P = S.xflt_alg2(c, w, eps)
    assert oracle.error_E(f, fa, c) <= eps


def test_algorithm2_special_cases():
    N = 256
    c = W.coefficients(N, seed=2)
    # all nodes on the unit circle, equispaced: Z_M band only -> DFT
    w = W.nodes_equispaced_circle(N)
    fa, P = S.xflt_alg2(c, w, 1e-8)
    assert oracle.error_E(np.fft.ifft(c) * N, fa, c) < 1e-14
    # Z^0 nodes: |z| < eps -> exactly c_0
    w0 = np.array([[0.25, 5.0], [0.6, 3.0]])          # |z| = e^{-10 pi}, e^{-6 pi}
    f0, _ = S.xflt_alg2(c, w0, 1e-6)
    assert np.array_equal(f0, np.full(2, c[0]))
    # N = 1: f = c_0 everywhere
    f1, _ = S.xflt_alg2(c[:1], W.nodes_disk_uniform(5, 0), 1e-6)
    assert np.array_equal(f1, np.full(5, c[0]))


# --------------------------------------------------------------------------
# One-sided variant

@pytest.mark.parametrize("q", [4, 8, 10, 14])
def test_onesided_entries_within_interpolation_bound(q):
    y1 = math.log(1e6)
    for m in (3, 9, 17):
        a, b = S.band_interval(y1, m)
        ys = S.interval_points(a, b, q)
        yg = np.linspace(a, b, 2001)
        L = S.lagrange_barycentric(yg, a, b, q)
        for ka in (0.1, 1.0, q / 2.0, float(q), 2.0 * q, 40.0):
            k = ka / a
            err = np.max(np.abs(np.exp(-yg * k) - L @ np.exp(-ys * k)))
            assert err <= float(S.onesided_entry_bound(ka, q)) * (1 + 1e-9) + 1e-15, (m, ka, err)
            if ka == 1.0 and q <= 10:
                # for small k a the derivative bound is nearly attained: the
                # formula's constant is not loose by more than a small factor
                assert err >= float(S.onesided_entry_bound(ka, q)) / 3.0, (m, q, err)


def test_onesided_rank_rule_by_brute_force():
    kag = np.linspace(0.0, 200.0, 400001)
    for eps in (1e-3, 1e-6 / 3, 1e-10 / 3, 1e-12 / 3):
        q = S.rank_q_onesided(eps)
        worst = lambda qq: float(np.max(S.onesided_entry_bound(kag, qq)))
        assert worst(q) <= eps * (1 + 1e-6)
        assert worst(q - 1) > eps
    assert S.rank_q_onesided(1e-6 / 3) == 10 and S.rank_q_onesided(1e-12 / 3) == 20


@pytest.mark.parametrize("eps", [1e-4, 1e-6, 1e-10])
@pytest.mark.parametrize("kind", ["disk", "clustered", "paper"])
def test_onesided_meets_eps(eps, kind):
    N, M = 512, 256
    c = W.coefficients(N, seed=22)
    if kind == "disk":
        w = W.nodes_disk_uniform(M, seed=23)
    elif kind == "clustered":
        w = W.nodes_circle_clustered(M, seed=24)
    else:
        w = W.nodes_paper_section5(M, S.rank_q(eps), seed=25)
    f = oracle.flt_direct(c, w)
    fa, q = S.xflt_alg2_onesided(c, w, eps)
    assert q == S.rank_q_onesided(eps / 3)
    assert oracle.error_E(f, fa, c) <= eps


def test_onesided_error_decreases_with_q():
    N, M = 400, 300
    c = W.coefficients(N, seed=31)
    w = W.nodes_disk_uniform(M, seed=32)
    f = oracle.flt_direct(c, w)
    errs = [oracle.error_E(f, S.xflt_alg2_onesided(c, w, 1e-12, q=q)[0], c) for q in (3, 5, 7, 9)]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    # Z^0 and the Y_M band are those of Algorithm 2
    w0 = np.array([[0.25, 5.0], [0.5, 0.0]])
    f0, _ = S.xflt_alg2_onesided(c, w0, 1e-6)
    assert f0[0] == c[0]
    assert abs(f0[1] - np.sum(c * (-1.0) ** np.arange(N))) < 1e-12 * np.sum(np.abs(c))


# --------------------------------------------------------------------------
# Generalised Algorithm 1 (asymptotically smooth kernels)

def test_bessel_half_kernel_closed_form():
    special = pytest.importorskip("scipy.special")
    x = np.geomspace(1e-6, 50.0, 200)
    got = S.smooth_kernel("bessel_half", x, np.ones(1))[:, 0]
    assert np.allclose(got, special.kv(0.5, x), rtol=1e-13, atol=0)
    # the Laplace kernel of the generalised algorithm is the plain exponential
    assert np.array_equal(S.smooth_kernel("exp", x, np.ones(1))[:, 0], np.exp(-x))


def test_bessel_half_derivative_identity_and_smoothness():
    sympy = pytest.importorskip("sympy")
    y, xi = sympy.symbols("y xi", positive=True)
    kappa = sympy.sqrt(sympy.pi / (2 * y * xi)) * sympy.exp(-y * xi)
    for q in range(0, 7):
        d = sympy.diff(kappa, y, q)
        # the identity of the example: sqrt(pi/2) (-xi)^q e^(-y xi)
        #   * sum_k binom(q,k) prod_{j<k} (2j+1) / 2^k (y xi)^(-(2k+1)/2)
        ident = sympy.sqrt(sympy.pi / 2) * (-xi) ** q * sympy.exp(-y * xi) * sum(
            sympy.binomial(q, k) * sympy.prod([2 * j + 1 for j in range(k)]) / 2 ** k
            * (y * xi) ** (-sympy.Rational(2 * k + 1, 2)) for k in range(q + 1))
        for yv, xv in ((0.3, 2.0), (1.7, 0.25), (5.0, 3.0)):
            dv = float(d.subs({y: yv, xi: xv}))
            iv = float(ident.subs({y: yv, xi: xv}))
            assert abs(dv - iv) <= 1e-12 * max(1.0, abs(dv))
            # asymptotic smoothness: C = sqrt(pi/2), mu = 1, nu = 0, s = 1/2
            bound = math.sqrt(math.pi / 2) * math.factorial(q) * (yv * xv) ** -0.5 * yv ** -q
            assert abs(dv) <= bound * (1 + 1e-12)


@pytest.mark.parametrize("kind", ["exp", "bessel_half"])
def test_general_blocks_within_bound(kind):
    # every interpolated block of a small partition, checked on a dense grid
    q = 8
    P = S.general_params(kind, 1e-6, 40.0, 1.0, 64, q=q)
    dmin = (P.y1 / 2.0 ** (P.M - 1)) * (P.xi1 / 2.0 ** (P.M - 1))
    bound = S.general_block_bound(kind, q, dmin)
    worst = 0.0
    for m in (1, 5, P.M - 1):
        ya, yb = S.band_interval(P.y1, m)
        yg = np.linspace(ya, yb, 60)
        Ly = S.lagrange_barycentric(yg, ya, yb, q)
        ys = S.interval_points(ya, yb, q)
        for l in (1, 7, P.M - 1):
            xa, xb = S.band_interval(P.xi1, l)
            xg = np.linspace(xa, xb, 60)
            Lx = S.lagrange_barycentric(xg, xa, xb, q)
            xs = S.interval_points(xa, xb, q)
            approx = Ly @ S.smooth_kernel(kind, ys, xs) @ Lx.T
            err = np.max(np.abs(S.smooth_kernel(kind, yg, xg) - approx))
            local = S.general_block_bound(kind, q, ya * xa)
            assert err <= local * (1 + 1e-9) + 1e-14, (m, l, err, local)
            worst = max(worst, err)
    assert worst <= bound


@pytest.mark.parametrize("kind", ["exp", "bessel_half"])
@pytest.mark.parametrize("eps", [1e-4, 1e-6, 1e-10])
def test_general_algorithm1_meets_eps(kind, eps):
    rng = np.random.default_rng(7)
    N, M = 700, 400
    t = rng.uniform(0.0, 1.0, N)
    s = rng.uniform(0.0, 2.0 * N, M)
    # near fields: a few t in Omega_M and s in Y_M (tiny but positive)
    t[:3] = [1e-12, 3e-13, 1e-11]
    s[:3] = [1e-9, 2e-10, 5e-9]
    t[t == 0] = 0.5
    s[s == 0] = 1.0
    c = rng.standard_normal(N)
    f, P = S.laplace_alg1_general(kind, c, t, s, eps)
    assert P.M == int(math.ceil(math.log2(s.max() * t.max() * N / eps))) + 1
    ref = oracle.kernel_direct(kind, c, t, s)
    # Theorem (generalised Algorithm 1): E <= eps in exact arithmetic.  Both
    # sides round sums whose terms reach |c_k kappa| ~ 1e10 next to the
    # singularity (s t ~ 1e-21 in the near fields), so rounding of order
    # u * sum_k |c_k kappa(s_j, t_k)| is allowed on top.
    absum = np.abs(S.smooth_kernel(kind, s, t)) @ np.abs(c)
    allow = 64 * 2.0 ** -53 * np.max(absum)
    assert np.max(np.abs(f - ref)) <= eps * np.sum(np.abs(c)) + allow
    # the generalised algorithm on exp(-s t) agrees with Algorithm 1
    if kind == "exp":
        f1, _ = S.laplace_alg1(c, t, s, eps)
        assert np.max(np.abs(f - f1)) <= 2 * eps * np.sum(np.abs(c))


# --------------------------------------------------------------------------
# Real exponents (eq. 4.1 with xi_k in [1, N]) with exact NNDFTs

@pytest.mark.parametrize("eps", [1e-4, 1e-6, 1e-10])
@pytest.mark.parametrize("kind", ["disk", "clustered", "integer"])
def test_algorithm2_real_exponents_meets_eps(eps, kind):
    rng = np.random.default_rng(41)
    N, M = 500, 300
    c = W.coefficients(N, seed=42)
    xi = np.arange(N) + 1.0 if kind == "integer" else np.sort(rng.uniform(1.0, N, N))
    w = (W.nodes_circle_clustered(M, seed=43) if kind == "clustered"
         else W.nodes_disk_uniform(M, seed=44)).copy()
    w[:, 0] -= 0.5
    w = np.concatenate([w, [[0.1, 4.0], [-0.5, 0.0], [0.5, 0.3]]])   # Z^0 node, branch edges
    ref = oracle.xi_direct(c, xi, w)
    f, P = S.xflt_alg2_xi(c, xi, w, eps)
    assert oracle.error_E(ref, f, c) <= eps
    assert f[M] == 0                                   # Z^0 -> 0 (xi_k >= 1)
