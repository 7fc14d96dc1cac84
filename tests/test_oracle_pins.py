"""Pins of the plain oracle (oracle/fl_oracle.c) to things fixed by mathematics.

Each test is chosen so that a plausible slip in the oracle -- a dropped term,
a wrong sign of the phase, an index shifted by one, conj/transpose mixed up,
a wrong radial factor -- fails at least one of them:

* geometric sum c_k = 1 -> (1 - z^N) / (1 - z)            (dropped/extra term)
* equispaced nodes on |z| = 1 -> unnormalised inverse DFT  (sign, index)
* equispaced nodes on |z| = r -> DFT of c_k r^k            (radial factor)
* c = e_k -> z^k, checked in 50-digit arithmetic           (index shift)
* 50-digit brute force on tiny random inputs               (everything)
* adjoint: <C c, r> = <c, C^* r>                           (conj / transpose)
* Laplace: geometric sum and single term                   (eq. 3.2)
"""
import cmath
import math
from fractions import Fraction

import mpmath
import numpy as np
import pytest

import oracle
from paper_1606_03255_gb300 import workloads as W

U = np.finfo(np.float64).eps / 2


def _expm1_2pii(N, w):
    """expm1(2 pi i N w) for complex w, accurate near 0 (phase reduced exactly)."""
    x, v = w.real, w.imag
    a = -2.0 * math.pi * N * v
    # frac(N x) exactly in rational arithmetic, rounded once
    p = Fraction(x) * N
    fr = p - math.floor(p)
    ph = float(fr - 1 if fr >= Fraction(1, 2) else fr)   # in [-1/2, 1/2)
    th = 2.0 * math.pi * ph
    re = math.expm1(a) * math.cos(th) - 2.0 * math.sin(th / 2.0) ** 2
    im = math.exp(a) * math.sin(th)
    return complex(re, im)


def test_geometric_sum_closed_form():
    rng = np.random.default_rng(11)
    for N in (1, 2, 7, 64, 1000, 1 << 16):
        w = W.nodes_disk_uniform(40, seed=N)
        # a few nodes near z = 1 where 1 - z is tiny
        extra = np.array([[1e-7, 0.0], [0.0, 1e-9], [1 - 1e-8, 1e-10], [0.0, 0.0]])
        w = np.concatenate([w, extra])
        c = np.ones(N, dtype=np.complex128)
        f = oracle.flt_direct(c, w)
        for j, (x, v) in enumerate(w):
            wj = complex(x, v)
            if x == 0.0 and v == 0.0:
                exact = complex(N, 0)
            else:
                exact = _expm1_2pii(N, wj) / _expm1_2pii(1, wj)
            tol = 64 * U * N
            assert abs(f[j] - exact) <= tol, (N, j, f[j], exact)
    assert rng is not None


def test_equispaced_circle_is_inverse_dft():
    for N in (8, 100, 1024, 4096):
        c = W.coefficients(N, seed=3)
        w = W.nodes_equispaced_circle(N)
        f = oracle.flt_direct(c, w)
        ref = np.fft.ifft(c) * N              # sum_k c_k exp(+2 pi i jk/N)
        assert oracle.error_E(ref, f, c) < 64 * U  # roundoff of both sides
        # the conjugate convention must fail: pins the sign of the phase
        wrong = np.fft.fft(c)
        assert oracle.error_E(wrong, f, c) > 1e-3


def test_equispaced_radius_is_weighted_dft():
    N = 512
    for r in (0.9, 0.5, 0.999):
        c = W.coefficients(N, seed=5)
        w = W.nodes_equispaced_circle(N, radius=r)
        f = oracle.flt_direct(c, w)
        ref = np.fft.ifft(c * r ** np.arange(N)) * N
        assert oracle.error_E(ref, f, c) < 1e-14


def test_unit_vector_gives_power_in_50_digits():
    mpmath.mp.dps = 50
    w = W.nodes_disk_uniform(8, seed=9)
    w = np.concatenate([w, [[0.123456789, 0.0], [0.5, 0.01]]])
    for N, k in ((5, 0), (5, 4), (300, 1), (300, 299), (1 << 14, 12345)):
        c = np.zeros(N, dtype=np.complex128)
        c[k] = 1.0
        f = oracle.flt_direct(c, w)
        for j, (x, v) in enumerate(w):
            zk = mpmath.exp(2j * mpmath.pi * k * (mpmath.mpf(x) + 1j * mpmath.mpf(v)))
            assert abs(complex(zk) - f[j]) <= 8 * U, (N, k, j)


def test_random_tiny_against_50_digit_brute_force():
    mpmath.mp.dps = 40
    N, M = 48, 12
    c = W.coefficients(N, seed=21)
    w = np.concatenate([W.nodes_disk_uniform(M - 2, seed=22), [[0.3, 0.0], [0.77, 2.0]]])
    f = oracle.flt_direct(c, w)
    fld = oracle.flt_brute_ld(c, w)
    for j, (x, v) in enumerate(w):
        z = mpmath.exp(2j * mpmath.pi * (mpmath.mpf(x) + 1j * mpmath.mpf(v)))
        acc = mpmath.mpc(0)
        for k in range(N - 1, -1, -1):
            acc = acc * z + mpmath.mpc(c[k].real, c[k].imag)
        ref = complex(acc)
        assert abs(ref - f[j]) <= 16 * U * np.sum(np.abs(c))
        assert abs(ref - fld[j]) <= 16 * U * np.sum(np.abs(c))


def test_adjoint_inner_product_and_brute_force():
    N, M = 300, 200
    c = W.coefficients(N, seed=31)
    r = W.coefficients(M, seed=32)
    w = W.nodes_disk_uniform(M, seed=33)
    Cc = oracle.flt_direct(c, w)
    Chr = oracle.flt_adjoint(r, w, N)
    lhs = np.vdot(r, Cc)        # <Cc, r> = r^H C c
    rhs = np.vdot(Chr, c)       # <c, C^H r> = (C^H r)^H c
    scale = np.sum(np.abs(c)) * np.sum(np.abs(r))
    assert abs(lhs - rhs) <= 64 * U * scale
    # adjoint entries against the explicit conjugate-transpose matrix
    k = np.arange(N)
    z = np.exp(2j * np.pi * (w[:, 0] + 1j * w[:, 1]))
    C = z[:, None] ** k[None, :]
    ref = C.conj().T @ r
    assert np.max(np.abs(ref - Chr)) <= 1e-11 * np.sum(np.abs(r))
    # transposed without conjugation must fail
    assert np.max(np.abs(C.T @ r - Chr)) > 1e-3
    # the selected-frequency variant returns the same entries
    ks = np.array([0, 7, 299, 150, 7])
    assert np.array_equal(oracle.flt_adjoint_at(r, w, ks), Chr[ks])


def test_laplace_geometric_and_single_term():
    N = 2000
    h = 1e-3
    t = h * np.arange(N)
    c = np.ones(N)
    s = np.array([0.0, 1e-3, 0.5, 3.0, 100.0, 1e4])
    f = oracle.laplace_direct(c, t, s)
    for j, sj in enumerate(s):
        exact = float(N) if sj == 0 else math.expm1(-sj * N * h) / math.expm1(-sj * h)
        assert abs(f[j] - exact) <= 32 * U * N
    c1 = np.zeros(N)
    c1[1234] = 2.5
    f1 = oracle.laplace_direct(c1, t, s)
    assert np.allclose(f1, 2.5 * np.exp(-s * t[1234]), rtol=4 * U, atol=0)


def test_invalid_nodes_rejected():
    with pytest.raises(ValueError):
        oracle.flt_direct(np.ones(4), np.array([[0.1, -0.2]]))


def test_error_measure():
    c = np.array([1 + 1j, -2.0, 0.5j])
    assert oracle.error_E([1, 2], [1, 2.5], c) == pytest.approx(0.5 / (math.sqrt(2) + 2.5))
    assert cmath.isclose(1, 1)


def test_kernel_direct_pins():
    # kind "exp" is eq. (3.2) itself; "bessel_half" single terms against the
    # library Bessel function K_{1/2} and a 40-digit brute force.
    special = pytest.importorskip("scipy.special")
    mpmath = pytest.importorskip("mpmath")
    rng = np.random.default_rng(3)
    t = rng.uniform(0.01, 1.0, 50)
    s = rng.uniform(0.01, 100.0, 30)
    c = rng.standard_normal(50)
    assert np.array_equal(oracle.kernel_direct("exp", c, t, s), oracle.laplace_direct(c, t, s))
    for k in (0, 17, 49):
        e = np.zeros(50)
        e[k] = 1.0
        got = oracle.kernel_direct("bessel_half", e, t, s)
        assert np.allclose(got, special.kv(0.5, s * t[k]), rtol=1e-13, atol=0)
    mpmath.mp.dps = 40
    ref = [sum(mpmath.mpf(c[k]) * mpmath.besselk(0.5, mpmath.mpf(sj) * mpmath.mpf(t[k]))
               for k in range(50)) for sj in s[:5]]
    got = oracle.kernel_direct("bessel_half", c, t, s[:5])
    assert np.max(np.abs(got - np.array([float(r) for r in ref]))) <= 1e-13 * np.sum(np.abs(c))
    with pytest.raises(ValueError):
        oracle.kernel_direct("bessel_half", c, np.zeros(50), s)   # singular at s t = 0


def test_xi_direct_pins():
    # real exponents: integer xi_k = k + 1 reduce to z * (the integer sum); single
    # terms and a 40-digit brute force for fractional xi_k
    mpmath = pytest.importorskip("mpmath")
    rng = np.random.default_rng(11)
    N, M = 60, 25
    c = W.coefficients(N, seed=12)
    w = W.nodes_disk_uniform(M, seed=13)
    w[:, 0] -= 0.5                         # principal branch: Re w in [-1/2, 1/2)
    z = np.exp(2j * np.pi * (w[:, 0] + 1j * w[:, 1]))
    got = oracle.xi_direct(c, np.arange(N) + 1.0, w)
    assert np.max(np.abs(got - z * oracle.flt_direct(c, w))) <= 1e-13 * np.sum(np.abs(c))
    xi = np.sort(rng.uniform(1.0, N, N))
    mpmath.mp.dps = 40
    two_pi_i = 2j * mpmath.pi
    ref = []
    for j in range(M):
        wj = mpmath.mpc(w[j, 0], w[j, 1])
        ref.append(complex(sum(mpmath.mpc(c[k].real, c[k].imag) * mpmath.exp(two_pi_i * mpmath.mpf(xi[k]) * wj)
                               for k in range(N))))
    got = oracle.xi_direct(c, xi, w)
    assert np.max(np.abs(got - np.array(ref))) <= 1e-14 * np.sum(np.abs(c))
    with pytest.raises(ValueError):
        oracle.xi_direct(c, -xi, w)


def test_xi_transposed_pins():
    # the transposed real-exponent sum g_k = sum_j h_j z_j^{xi_k}:
    # (1) integer exponents xi_k = k give conj(C^* conj h), the independently
    #     written adjoint; (2) the bilinear identity h . (C c) = (C^T h) . c with
    #     the pinned forward sum; (3) a 40-digit brute force at fractional xi_k
    rng = np.random.default_rng(21)
    N, M = 50, 30
    h = W.targets(M, seed=22)
    w = W.nodes_disk_uniform(M, seed=23)
    w[:, 0] -= 0.5
    got = oracle.xi_transposed(h, np.arange(N, dtype=np.float64), w)
    ref = np.conj(oracle.flt_adjoint(np.conj(h), w, N))
    assert np.max(np.abs(got - ref)) <= 1e-14 * np.sum(np.abs(h))
    xi = np.sort(rng.uniform(1.0, N, N))
    c = W.coefficients(N, seed=24)
    lhs = np.dot(h, oracle.xi_direct(c, xi, w))
    rhs = np.dot(oracle.xi_transposed(h, xi, w), c)
    assert abs(lhs - rhs) <= 1e-13 * np.sum(np.abs(h)) * np.sum(np.abs(c))
    mpmath.mp.dps = 40
    two_pi_i = 2j * mpmath.pi
    brute = []
    for k in range(N):
        brute.append(complex(sum(mpmath.mpc(h[j].real, h[j].imag) *
                                 mpmath.exp(two_pi_i * mpmath.mpf(xi[k]) * mpmath.mpc(w[j, 0], w[j, 1]))
                                 for j in range(M))))
    got = oracle.xi_transposed(h, xi, w)
    assert np.max(np.abs(got - np.array(brute))) <= 1e-14 * np.sum(np.abs(h))
    with pytest.raises(ValueError):
        oracle.xi_transposed(h, -xi, w)
    with pytest.raises(ValueError):
        oracle.xi_transposed(h[:-1], xi, w)
