"""GPU parity at the largest sizes each plan call accepts.

* fl_plan at N = 2^23 (its limit): the full-bandwidth bands use the largest
  grids, 2^24 points, i.e. both four-step passes at 2^12; FP32 at eps = 1e-6
  and the float-pair FP64-accuracy form at eps = 1e-12, on clustered nodes;
* fl_plan_xi at N = 2^22 (its limit), FP32;
* Laplace at N = M = 2^22;
* real exponents in FP64 at N = 2^22 with data coherent at one node, where
  the band-centre phase must keep the full double precision.
Every result is checked against the oracle on a seeded sample of outputs
(the oracle sums all N terms for each sampled node), with the same bounds as
the smaller parity tests.
"""
import numpy as np
import pytest

import oracle
from paper_1606_03255_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def fl():
    from paper_1606_03255_gb300 import build as libbuild
    libbuild.build()
    from paper_1606_03255_gb300 import fl as flmod
    flmod.load()
    return flmod


@pytest.mark.parametrize("prec,eps", [("fp32", 1e-6), ("fp64ff", 1e-12)])
def test_forward_at_max_N(fl, prec, eps):
    N, M = 1 << 23, 1 << 18
    c = W.coefficients(N, seed=1)
    w = W.nodes_circle_clustered(M, seed=2)
    cdt = torch.complex64 if prec == "fp32" else torch.complex128
    p = fl.Plan(N, torch.from_numpy(w).cuda(), eps, precision=prec)
    info = p.info()
    assert max(info["band_n"]) == 1 << 24
    f = p.execute(torch.from_numpy(c).to(cdt).cuda()).cpu().numpy().astype(np.complex128)
    p.close()
    idx = np.random.default_rng(3).choice(M, 96, replace=False)
    cref = c.astype(np.complex64).astype(np.complex128) if prec == "fp32" else c
    ref = oracle.flt_direct(cref, w[idx])
    bound = eps if prec != "fp32" else eps + 32 * U32 * np.max(np.abs(ref)) / np.sum(np.abs(cref))
    assert oracle.error_E(ref, f[idx], cref) <= bound


def test_xi_at_max_N(fl):
    N, M = 1 << 22, 1 << 16
    rng = np.random.default_rng(4)
    xi = rng.uniform(1.0, N, N)
    c = W.coefficients(N, seed=5).astype(np.complex64).astype(np.complex128)
    w = W.nodes_circle_clustered(M, seed=6).copy()
    w[:, 0] -= 0.5
    p = fl.XiPlan(torch.from_numpy(xi).cuda(), torch.from_numpy(w).cuda(), 1e-6, precision="fp32")
    f = p.execute(torch.from_numpy(c).to(torch.complex64).cuda()).cpu().numpy().astype(np.complex128)
    p.close()
    idx = np.random.default_rng(7).choice(M, 64, replace=False)
    ref = oracle.xi_direct(c, xi, w[idx])
    bound = 1e-6 + 32 * U32 * np.max(np.abs(ref)) / np.sum(np.abs(c))
    assert oracle.error_E(ref, f[idx], c) <= bound


def test_laplace_large(fl):
    N = M = 1 << 22
    c, t, s = W.laplace_inputs(N, M, seed=8)
    p = fl.LaplacePlan(torch.from_numpy(t).cuda(), torch.from_numpy(s).cuda(), 1e-10, precision="fp64")
    f = p.execute(torch.from_numpy(c).cuda()).cpu().numpy()
    p.close()
    idx = np.random.default_rng(9).choice(M, 256, replace=False)
    ref = oracle.laplace_direct(c, t, s[idx])
    assert np.max(np.abs(ref - f[idx])) <= 1e-10 * np.sum(np.abs(c))


def _phase_sensitive_node(xi, rng):
    """Re w in [1/4, 1/2) whose product with the last band's centre xc
    (2 xc = floor(min xi + max xi)) loses nearly half an ulp when rounded to
    double, so an epilogue exp(2 pi i xc x) formed from the rounded product is
    off by almost 2 pi ulp / 2 radians."""
    from fractions import Fraction
    xc = 0.5 * np.floor(xi.min() + xi.max())
    best, dbest = 0.0, 0.0
    for x in rng.uniform(0.25, 0.5, 400):
        d = abs(float(Fraction(xc) * Fraction(float(x)) - Fraction(xc * float(x))))
        if d > dbest:
            best, dbest = float(x), d
    return best, dbest


def test_xi_fp64_epilogue_phase_at_max_N(fl):
    # Real exponents in FP64 at N = 2^22, eps = 1e-10, with the data made
    # coherent at one node on |z| = 1: c_k = exp(-2 pi i xi_k x0) gives
    # |f(z0)| = ||c||_1 and, transposed, h = e_0 gives |g_k| = ||h||_1, so the
    # centre phase xc x0 (xc ~ 2^21) must carry the full double precision.
    N, M, eps = 1 << 22, 64, 1e-10
    rng = np.random.default_rng(51)
    xi = rng.uniform(1.0, N, N)
    x0, dphase = _phase_sensitive_node(xi, rng)
    assert 2 * np.pi * dphase >= 3 * eps        # a rounded product would fail
    w = np.zeros((M, 2))
    w[:, 0] = rng.uniform(-0.5, 0.5, M)
    w[0, 0] = x0
    c = np.exp(-2j * np.pi * np.mod(xi * x0, 1.0))
    h = np.zeros(M, dtype=np.complex128)
    h[0] = 1.0
    p = fl.XiPlan(torch.from_numpy(xi).cuda(), torch.from_numpy(w).cuda(), eps, precision="fp64")
    f = p.execute(torch.from_numpy(c).cuda()).cpu().numpy()
    g = p.transposed(torch.from_numpy(h).cuda()).cpu().numpy()
    p.close()
    ref = oracle.xi_direct(c, xi, w)
    assert abs(ref[0]) >= 0.999 * N
    assert oracle.error_E(ref, f, c) <= eps
    gref = oracle.xi_transposed(h, xi, w)
    assert np.max(np.abs(gref - g)) <= eps * np.sum(np.abs(h))
