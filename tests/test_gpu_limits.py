"""GPU parity at the largest sizes each plan call accepts.

* fl_plan at N = 2^23 (its limit): the full-bandwidth bands use the largest
  grids, 2^24 points, i.e. both four-step passes at 2^12; FP32 at eps = 1e-6
  and the float-pair FP64-accuracy form at eps = 1e-12, on clustered nodes;
* fl_plan_xi at N = 2^22 (its limit), FP32;
* Laplace at N = M = 2^22.
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
