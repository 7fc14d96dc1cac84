"""GPU parity of the adjoint C^* r (Section 4, remark after Algorithm 2)."""
import numpy as np
import pytest

import oracle
from paper_1606_03255_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fl():
    from paper_1606_03255_gb300 import build as libbuild
    libbuild.build()
    from paper_1606_03255_gb300 import fl as flmod
    flmod.load()
    return flmod


def _adjoint(fl, r, w, N, eps, prec, route="nfft"):
    dev = torch.device("cuda")
    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    plan = fl.Plan(N, torch.from_numpy(w).to(dev), eps, precision=prec, route=route)
    g = plan.adjoint(torch.from_numpy(r).to(cdt).to(dev))
    torch.cuda.synchronize()
    plan.close()
    return g.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("N,M", [(1, 4), (64, 100), (1000, 1000), (5000, 3000), (20000, 1500)])
@pytest.mark.parametrize("prec,eps", [("fp64", 1e-12), ("fp32", 1e-6)])
@pytest.mark.parametrize("kind", ["disk", "clustered"])
@pytest.mark.parametrize("route", ["nfft", "auto", "direct"])
def test_adjoint_against_oracle(fl, N, M, prec, eps, kind, route):
    w = W.nodes_disk_uniform(M, seed=M) if kind == "disk" else W.nodes_circle_clustered(M, seed=M)
    w = np.concatenate([w, [[0.5, 9.0]]])        # one Z^0 node
    r = W.coefficients(M + 1, seed=N)
    g = _adjoint(fl, r, w, N, eps, prec, route)
    ref = oracle.flt_adjoint(r, w, N)
    E = oracle.error_E(ref, g, r)
    bound = eps if prec == "fp64" else eps + 32 * 2.0 ** -24 * np.max(np.abs(ref)) / np.sum(np.abs(r))
    assert E <= bound, E


def test_adjoint_inner_product(fl):
    N, M, eps = 3000, 2000, 1e-12
    dev = torch.device("cuda")
    c = W.coefficients(N, seed=1)
    r = W.coefficients(M, seed=2)
    w = W.nodes_disk_uniform(M, seed=3)
    plan = fl.Plan(N, torch.from_numpy(w).to(dev), eps, precision="fp64")
    f = plan.execute(torch.from_numpy(c).to(dev)).cpu().numpy()
    g = plan.adjoint(torch.from_numpy(r).to(dev)).cpu().numpy()
    plan.close()
    lhs, rhs = np.vdot(r, f), np.vdot(g, c)
    assert abs(lhs - rhs) <= 4 * eps * np.sum(np.abs(c)) * np.sum(np.abs(r))
