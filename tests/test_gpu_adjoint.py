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


def _transposed_definition(g, w, N):
    """g_k = sum_j g_j exp(2 pi i k w_j) by the definition (small sizes), with the
    phase k Re w reduced mod 1 before the exponential."""
    k = np.arange(N, dtype=np.float64)[:, None]
    x, y = w[:, 0][None, :], w[:, 1][None, :]
    ph = k * x
    ph = ph - np.floor(ph)
    return (np.exp(-2 * np.pi * k * y) * np.exp(2j * np.pi * ph)) @ g


@pytest.mark.parametrize("prec,eps", [("fp64", 1e-12), ("fp32", 1e-6)])
@pytest.mark.parametrize("variant", ["alg2", "onesided"])
@pytest.mark.parametrize("N,M,kind", [(700, 500, "disk"), (9000, 800, "clustered"), (1, 5, "disk")])
def test_transposed_evaluation(fl, prec, eps, variant, N, M, kind):
    # remark after Algorithm 2: g(xi) = sum_j ghat_j z_j^xi at xi = 0 .. N-1
    w = W.nodes_disk_uniform(M, seed=3) if kind == "disk" else W.nodes_circle_clustered(M, seed=3)
    g = W.coefficients(M, seed=4)
    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    plan = fl.Plan(N, torch.from_numpy(w).cuda(), eps, precision=prec, variant=variant)
    out = plan.transposed(torch.from_numpy(g).to(cdt).cuda()).cpu().numpy().astype(np.complex128)
    plan.close()
    ref = _transposed_definition(g, w, N)
    # the same number through the oracle's adjoint: C^T g = conj(C^* conj(g))
    ref2 = np.conj(oracle.flt_adjoint(np.conj(g), w, N))
    assert np.max(np.abs(ref - ref2)) <= 1e-12 * np.sum(np.abs(g))
    bound = eps if prec == "fp64" else eps + 32 * 2.0 ** -24 * np.max(np.abs(ref)) / np.sum(np.abs(g))
    assert oracle.error_E(ref, out, g) <= bound
