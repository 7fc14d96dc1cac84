"""GPU parity of real exponents (fl_plan_xi): f_j = sum_k c_k exp(2 pi i xi_k w_j).

Algorithm 2 with the exponent values xi_k >= 1 and an NNFFT per band
(frequency spreading on a grid of spacing 1/2, NFFT at x/2, division by the
window's transform), through the C ABI:
* E <= eps (FP64) or eps + 32 u_32 ||f||_inf / ||c||_1 (FP32) against the
  plain oracle, for random and integer exponents, disk and clustered nodes with
  |Re w| <= 1/2, a Z^0 node (-> 0) and the branch edges Re w = +-1/2;
* integer exponents xi_k = k + 1 agree with z times the integer transform;
* the GPU result differs from the structured reference (exact NNDFTs) by at
  most the NNFFT share eps/3;
* the adjoint and the transposed evaluation g_k = sum_j ghat_j z_j^{xi_k}
  (remark after Algorithm 2 at real exponents) against the plain oracle sum
  over nodes, max_k |g_k - g~_k| <= eps sum_j |ghat_j| (FP64; the FP32 bound
  adds the same rounding term), and the inner-product identity;
* invalid exponents and nodes are rejected.
"""
import numpy as np
import pytest

import oracle
from oracle import structured as S
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


def _tol(eps, prec, ref, c):
    if prec == "fp64":
        return eps
    return eps + 32 * U32 * np.max(np.abs(ref)) / np.sum(np.abs(c))


def _nodes(kind, M, seed):
    w = (W.nodes_circle_clustered(M, seed) if kind == "clustered" else W.nodes_disk_uniform(M, seed)).copy()
    w[:, 0] -= 0.5                               # principal branch: Re w in [-1/2, 1/2)
    return np.concatenate([w, [[0.1, 9.0], [-0.5, 0.0], [0.5, 0.01]]])   # Z^0, branch edges


def _run(fl, c, xi, w, eps, prec, q=0):
    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    p = fl.XiPlan(torch.from_numpy(xi).cuda(), torch.from_numpy(w).cuda(), eps, precision=prec, q=q)
    f = p.execute(torch.from_numpy(c).to(cdt).cuda()).cpu().numpy().astype(np.complex128)
    info = p.info()
    p.close()
    return f, info


@pytest.mark.parametrize("prec,eps", [("fp64", 1e-10), ("fp64", 1e-6), ("fp32", 1e-6)])
@pytest.mark.parametrize("kind", ["disk", "clustered"])
@pytest.mark.parametrize("N,M,xikind", [(500, 300, "uniform"), (3000, 1000, "uniform"),
                                        (20000, 1500, "uniform"), (4096, 700, "integer")])
def test_xi_against_oracle(fl, prec, eps, kind, N, M, xikind):
    rng = np.random.default_rng(N + M)
    xi = np.arange(N) + 1.0 if xikind == "integer" else rng.uniform(1.0, N, N)
    c = W.coefficients(N, seed=N)
    w = _nodes(kind, M, seed=M)
    f, info = _run(fl, c, xi, w, eps, prec)
    ref = oracle.xi_direct(c, xi, w)
    assert oracle.error_E(ref, f, c) <= _tol(eps, prec, ref, c)
    assert f[M] == 0                                     # Z^0 -> 0


def test_xi_integer_exponents_match_integer_transform(fl):
    N, M, eps = 5000, 800, 1e-10
    c = W.coefficients(N, seed=3)
    w = _nodes("disk", M, seed=4)
    f, _ = _run(fl, c, np.arange(N) + 1.0, w, eps, "fp64")
    pi = fl.Plan(N, torch.from_numpy(w).cuda(), eps, precision="fp64")
    fi = pi.execute(torch.from_numpy(c).cuda()).cpu().numpy()
    pi.close()
    z = np.exp(2j * np.pi * (w[:, 0] + 1j * w[:, 1]))
    assert np.max(np.abs(f - z * fi)) <= 2 * eps * np.sum(np.abs(c))


@pytest.mark.parametrize("q", [0, 3, 7])
def test_xi_matches_structured(fl, q):
    # q = 0: the rank from eps (15, right-hand sides in one chunk of 16); q = 3
    # and 7: chunks of 4 and 8 (the ranks of eps around 1e-1 and 1e-3)
    rng = np.random.default_rng(8)
    N, M, eps = 400, 250, 1e-8
    xi = rng.uniform(1.0, N, N)
    c = W.coefficients(N, seed=9)
    w = _nodes("clustered", M, seed=10)
    f, info = _run(fl, c, xi, w, eps, "fp64", q=q)
    fs, P = S.xflt_alg2_xi(c, xi, w, eps, q=q or None)
    assert info["q"] == P.lap.q and info["levels"] == P.lap.M
    assert oracle.error_E(fs, f, c) <= eps / 3


def test_xi_full_size_sampled(fl):
    N = M = 1 << 18
    rng = np.random.default_rng(11)
    xi = rng.uniform(1.0, N, N)
    c = W.coefficients(N, seed=12)
    w = _nodes("clustered", M, seed=13)
    f, _ = _run(fl, c, xi, w, 1e-6, "fp32")
    idx = np.random.default_rng(14).choice(M, 256, replace=False)
    ref = oracle.xi_direct(c, xi, w[idx])
    assert oracle.error_E(ref, f[idx], c) <= _tol(1e-6, "fp32", ref, c)


def test_xi_invalid(fl):
    w = torch.tensor([[0.1, 0.2]], dtype=torch.float64, device="cuda")
    with pytest.raises(fl.FLError) as ei:
        fl.XiPlan(torch.tensor([0.5, 2.0], dtype=torch.float64, device="cuda"), w, 1e-6)
    assert ei.value.status == fl.FL_EINVAL
    with pytest.raises(fl.FLError) as ei:
        fl.XiPlan(torch.tensor([1.5, 2.0], dtype=torch.float64, device="cuda"),
                  torch.tensor([[0.7, 0.2]], dtype=torch.float64, device="cuda"), 1e-6)
    assert ei.value.status == fl.FL_EINVAL
    p = fl.XiPlan(torch.tensor([1.5, 2.0], dtype=torch.float64, device="cuda"), w, 1e-6)
    c = torch.zeros(2, dtype=torch.complex64, device="cuda")
    out = torch.zeros(1, dtype=torch.complex64, device="cuda")
    assert fl.fl_execute_deriv(p.handle, c.data_ptr(), out.data_ptr(), None) == fl.FL_EUNSUPPORTED
    p.close()


def _tol_t(eps, prec, ref, g):
    if prec == "fp64":
        return eps
    return eps + 32 * U32 * np.max(np.abs(ref)) / np.sum(np.abs(g))


@pytest.mark.parametrize("prec,eps", [("fp64", 1e-10), ("fp64", 1e-6), ("fp32", 1e-6)])
@pytest.mark.parametrize("kind", ["disk", "clustered"])
@pytest.mark.parametrize("N,M,xikind", [(500, 300, "uniform"), (3000, 1000, "uniform"),
                                        (20000, 1500, "uniform"), (4096, 700, "integer")])
def test_xi_transposed_against_oracle(fl, prec, eps, kind, N, M, xikind):
    rng = np.random.default_rng(N + 7 * M)
    xi = np.arange(N) + 1.0 if xikind == "integer" else rng.uniform(1.0, N, N)
    w = _nodes(kind, M, seed=M + 1)
    g = W.targets(w.shape[0], seed=M + 2)
    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    p = fl.XiPlan(torch.from_numpy(xi).cuda(), torch.from_numpy(w).cuda(), eps, precision=prec)
    gd = torch.from_numpy(g).to(cdt).cuda()
    out = p.transposed(gd).cpu().numpy().astype(np.complex128)
    adj = p.adjoint(gd).cpu().numpy().astype(np.complex128)
    p.close()
    ref = oracle.xi_transposed(g, xi, w)
    assert oracle.error_E(ref, out, g) <= _tol_t(eps, prec, ref, g)
    ref_adj = np.conj(oracle.xi_transposed(np.conj(g), xi, w))
    assert oracle.error_E(ref_adj, adj, g) <= _tol_t(eps, prec, ref_adj, g)


def test_xi_adjoint_inner_product(fl):
    # <C c, r> = <c, C^* r> with both sides from the GPU plan
    rng = np.random.default_rng(31)
    N, M, eps = 6000, 2000, 1e-10
    xi = rng.uniform(1.0, N, N)
    w = _nodes("clustered", M, seed=32)
    c = W.coefficients(N, seed=33)
    r = W.targets(w.shape[0], seed=34)
    p = fl.XiPlan(torch.from_numpy(xi).cuda(), torch.from_numpy(w).cuda(), eps, precision="fp64")
    f = p.execute(torch.from_numpy(c).cuda()).cpu().numpy()
    a = p.adjoint(torch.from_numpy(r).cuda()).cpu().numpy()
    p.close()
    lhs = np.vdot(r, f)
    rhs = np.vdot(a, c)
    assert abs(lhs - rhs) <= 4 * eps * np.sum(np.abs(c)) * np.sum(np.abs(r))


def test_xi_transposed_full_size_sampled(fl):
    N = M = 1 << 18
    rng = np.random.default_rng(41)
    xi = rng.uniform(1.0, N, N)
    w = _nodes("clustered", M, seed=42)
    g = W.targets(w.shape[0], seed=43)
    p = fl.XiPlan(torch.from_numpy(xi).cuda(), torch.from_numpy(w).cuda(), 1e-6, precision="fp32")
    out = p.transposed(torch.from_numpy(g).to(torch.complex64).cuda()).cpu().numpy().astype(np.complex128)
    p.close()
    idx = np.random.default_rng(44).choice(N, 256, replace=False)
    ref = oracle.xi_transposed(g, xi[idx], w)
    assert oracle.error_E(ref, out[idx], g) <= _tol_t(1e-6, "fp32", ref, g)
