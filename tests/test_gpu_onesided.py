"""GPU parity of the one-sided variant (fl_options.variant = 1).

The band weights are exp(-y_s k) at the Chebyshev points y_s of each node band
(interpolation in y only); q comes from the one-sided bound 2 q^q e^-q /
(4^q q!) <= eps/3.  Checked through the C ABI:

* E <= eps (FP64) or eps + 32 u_32 ||f||_inf / ||c||_1 (FP32) against the
  plain oracle on three node distributions, two-pass grids included, routes
  "nfft" and "auto";
* the GPU result differs from the structured one-sided oracle (exact NDFTs)
  by at most the NFFT share eps/3;
* q, levels and l_m follow the rule the oracle states;
* the adjoint and the k-weighted transform of the variant against the oracle;
* N = M = 2^20 FP32 on a seeded sample of 512 outputs.
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


def tol(eps, prec, ref, c):
    if prec == "fp64":
        return eps
    return eps + 32 * U32 * np.max(np.abs(ref)) / np.sum(np.abs(c))


def _plan(fl, N, w, eps, prec, route="nfft"):
    return fl.Plan(N, torch.from_numpy(np.ascontiguousarray(w)).cuda(), eps, precision=prec,
                   route=route, variant="onesided")


def _fwd(fl, c, w, eps, prec, route="nfft", deriv=False):
    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    p = _plan(fl, len(c), w, eps, prec, route)
    f = p.execute(torch.from_numpy(np.asarray(c)).to(cdt).cuda(), deriv=deriv)
    out = f.cpu().numpy().astype(np.complex128)
    info = p.info()
    p.close()
    return out, info


def _nodes(kind, M, seed, eps):
    if kind == "disk":
        return W.nodes_disk_uniform(M, seed)
    if kind == "clustered":
        return W.nodes_circle_clustered(M, seed)
    return W.nodes_paper_section5(M, S.rank_q(eps), seed)


@pytest.mark.parametrize("route", ["nfft", "auto"])
@pytest.mark.parametrize("prec,eps", [("fp64", 1e-12), ("fp64", 1e-8), ("fp32", 1e-6)])
@pytest.mark.parametrize("kind,N,M", [("disk", 1024, 1024), ("clustered", 20000, 3000),
                                      ("paper", 4097, 777), ("clustered", 1 << 16, 2048)])
def test_onesided_against_oracle(fl, route, prec, eps, kind, N, M):
    c = W.coefficients(N, seed=N)
    w = _nodes(kind, M, 7, eps)
    f, info = _fwd(fl, c, w, eps, prec, route)
    assert info["variant"] == "onesided"
    ref = oracle.flt_direct(c, w)
    E = oracle.error_E(ref, f, c)
    assert E <= tol(eps, prec, ref, c), E


def test_onesided_matches_structured(fl):
    N, M, eps = 512, 300, 1e-8
    c = W.coefficients(N, seed=4)
    w = W.nodes_circle_clustered(M, seed=5)
    f, info = _fwd(fl, c, w, eps, "fp64")
    fs, q = S.xflt_alg2_onesided(c, w, eps)
    P = S.xflt_params(N, eps)
    assert info["q"] == q and info["levels"] == P.lap.M
    for b in range(1, info["levels"]):
        assert info["band_ell"][b] == P.lap.ell[b]
    assert oracle.error_E(fs, f, c) <= eps / 3


def test_onesided_rank(fl):
    w = W.nodes_disk_uniform(8, seed=1)
    for eps, q in ((1e-6, 10), (1e-10, 17), (1e-12, 20)):
        _, info = _fwd(fl, W.coefficients(1 << 12, 0), w, eps, "fp64")
        assert info["q"] == q == S.rank_q_onesided(eps / 3)


@pytest.mark.parametrize("prec,eps", [("fp64", 1e-10), ("fp32", 1e-6)])
def test_onesided_adjoint_and_derivative(fl, prec, eps):
    N, M = 3000, 1500
    c = W.coefficients(N, seed=8)
    w = W.nodes_circle_clustered(M, seed=9)
    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    p = _plan(fl, N, w, eps, prec)
    r = W.targets(M, seed=10)
    g = p.adjoint(torch.from_numpy(r).to(cdt).cuda()).cpu().numpy().astype(np.complex128)
    ref = oracle.flt_adjoint(r, w, N)
    # the adjoint's entries are bounded by eps ||r||_1 (the transpose of Theorem 4.3)
    bound = eps if prec == "fp64" else eps + 32 * U32 * np.max(np.abs(ref)) / np.sum(np.abs(r))
    assert np.max(np.abs(g - ref)) / np.sum(np.abs(r)) <= bound
    cd = 2j * np.pi * np.arange(N) * c
    fd = p.execute(torch.from_numpy(c).to(cdt).cuda(), deriv=True).cpu().numpy().astype(np.complex128)
    refd = oracle.flt_direct(cd, w)
    assert oracle.error_E(refd, fd, cd) <= tol(eps, prec, refd, cd)
    p.close()


def test_onesided_full_size_sampled(fl):
    N = M = 1 << 20
    c = W.coefficients(N, seed=0)
    w = W.nodes_circle_clustered(M, seed=1)
    f, info = _fwd(fl, c, w, 1e-6, "fp32", route="auto")
    assert info["q"] == 10
    idx = np.random.default_rng(2).choice(M, 512, replace=False)
    ref = oracle.flt_direct(c, w[idx])
    E = oracle.error_E(ref, f[idx], c)
    assert E <= 1e-6, E
