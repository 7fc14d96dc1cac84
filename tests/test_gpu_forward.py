"""GPU parity of the forward transform (Algorithm 2) against the CPU oracle.

Unless a test says otherwise every band goes through the NFFT (route "nfft",
Algorithm 2 as printed); the routed and the all-direct plans are checked at
the end.

Element-by-element comparison through the C ABI, with E = ||f - f~||_inf /
||c||_1 (eq. 5.1).  Tolerance: E <= eps is what Theorem 4.3 guarantees in exact
arithmetic.  The FP64 form is held to exactly that.  The FP32 form adds float
rounding, which scales with the magnitude of the values it rounds -- the grids
and the output, all O(||f||_inf) -- so its bound is
    E <= eps + 32 u_32 ||f||_inf / ||c||_1,     u_32 = 2^-24,
(32 ~ log2(n) FFT stages plus the q-term recombination).  For random c at large
N, ||f||_inf ~ sqrt(N) << ||c||_1 ~ N and the extra term vanishes; at N = 3 it
is what dominates.
"""
import numpy as np
import pytest

import oracle
from oracle import structured as S
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


def _run(fl, c, w, eps, prec, q=0, deriv=False, route="nfft"):
    dev = torch.device("cuda")
    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    plan = fl.Plan(len(c), torch.from_numpy(np.ascontiguousarray(w)).to(dev), eps, precision=prec, q=q,
                   route=route)
    f = plan.execute(torch.from_numpy(np.asarray(c)).to(cdt).to(dev), deriv=deriv)
    torch.cuda.synchronize()
    out = f.cpu().numpy().astype(np.complex128)
    info = plan.info()
    plan.close()
    return out, info


U32 = 2.0 ** -24


def tol(eps, prec, fref, c):
    """Allowed E for a plan of accuracy eps (see the module docstring)."""
    if prec == "fp64":
        return eps
    return eps + 32 * U32 * np.max(np.abs(fref)) / np.sum(np.abs(c))


def _nodes(kind, M, seed, eps=1e-6):
    if kind == "disk":
        return W.nodes_disk_uniform(M, seed)
    if kind == "clustered":
        return W.nodes_circle_clustered(M, seed)
    if kind == "paper":
        return W.nodes_paper_section5(M, S.rank_q(eps), seed)
    if kind == "circle":
        return W.nodes_equispaced_circle(M)
    raise ValueError(kind)


@pytest.mark.parametrize("prec,eps", [("fp64", 1e-10), ("fp32", 1e-6)])
def test_config0_disk_uniform_1024(fl, prec, eps):
    c = W.coefficients(1024, seed=0)
    w = W.nodes_disk_uniform(1024, seed=1)
    f, info = _run(fl, c, w, eps, prec)
    ref = oracle.flt_direct(c, w)
    E = oracle.error_E(ref, f, c)
    assert E <= tol(eps, prec, ref, c), E


@pytest.mark.parametrize("N,M", [(1, 5), (2, 3), (3, 17), (100, 1), (1000, 999), (4097, 300),
                                 (20000, 2000), (5, 0)])
@pytest.mark.parametrize("prec,eps", [("fp64", 1e-12), ("fp32", 1e-6)])
def test_sizes_and_ragged_tails(fl, N, M, prec, eps):
    c = W.coefficients(N, seed=N)
    w = W.nodes_disk_uniform(M, seed=M + 1)
    f, info = _run(fl, c, w, eps, prec)
    if M:
        ref = oracle.flt_direct(c, w)
        E = oracle.error_E(ref, f, c)
        assert E <= tol(eps, prec, ref, c), (E, info["q"], info["m_w"])


@pytest.mark.parametrize("kind", ["disk", "clustered", "paper", "circle"])
@pytest.mark.parametrize("prec,eps", [("fp64", 1e-12), ("fp64", 1e-8), ("fp32", 1e-6),
                                      ("fp32", 1e-4)])
def test_node_distributions(fl, kind, prec, eps):
    N, M = 3000, 2500
    c = W.coefficients(N, seed=7)
    w = _nodes(kind, M, seed=8, eps=eps)
    f, _ = _run(fl, c, w, eps, prec)
    ref = oracle.flt_direct(c, w)
    E = oracle.error_E(ref, f, c)
    assert E <= tol(eps, prec, ref, c), E


def test_special_nodes(fl):
    N = 777
    c = W.coefficients(N, seed=9)
    w = np.array([
        [0.0, 0.0], [0.5, 0.0], [-0.25, 0.0], [3.75, 0.0], [-7.1, 0.01],  # any real x
        [0.3, 5.0], [0.9, 40.0],                                           # Z^0: |z| < eps
        [0.123, 1e-15], [0.123, 1e-9], [0.77, 0.3],
    ])
    for prec, eps in (("fp64", 1e-12), ("fp32", 1e-6)):
        f, info = _run(fl, c, w, eps, prec)
        ref = oracle.flt_direct(c, w)
        assert oracle.error_E(ref, f, c) <= tol(eps, prec, ref, c)
        t0 = 0 if prec == "fp64" else 1e-7 * abs(c[0])
        assert abs(f[5] - c[0]) <= t0 and abs(f[6] - c[0]) <= t0   # Z^0 -> c_0
        assert info["z0_nodes"] == 2


@pytest.mark.parametrize("prec,eps", [("fp64", 1e-12), ("fp32", 1e-6)])
def test_two_pass_fft_bands(fl, prec, eps):
    # N = 2^14 and 2^16 put the Y_M band and the top bands on grids of 2^15..2^17
    # points (the four-step path); clustered nodes fill the near-circle bands.
    for N in (1 << 14, 1 << 16):
        c = W.coefficients(N, seed=N)
        w = W.nodes_circle_clustered(4096, seed=3)
        f, info = _run(fl, c, w, eps, prec)
        assert max(info["band_n"]) > 4096
        ref = oracle.flt_direct(c, w)
        E = oracle.error_E(ref, f, c)
        assert E <= tol(eps, prec, ref, c), E


def test_matches_structured_algorithm2(fl):
    # Same Laplace factorisation with exact NDFTs: the two differ only by the
    # NFFT error (<= eps/3 per Lemma 4.1) and rounding.
    N, M, eps = 512, 300, 1e-8
    c = W.coefficients(N, seed=4)
    w = W.nodes_circle_clustered(M, seed=5)
    f, info = _run(fl, c, w, eps, "fp64")
    fs, P = S.xflt_alg2(c, w, eps)
    assert info["q"] == P.lap.q and info["levels"] == P.lap.M
    for b in range(1, info["levels"]):
        assert info["band_ell"][b] == P.lap.ell[b]
    assert oracle.error_E(fs, f, c) <= eps / 3


def test_parameters_follow_definition(fl):
    N = 1 << 20
    w = W.nodes_disk_uniform(8, seed=1)
    for eps, q in ((1e-6, 12), (1e-10, 18), (1e-12, 22)):
        _, info = _run(fl, W.coefficients(N, 0)[:N], w, eps, "fp32")
        assert info["q"] == q == S.rank_q(eps / 3)
        P = S.xflt_params(N, eps)
        assert info["levels"] == P.lap.M
        assert info["y1"] == P.y1 and info["xi1"] == P.xi1


@pytest.mark.parametrize("prec,eps", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_derivative_in_w(fl, prec, eps):
    N, M = 2000, 700
    c = W.coefficients(N, seed=11)
    w = W.nodes_disk_uniform(M, seed=12)
    k = np.arange(N)
    cd = 2j * np.pi * k * c
    ref = oracle.flt_direct(cd, w)
    f, _ = _run(fl, c, w, eps, prec, deriv=True)
    assert oracle.error_E(ref, f, cd) <= tol(eps, prec, ref, cd)


def test_invalid_nodes_rejected(fl):
    w = torch.tensor([[0.1, 0.2], [0.3, -1e-3]], dtype=torch.float64, device="cuda")
    with pytest.raises(fl.FLError) as ei:
        fl.Plan(10, w, 1e-6)
    assert ei.value.status == fl.FL_EINVAL
    w2 = torch.tensor([[float("nan"), 0.2]], dtype=torch.float64, device="cuda")
    with pytest.raises(fl.FLError):
        fl.Plan(10, w2, 1e-6)


@pytest.mark.parametrize("prec,eps", [("fp32", 1e-6), ("fp64", 1e-12)])
def test_full_size_config2_sampled(fl, prec, eps):
    # N = M = 2^20, half the nodes on |z| = 1, half clustered near it; the
    # oracle checks a seeded sample of 512 outputs.
    N = M = 1 << 20
    c = W.coefficients(N, seed=0)
    w = W.nodes_circle_clustered(M, seed=1)
    f, info = _run(fl, c, w, eps, prec)
    idx = np.random.default_rng(2).choice(M, 512, replace=False)
    ref = oracle.flt_direct(c, w[idx])
    E = oracle.error_E(ref, f[idx], c)
    assert E <= tol(eps, prec, ref, c), E
    assert E <= eps, E


@pytest.mark.parametrize("route", ["auto", "direct"])
@pytest.mark.parametrize("prec,eps", [("fp64", 1e-12), ("fp32", 1e-6)])
@pytest.mark.parametrize("kind,N,M", [("disk", 1024, 1024), ("disk", 1 << 16, 3000),
                                      ("clustered", 20000, 5000), ("paper", 4097, 777)])
def test_routed_and_direct(fl, route, prec, eps, kind, N, M):
    c = W.coefficients(N, seed=21)
    w = _nodes(kind, M, seed=22, eps=eps)
    w = np.concatenate([w, [[0.4, 7.0]]])          # plus a Z^0 node
    f, info = _run(fl, c, w, eps, prec, route=route)
    if route == "direct":
        assert info["n_bands_fft"] == 0 and info["n_bands_direct"] > 0
    ref = oracle.flt_direct(c, w)
    E = oracle.error_E(ref, f, c)
    assert E <= tol(eps, prec, ref, c), E


def test_auto_route_sends_sparse_full_bands_to_direct(fl):
    # uniform-disk nodes put only a handful of nodes in each full-bandwidth band
    N = M = 1 << 18
    w = W.nodes_disk_uniform(M, seed=1)
    c = W.coefficients(N, seed=0)
    f, info = _run(fl, c, w, 1e-6, "fp32", route="auto")
    assert info["n_bands_direct"] > 0 and info["n_bands_fft"] > 0
    sparse_full = [b for b in range(1, info["levels"] + 1)
                   if info["band_K"][b] == N and 0 < info["band_nodes"][b] < 50]
    assert sparse_full, "expected full-bandwidth bands with few nodes"
    for b in sparse_full:
        assert info["band_route"][b] == 2
    idx = np.random.default_rng(3).choice(M, 256, replace=False)
    ref = oracle.flt_direct(c, w[idx])
    assert oracle.error_E(ref, f[idx], c) <= tol(1e-6, "fp32", ref, c)


@pytest.mark.parametrize("route", ["auto", "direct"])
def test_derivative_and_node_gradient_routes(fl, route):
    N, M = 3000, 900
    c = W.coefficients(N, seed=31)
    w = W.nodes_disk_uniform(M, seed=32)
    cd = 2j * np.pi * np.arange(N) * c
    ref = oracle.flt_direct(cd, w)
    f, _ = _run(fl, c, w, 1e-10, "fp64", deriv=True, route=route)
    assert oracle.error_E(ref, f, cd) <= 1e-10


@pytest.mark.parametrize("prec,eps", [("fp32", 1e-6), ("fp64", 1e-12)])
def test_nodes_on_and_next_to_chebyshev_points(fl, prec, eps):
    # y = 2 pi Im w on (or a few ulps from) a Chebyshev point of its band: the
    # barycentric weights take their hit / near-hit branches (FP32 form: the
    # differences tau - t_s from float pairs; FP64 form: in double).
    N = 3000
    c = W.coefficients(N, seed=21)
    P = S.xflt_params(N, eps)
    q = P.lap.q
    ts = S.chebyshev_points(q)
    rows = []
    rng = np.random.default_rng(22)
    for m in (2, 5, 9, 14):
        a = P.y1 / 2.0 ** m
        for s in (0, q // 2, q - 1):
            y = 1.5 * a + 0.5 * a * ts[s]
            for rel in (0.0, 1e-15, -3e-16, 1e-9):
                rows.append([rng.uniform(), y * (1 + rel) / (2 * np.pi)])
    w = np.array(rows)
    f, _ = _run(fl, c, w, eps, prec)
    ref = oracle.flt_direct(c, w)
    assert oracle.error_E(ref, f, c) <= tol(eps, prec, ref, c)


@pytest.mark.parametrize("prec,eps", [("fp32", 1e-6), ("fp64", 1e-12)])
def test_direct_bands_with_many_nodes(fl, prec, eps):
    # every band summed directly; on 2^16 disk nodes the low bands hold
    # thousands of nodes each with K <= 256 (the thread-per-node kernel in FP32)
    N, M = 1 << 12, 1 << 16
    c = W.coefficients(N, seed=31)
    w = W.nodes_disk_uniform(M, seed=32)
    f, info = _run(fl, c, w, eps, prec, route="direct")
    many = [b for b in range(1, info["levels"] + 1)
            if info["band_route"][b] == 2 and info["band_K"][b] <= 256 and info["band_nodes"][b] >= 2048]
    assert many, "expected direct bands with K <= 256 and >= 2048 nodes"
    idx = np.random.default_rng(33).choice(M, 2048, replace=False)
    ref = oracle.flt_direct(c, w[idx])
    assert oracle.error_E(ref, f[idx], c) <= tol(eps, prec, ref, c)
