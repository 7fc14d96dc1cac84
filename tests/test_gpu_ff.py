"""GPU parity of the FP64-accuracy form in float pairs (precision "fp64ff").

The FFTs of the band grids run in float pairs (about 48 significant bits from
FP32 arithmetic); weights and twiddles are rounded once from FP64, and the
gather, recombination, phases and direct bands run in double.  The bar is the
FP64 one: E <= eps against the oracle, with nothing added for rounding --
for the forward transform, and for the adjoint C^* r, the transposed
evaluation C^T g, the derivative in w and the node gradient, each against
its oracle (the adjoint's and the transposed sum's error relative to
||r||_1, the derivative's to the k-weighted ||2 pi k c_k||_1), and the
adjoint identity <r, C c> = <C^* r, c>.
"""
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


def _run(fl, c, w, eps, precision="fp64ff", route="auto", use_graph=False):
    p = fl.Plan(len(c), torch.from_numpy(np.ascontiguousarray(w)).cuda(), eps,
                precision=precision, route=route, use_graph=use_graph)
    f = p.execute(torch.from_numpy(c).cuda()).cpu().numpy()
    info = p.info()
    p.close()
    return f, info


@pytest.mark.parametrize("eps", [1e-12, 1e-10, 1e-6])
@pytest.mark.parametrize("route", ["auto", "nfft"])
@pytest.mark.parametrize("kind,N,M", [("disk", 1024, 1024), ("clustered", 1 << 14, 3000),
                                      ("clustered", 1 << 16, 2000), ("paper", 4097, 777)])
def test_ff_against_oracle(fl, eps, route, kind, N, M):
    c = W.coefficients(N, seed=N)
    if kind == "disk":
        w = W.nodes_disk_uniform(M, seed=M)
    elif kind == "clustered":
        w = W.nodes_circle_clustered(M, seed=M)
    else:
        w = W.nodes_paper_section5(M, 22, seed=M)
    w = np.concatenate([w, [[0.5, 9.0]]])          # a Z^0 node
    f, _ = _run(fl, c, w, eps, route=route)
    ref = oracle.flt_direct(c, w)
    assert oracle.error_E(ref, f, c) <= eps
    assert f[-1] == c[0]


def test_ff_two_pass_bands(fl):
    # grids above 4096 points take the four-step passes in float pairs
    N, M, eps = 1 << 18, 4000, 1e-12
    c = W.coefficients(N, seed=3)
    w = W.nodes_circle_clustered(M, seed=4)
    f, info = _run(fl, c, w, eps, route="nfft")
    assert max(info["band_n"][1:]) > 4096
    ref = oracle.flt_direct(c, w)
    assert oracle.error_E(ref, f, c) <= eps


def test_ff_full_size_sampled(fl):
    N = M = 1 << 20
    c = W.coefficients(N, seed=0)
    w = W.nodes_circle_clustered(M, seed=1)
    f, _ = _run(fl, c, w, 1e-12)
    idx = np.random.default_rng(2).choice(M, 256, replace=False)
    ref = oracle.flt_direct(c, w[idx])
    assert oracle.error_E(ref, f[idx], c) <= 1e-12


def test_ff_agrees_with_fp64_and_replays(fl):
    N, M, eps = 20000, 4000, 1e-12
    c = W.coefficients(N, seed=5)
    w = W.nodes_circle_clustered(M, seed=6)
    f_ff, _ = _run(fl, c, w, eps)
    f_64, _ = _run(fl, c, w, eps, precision="fp64")
    assert np.max(np.abs(f_ff - f_64)) <= 2 * eps * np.sum(np.abs(c))
    s = torch.cuda.Stream()
    p = fl.Plan(N, torch.from_numpy(w).cuda(), eps, precision="fp64ff", use_graph=True)
    cc = torch.from_numpy(c).cuda()
    with torch.cuda.stream(s):
        a = p.execute(cc)
        b = p.execute(cc)
    s.synchronize()
    assert torch.equal(a, b)
    assert np.array_equal(a.cpu().numpy(), f_ff)
    p.close()


def test_ff_batched_and_rejections(fl):
    Ns = [1, 300, 5000, 20000, 777, 4096]
    Ms = [7, 250, 3000, 2000, 0, 4096]
    cs = [W.coefficients(N, seed=60 + i) for i, N in enumerate(Ns)]
    ws = [W.nodes_circle_clustered(M, seed=70 + i) for i, M in enumerate(Ms)]
    dev = torch.device("cuda")
    plan = fl.BatchedPlan(Ns, Ms, torch.from_numpy(np.concatenate(ws)).to(dev), 1e-12,
                          precision="fp64ff")
    f = plan.execute(torch.from_numpy(np.concatenate(cs)).to(dev)).cpu().numpy()
    moff = 0
    for c, w, M in zip(cs, ws, Ms):
        if M:
            ref = oracle.flt_direct(c, w)
            assert oracle.error_E(ref, f[moff:moff + M], c) <= 1e-12
        moff += M
    plan.close()
    t = torch.linspace(0, 1, 64, dtype=torch.float64, device=dev)
    with pytest.raises(fl.FLError):
        fl.LaplacePlan(t, t + 1, 1e-10, precision="fp64ff")
    with pytest.raises(fl.FLError):
        fl.XiPlan(t * 10, torch.zeros(4, 2, dtype=torch.float64, device=dev), 1e-10,
                  precision="fp64ff")


def _ff_plan(fl, N, w, eps, route="auto"):
    return fl.Plan(N, torch.from_numpy(np.ascontiguousarray(w)).cuda(), eps, precision="fp64ff",
                   route=route)


@pytest.mark.parametrize("eps", [1e-12, 1e-10])
@pytest.mark.parametrize("route", ["auto", "nfft", "direct"])
@pytest.mark.parametrize("kind,N,M", [("disk", 1000, 1000), ("clustered", 20000, 1500),
                                      ("clustered", 1 << 16, 2000), ("disk", 1, 5)])
def test_ff_adjoint_against_oracle(fl, eps, route, kind, N, M):
    w = W.nodes_disk_uniform(M, seed=M) if kind == "disk" else W.nodes_circle_clustered(M, seed=M)
    w = np.concatenate([w, [[0.5, 9.0]]])        # one Z^0 node
    r = W.coefficients(M + 1, seed=N)
    p = _ff_plan(fl, N, w, eps, route)
    g = p.adjoint(torch.from_numpy(r).cuda()).cpu().numpy()
    p.close()
    ref = oracle.flt_adjoint(r, w, N)
    assert oracle.error_E(ref, g, r) <= eps


def test_ff_adjoint_identity_and_two_pass(fl):
    # grids of 2^17 points (four-step passes of sign -1 in pairs)
    N, M, eps = 1 << 16, 3000, 1e-12
    c = W.coefficients(N, seed=11)
    r = W.coefficients(M, seed=12)
    w = W.nodes_circle_clustered(M, seed=13)
    p = _ff_plan(fl, N, w, eps, "nfft")
    assert max(p.info()["band_n"][1:]) > 4096
    f = p.execute(torch.from_numpy(c).cuda()).cpu().numpy()
    g = p.adjoint(torch.from_numpy(r).cuda()).cpu().numpy()
    p.close()
    assert abs(np.vdot(r, f) - np.vdot(g, c)) <= 4 * eps * np.sum(np.abs(c)) * np.sum(np.abs(r))
    ref = oracle.flt_adjoint(r, w, N)
    assert oracle.error_E(ref, g, r) <= eps


@pytest.mark.parametrize("N,M,kind", [(700, 500, "disk"), (9000, 800, "clustered")])
def test_ff_transposed(fl, N, M, kind):
    eps = 1e-12
    w = W.nodes_disk_uniform(M, seed=3) if kind == "disk" else W.nodes_circle_clustered(M, seed=3)
    g = W.coefficients(M, seed=4)
    p = _ff_plan(fl, N, w, eps)
    out = p.transposed(torch.from_numpy(g).cuda()).cpu().numpy()
    p.close()
    ref = np.conj(oracle.flt_adjoint(np.conj(g), w, N))
    assert oracle.error_E(ref, out, g) <= eps


@pytest.mark.parametrize("route", ["auto", "nfft", "direct"])
@pytest.mark.parametrize("N,M", [(3000, 2000), (1 << 16, 1500)])
def test_ff_derivative_and_node_gradient(fl, route, N, M):
    eps = 1e-12
    c = W.coefficients(N, seed=21)
    w = np.concatenate([W.nodes_circle_clustered(M, seed=22), [[0.3, 9.0]]])   # and a Z^0 node
    r = W.targets(M + 1, seed=23)
    cd = 2j * np.pi * np.arange(N) * c
    ref = oracle.flt_direct(cd, w)
    p = _ff_plan(fl, N, w, eps, route)
    cc = torch.from_numpy(c).cuda()
    fd = p.execute(cc, deriv=True).cpu().numpy()
    gw = p.grad_w(cc, torch.from_numpy(r).cuda()).cpu().numpy()
    p.close()
    assert oracle.error_E(ref, fd, cd) <= eps
    assert fd[-1] == 0 and gw[-1] == 0
    gref = r * np.conj(ref)
    assert np.max(np.abs(gw - gref)) <= np.max(np.abs(r)) * eps * np.sum(np.abs(cd))


def test_ff_gradients_full_size_sampled(fl):
    # N = M = 2^18 disk-uniform: the adjoint and the derivative on sampled entries
    N = M = 1 << 18
    eps = 1e-12
    c = W.coefficients(N, seed=31)
    r = W.coefficients(M, seed=32)
    w = W.nodes_disk_uniform(M, seed=33)
    p = _ff_plan(fl, N, w, eps)
    g = p.adjoint(torch.from_numpy(r).cuda()).cpu().numpy()
    fd = p.execute(torch.from_numpy(c).cuda(), deriv=True).cpu().numpy()
    p.close()
    rng = np.random.default_rng(34)
    ks = rng.choice(N, 96, replace=False)
    ref_g = oracle.flt_adjoint_at(r, w, ks)
    assert oracle.error_E(ref_g, g[ks], r) <= eps
    js = rng.choice(M, 96, replace=False)
    cd = 2j * np.pi * np.arange(N) * c
    ref_d = oracle.flt_direct(cd, w[js])
    assert oracle.error_E(ref_d, fd[js], cd) <= eps
