"""GPU parity of the FP64-accuracy form in float pairs (precision "fp64ff").

The FFTs of the band grids run in float pairs (about 48 significant bits from
FP32 arithmetic); weights and twiddles are rounded once from FP64, and the
gather, recombination, phases and direct bands run in double.  The bar is the
FP64 one: E <= eps against the oracle, with nothing added for rounding.
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
    r = torch.zeros(M, dtype=torch.complex128, device="cuda")
    out = torch.zeros(N, dtype=torch.complex128, device="cuda")
    for fn in (fl.fl_adjoint, fl.fl_transposed):
        assert fn(p.handle, r.data_ptr(), out.data_ptr(), None) == fl.FL_EUNSUPPORTED
    assert fl.fl_execute_deriv(p.handle, cc.data_ptr(), r.data_ptr(), None) == fl.FL_EUNSUPPORTED
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
