"""GPU parity of the window gather fused into the FFT's second pass.

With fuse_gather on, a band's grid is never written: pass 2 sums each node's
taps over the rows of its tile into partial sums, and the gather kernel adds a
node's partials and recombines the right-hand sides with the barycentric
weights.  The result is the same NFFT of Algorithm 2 in another summation
order, so each fused result is checked (a) against the plain FP64 oracle at the
forward tests' bound, E <= eps + 32 u_32 ||f||_inf / ||c||_1, and (b) against
the unfused plan on the same inputs to float rounding.  Sizes span four-step
grids of 2^13 to 2^18 points (pass-2 tiles of 2 to 8 rows), ragged N, nodes on
the cell and tile boundaries and at the grid's wrap-around, Z^0 nodes, the
derivative and node-gradient calls, and a batch.

Oversampling below 2 (fl_options.oversampling): a band's frequencies split
into P contiguous sub-bands, each an NFFT on a power-of-two grid of about
sigma K/P points, whose partial sums the gather combines with the sub-bands'
centre phases.  A different NFFT (grids, windows), so those plans are checked
against the oracle at the same bound, forward, derivative, node gradient,
adjoint and transposed evaluation, and in a batch; FP64 plans, whose
sub-bands are gathered from their grids, at the FP64 bar E <= eps.
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


def tol(eps, fref, c):
    return eps + 32 * U32 * np.max(np.abs(fref)) / np.sum(np.abs(c))


def _nodes(kind, M, seed):
    if kind == "clustered":
        return W.nodes_circle_clustered(M, seed)
    if kind == "disk":
        return W.nodes_disk_uniform(M, seed)
    # boundaries: x on multiples of 1/2^k (cell and tile edges of every grid),
    # just below 1 (the window wraps around the grid's end) and at 0, with
    # y spread over the bands; plus two Z^0 nodes
    rng = np.random.default_rng(seed)
    k = rng.integers(0, 1 << 18, M)
    x = k / float(1 << 18)
    x[:8] = [0.0, 1.0 - 2.0 ** -40, 1.0 - 2.0 ** -20, 0.5, 2.0 ** -18, 1.0 - 2.0 ** -18, 0.25, 0.75]
    y = 10.0 ** (-6.0 * rng.random(M)) / (2 * np.pi)
    y[::3] = 0.0
    w = np.stack([x, y], axis=1)
    return np.concatenate([w, [[0.3, 9.0], [0.9, 4.0]]])


def _plan_run(fl, c, w, eps, fuse, route="nfft", deriv=False, r=None, sigma="auto"):
    dev = torch.device("cuda")
    plan = fl.Plan(len(c), torch.from_numpy(np.ascontiguousarray(w)).to(dev), eps,
                   precision="fp32", route=route, fuse=fuse, sigma=sigma)
    ct = torch.from_numpy(np.asarray(c)).to(torch.complex64).to(dev)
    if r is not None:
        f = plan.grad_w(ct, torch.from_numpy(r).to(torch.complex64).to(dev))
    else:
        f = plan.execute(ct, deriv=deriv)
    torch.cuda.synchronize()
    out = f.cpu().numpy().astype(np.complex128)
    info = plan.info()
    plan.close()
    return out, info


@pytest.mark.parametrize("kind", ["clustered", "disk", "edges"])
@pytest.mark.parametrize("N", [5000, 40000, 70001])
def test_fused_matches_unfused_and_oracle(fl, kind, N):
    eps = 1e-6
    M = 3000
    c = W.coefficients(N, seed=N % 97)
    w = _nodes(kind, M, seed=N % 89)
    f_on, info_on = _plan_run(fl, c, w, eps, "on", sigma="2")
    f_off, info_off = _plan_run(fl, c, w, eps, "off")
    assert info_on["n_bands_fused"] > 0 and info_on["fused_entries"] > 0
    assert info_off["n_bands_fused"] == 0
    ref = oracle.flt_direct(c, w)
    assert oracle.error_E(ref, f_on, c) <= tol(eps, ref, c)
    # the same NFFT summed in another order: float rounding only
    assert np.max(np.abs(f_on - f_off)) <= 64 * U32 * max(np.max(np.abs(ref)), 1.0)


def test_fused_auto_routes(fl):
    # by cost: a few thousand nodes on 2^18-point grids are fused, and every
    # band with a grid of 4096 points or fewer is not
    eps = 1e-6
    N, M = 1 << 17, 4000
    c = W.coefficients(N, seed=3)
    w = W.nodes_circle_clustered(M, seed=4)
    f, info = _plan_run(fl, c, w, eps, "auto", route="auto")
    assert info["n_bands_fused"] > 0
    ref = oracle.flt_direct(c, w)
    assert oracle.error_E(ref, f, c) <= tol(eps, ref, c)


def test_fused_derivative_and_node_gradient(fl):
    eps = 1e-6
    N, M = 20000, 2000
    c = W.coefficients(N, seed=5)
    w = W.nodes_circle_clustered(M, seed=6)
    k = np.arange(N)
    cd = 2j * np.pi * k * c
    ref = oracle.flt_direct(cd, w)
    fd, info = _plan_run(fl, c, w, eps, "on", deriv=True, sigma="2")
    assert info["n_bands_fused"] > 0
    assert oracle.error_E(ref, fd, cd) <= tol(eps, ref, cd)
    r = W.targets(M, seed=7)
    gw, _ = _plan_run(fl, c, w, eps, "on", r=r, sigma="2")
    # gw_j = r_j conj(f'_j)
    gref = r * np.conj(ref)
    assert np.max(np.abs(gw - gref)) <= np.max(np.abs(r)) * tol(eps, ref, cd) * np.sum(np.abs(cd)) * 1.01


def test_fused_batched(fl):
    eps = 1e-6
    dev = torch.device("cuda")
    Ns = np.array([3000, 9000, 2500, 17000], dtype=np.int64)
    Ms = np.array([400, 1200, 0, 900], dtype=np.int64)
    cs = [W.coefficients(int(n), seed=40 + i) for i, n in enumerate(Ns)]
    ws = [W.nodes_circle_clustered(int(m), seed=50 + i) for i, m in enumerate(Ms)]
    outs = {}
    for fuse in ("on", "off"):
        bp = fl.BatchedPlan(Ns, Ms, torch.from_numpy(np.concatenate(ws)).to(dev), eps, fuse=fuse,
                            route="nfft", sigma="2")
        f = bp.execute(torch.from_numpy(np.concatenate(cs)).to(torch.complex64).to(dev))
        torch.cuda.synchronize()
        outs[fuse] = (f.cpu().numpy().astype(np.complex128), bp.info())
        bp.close()
    assert outs["on"][1]["n_bands_fused"] > 0 and outs["off"][1]["n_bands_fused"] == 0
    off = 0
    for i in range(len(Ns)):
        m = int(Ms[i])
        if m == 0:
            continue
        ref = oracle.flt_direct(cs[i], ws[i])
        fi = outs["on"][0][off:off + m]
        assert oracle.error_E(ref, fi, cs[i]) <= tol(eps, ref, cs[i]), i
        assert np.max(np.abs(fi - outs["off"][0][off:off + m])) <= 64 * U32 * max(np.max(np.abs(ref)), 1.0)
        off += m


# --------------------------------------------------------------------------
# Oversampling below 2: sub-band NFFTs

def _split_plan(fl, N, w, eps, sigma, route="nfft"):
    dev = torch.device("cuda")
    plan = fl.Plan(N, torch.from_numpy(np.ascontiguousarray(w)).to(dev), eps, precision="fp32",
                   route=route, sigma=sigma)
    info = plan.info()
    assert info["sigma_min"] < 2.0 and max(info["band_parts"]) > 1, info["band_parts"]
    # the FP32 limit on the deconvolution's gain keeps sigma near 1.5 or above
    b = np.pi * (2 - 1 / info["sigma_min"])
    gain = np.exp(info["m_w"] * (b - np.sqrt(b * b - (np.pi / info["sigma_min"]) ** 2)))
    assert gain <= 32.0 * (1 + 1e-12), (info["sigma_min"], info["m_w"])
    return plan, info


@pytest.mark.parametrize("sigma", ["min", "auto"])
@pytest.mark.parametrize("eps", [1e-6, 1e-4])
@pytest.mark.parametrize("kind,N", [("clustered", 40000), ("disk", 70001), ("edges", 1 << 17)])
def test_split_forward_matches_oracle(fl, sigma, eps, kind, N):
    c = W.coefficients(N, seed=N % 71)
    w = _nodes(kind, 2500, seed=N % 61)
    plan, info = _split_plan(fl, N, w, eps, sigma)
    f = plan.execute(torch.from_numpy(c).to(torch.complex64).cuda())
    torch.cuda.synchronize()
    plan.close()
    f = f.cpu().numpy().astype(np.complex128)
    ref = oracle.flt_direct(c, w)
    assert oracle.error_E(ref, f, c) <= tol(eps, ref, c), (info["m_w"], info["sigma_min"])


def test_split_auto_at_full_bandwidth(fl):
    # nodes clustered near the circle at N = 2^18: the cost model splits the
    # full-bandwidth bands (sigma from the tolerance) and E stays within eps
    eps, N = 1e-6, 1 << 18
    c = W.coefficients(N, seed=3)
    w = W.nodes_circle_clustered(6000, seed=4)
    plan, info = _split_plan(fl, N, w, eps, "auto", route="auto")
    f = plan.execute(torch.from_numpy(c).to(torch.complex64).cuda()).cpu().numpy()
    plan.close()
    ref = oracle.flt_direct(c, w)
    assert oracle.error_E(ref, f.astype(np.complex128), c) <= tol(eps, ref, c)


@pytest.mark.parametrize("sigma", ["min", "auto"])
def test_split_adjoint_transposed_and_gradients(fl, sigma):
    eps, N, M = 1e-6, 50000, 2000
    c = W.coefficients(N, seed=8)
    w = W.nodes_circle_clustered(M, seed=9)
    r = W.targets(M, seed=10)
    plan, _ = _split_plan(fl, N, w, eps, sigma)
    dev = torch.device("cuda")
    ct = torch.from_numpy(c).to(torch.complex64).to(dev)
    rt = torch.from_numpy(r).to(torch.complex64).to(dev)
    adj = plan.adjoint(rt).cpu().numpy().astype(np.complex128)
    tr = plan.transposed(rt).cpu().numpy().astype(np.complex128)
    fd = plan.execute(ct, deriv=True).cpu().numpy().astype(np.complex128)
    gw = plan.grad_w(ct, rt).cpu().numpy().astype(np.complex128)
    plan.close()
    aref = oracle.flt_adjoint(r, w, N)
    assert oracle.error_E(aref, adj, r) <= tol(eps, aref, r)
    # transposed: C^T r = conj(C^* conj r)
    tref = np.conj(oracle.flt_adjoint(np.conj(r), w, N))
    assert oracle.error_E(tref, tr, r) <= tol(eps, tref, r)
    cd = 2j * np.pi * np.arange(N) * c
    dref = oracle.flt_direct(cd, w)
    assert oracle.error_E(dref, fd, cd) <= tol(eps, dref, cd)
    gref = r * np.conj(dref)
    assert np.max(np.abs(gw - gref)) <= np.max(np.abs(r)) * tol(eps, dref, cd) * np.sum(np.abs(cd)) * 1.01


def test_split_batched(fl):
    eps = 1e-6
    dev = torch.device("cuda")
    Ns = np.array([30000, 9000, 2500, 47000], dtype=np.int64)
    Ms = np.array([700, 1200, 0, 900], dtype=np.int64)
    cs = [W.coefficients(int(n), seed=60 + i) for i, n in enumerate(Ns)]
    ws = [W.nodes_circle_clustered(int(m), seed=70 + i) for i, m in enumerate(Ms)]
    bp = fl.BatchedPlan(Ns, Ms, torch.from_numpy(np.concatenate(ws)).to(dev), eps, route="nfft",
                        sigma="min")
    info = bp.info()
    f = bp.execute(torch.from_numpy(np.concatenate(cs)).to(torch.complex64).to(dev))
    torch.cuda.synchronize()
    bp.close()
    assert info["sigma_min"] < 2.0
    f = f.cpu().numpy().astype(np.complex128)
    off = 0
    for i in range(len(Ns)):
        m = int(Ms[i])
        if m == 0:
            continue
        ref = oracle.flt_direct(cs[i], ws[i])
        assert oracle.error_E(ref, f[off:off + m], cs[i]) <= tol(eps, ref, cs[i]), i
        off += m


def _fp64_split_plan(fl, N, w, eps, sigma, route="nfft"):
    plan = fl.Plan(N, torch.from_numpy(np.ascontiguousarray(w)).cuda(), eps, precision="fp64",
                   route=route, sigma=sigma)
    info = plan.info()
    assert info["sigma_min"] < 2.0 and max(info["band_parts"]) > 1, info["band_parts"]
    # the FP64 limit on the deconvolution's gain: <= 2^47 eps/3
    b = np.pi * (2 - 1 / info["sigma_min"])
    gain = np.exp(info["m_w"] * (b - np.sqrt(b * b - (np.pi / info["sigma_min"]) ** 2)))
    assert gain <= 2.0 ** 47 * eps / 3 * (1 + 1e-12), (info["sigma_min"], info["m_w"])
    return plan, info


@pytest.mark.parametrize("sigma", ["min", "auto"])
@pytest.mark.parametrize("eps", [1e-10, 1e-6])
@pytest.mark.parametrize("kind,N", [("clustered", 40000), ("edges", 1 << 17)])
def test_fp64_split_forward(fl, sigma, eps, kind, N):
    # FP64 plans gather the sub-bands from their grids; the FP64 bar: E <= eps
    c = W.coefficients(N, seed=N % 53)
    w = _nodes(kind, 2500, seed=N % 47)
    plan, info = _fp64_split_plan(fl, N, w, eps, sigma)
    f = plan.execute(torch.from_numpy(c).cuda()).cpu().numpy()
    plan.close()
    ref = oracle.flt_direct(c, w)
    assert oracle.error_E(ref, f, c) <= eps, (info["m_w"], info["sigma_min"])


def test_fp64_split_adjoint_transposed_and_gradients(fl):
    eps, N, M = 1e-10, 50000, 2000
    c = W.coefficients(N, seed=18)
    w = W.nodes_circle_clustered(M, seed=19)
    r = W.targets(M, seed=20)
    plan, _ = _fp64_split_plan(fl, N, w, eps, "min")
    ct, rt = torch.from_numpy(c).cuda(), torch.from_numpy(r).cuda()
    adj = plan.adjoint(rt).cpu().numpy()
    tr = plan.transposed(rt).cpu().numpy()
    fd = plan.execute(ct, deriv=True).cpu().numpy()
    gw = plan.grad_w(ct, rt).cpu().numpy()
    plan.close()
    aref = oracle.flt_adjoint(r, w, N)
    assert oracle.error_E(aref, adj, r) <= eps
    tref = np.conj(oracle.flt_adjoint(np.conj(r), w, N))
    assert oracle.error_E(tref, tr, r) <= eps
    cd = 2j * np.pi * np.arange(N) * c
    dref = oracle.flt_direct(cd, w)
    assert oracle.error_E(dref, fd, cd) <= eps
    assert np.max(np.abs(gw - r * np.conj(dref))) <= np.max(np.abs(r)) * eps * np.sum(np.abs(cd))


def test_split_not_used_in_float_pairs(fl):
    # the float pairs' 48-bit grids would lose eps = 1e-12 to the gain
    dev = torch.device("cuda")
    w = W.nodes_circle_clustered(500, seed=1)
    plan = fl.Plan(40000, torch.from_numpy(w).to(dev), 1e-10, precision="fp64ff", route="nfft",
                   sigma="min")
    info = plan.info()
    plan.close()
    assert info["sigma_min"] == 2.0 and max(info["band_parts"]) == 1
