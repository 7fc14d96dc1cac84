"""GPU parity of the real discrete Laplace transform (Algorithm 1).

Two references:
* the plain oracle (direct FP64 sum): E <= eps (Theorem A.3), plus the float
  rounding term for the FP32 form;
* the structured reference (K~ c with K~ of eq. (A.1) assembled block by
  block in numpy): the GPU computes the same f~, so the two agree to rounding.
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


def _run(fl, c, t, s, eps, prec, q=0):
    dev = torch.device("cuda")
    rdt = torch.float64 if prec == "fp64" else torch.float32
    plan = fl.LaplacePlan(torch.from_numpy(t).to(dev), torch.from_numpy(s).to(dev), eps,
                          precision=prec, q=q)
    f = plan.execute(torch.from_numpy(np.asarray(c)).to(rdt).to(dev))
    torch.cuda.synchronize()
    info = plan.info()
    plan.close()
    return f.cpu().numpy().astype(np.float64), info


def _tol(eps, prec, ref, c):
    if prec == "fp64":
        return eps
    return eps + 32 * U32 * max(np.max(np.abs(ref)), 1.0) / max(np.sum(np.abs(c)), 1e-300)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_config1_laplace_2_16(fl, prec):
    N = M = 1 << 16
    c, t, s = W.laplace_inputs(N, M, seed=0)
    if prec == "fp32":
        c = c.astype(np.float32).astype(np.float64)
    f, info = _run(fl, c, t, s, 1e-6, prec)
    assert info["q"] == 11 and info["levels"] == 38
    ref = oracle.laplace_direct(c, t, s)
    E = oracle.error_E(ref, f, c)
    assert E <= _tol(1e-6, prec, ref, c), E


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-10])
def test_matches_structured_algorithm1(fl, eps):
    c, t, s = W.laplace_inputs(3000, 2000, seed=3)
    f, info = _run(fl, c, t, s, eps, "fp64")
    fs, P = S.laplace_alg1(c, t, s, eps)
    assert info["q"] == P.q and info["levels"] == P.M
    for m in range(1, P.M):
        assert info["band_ell"][m] == P.ell[m]
    assert np.max(np.abs(f - fs)) <= 1e-12 * np.sum(np.abs(c))
    ref = oracle.laplace_direct(c, t, s)
    assert oracle.error_E(ref, f, c) <= eps


@pytest.mark.parametrize("N,M", [(1, 1), (31, 5), (32, 33), (33, 1), (1000, 100), (4097, 77),
                                 (0, 10), (10, 0)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sizes_and_ragged_tails(fl, N, M, prec):
    c, t, s = W.laplace_inputs(N, M, seed=N + M)
    if prec == "fp32":
        c = c.astype(np.float32).astype(np.float64)
    f, _ = _run(fl, c, t, s, 1e-8 if prec == "fp64" else 1e-5, prec)
    if M == 0:
        assert f.size == 0
        return
    ref = oracle.laplace_direct(c, t, s)
    if N == 0:
        assert np.all(f == 0)
        return
    eps = 1e-8 if prec == "fp64" else 1e-5
    assert oracle.error_E(ref, f, c) <= _tol(eps, prec, ref, c)


def test_zero_nodes_and_degenerate_ranges(fl):
    rng = np.random.default_rng(1)
    c = rng.standard_normal(500)
    t = rng.random(500)
    s = rng.random(300) * 50
    t[:7] = 0.0             # xi = 0: kernel 1 for every s
    s[:5] = 0.0             # y = 0: f = sum c
    f, _ = _run(fl, c, t, s, 1e-9, "fp64")
    ref = oracle.laplace_direct(c, t, s)
    assert oracle.error_E(ref, f, c) <= 1e-9
    # all s = 0: a single level, f = sum(c) exactly to rounding
    f0, info = _run(fl, c, t, np.zeros(4), 1e-9, "fp64")
    assert info["levels"] == 1
    assert np.allclose(f0, c.sum(), rtol=0, atol=1e-12 * np.sum(np.abs(c)))


def test_q_override_and_decay(fl):
    c, t, s = W.laplace_inputs(2048, 512, seed=8)
    ref = oracle.laplace_direct(c, t, s)
    Es = []
    for q in (2, 4, 6, 8, 10):
        eps = 2.0 ** (1 - 2 * q)
        f, info = _run(fl, c, t, s, eps, "fp64", q=q)
        assert info["q"] == q
        Es.append(oracle.error_E(ref, f, c))
        assert Es[-1] <= eps
    assert all(b < a for a, b in zip(Es, Es[1:]))


def test_invalid_nodes(fl):
    t = torch.tensor([0.1, -0.5], dtype=torch.float64, device="cuda")
    s = torch.tensor([1.0], dtype=torch.float64, device="cuda")
    with pytest.raises(fl.FLError) as ei:
        fl.LaplacePlan(t, s, 1e-6)
    assert ei.value.status == fl.FL_EINVAL
    t2 = torch.tensor([0.1, float("inf")], dtype=torch.float64, device="cuda")
    with pytest.raises(fl.FLError):
        fl.LaplacePlan(t2, s, 1e-6)


def test_deterministic(fl):
    c, t, s = W.laplace_inputs(20000, 5000, seed=9)
    a, _ = _run(fl, c, t, s, 1e-6, "fp32")
    b, _ = _run(fl, c, t, s, 1e-6, "fp32")
    assert np.array_equal(a, b)


# --------------------------------------------------------------------------
# Generalised Algorithm 1 (fl_plan_kernel): exp(-s t) and K_{1/2}(s t)

def _run_kernel(fl, kernel, c, t, s, eps, prec, q=0):
    dev = torch.device("cuda")
    rdt = torch.float64 if prec == "fp64" else torch.float32
    plan = fl.LaplacePlan(torch.from_numpy(t).to(dev), torch.from_numpy(s).to(dev), eps,
                          precision=prec, q=q, kernel=kernel)
    f = plan.execute(torch.from_numpy(np.asarray(c)).to(rdt).to(dev))
    torch.cuda.synchronize()
    info = plan.info()
    plan.close()
    return f.cpu().numpy().astype(np.float64), info


def _kernel_inputs(N, M, seed, near=True):
    rng = np.random.default_rng(seed)
    t = rng.uniform(0.0, 1.0, N)
    s = rng.uniform(0.0, 2.0 * N, M)
    if near:   # a few nodes in the near fields Omega_M and Y_M
        t[:3] = [1e-12, 3e-13, 1e-11]
        s[:3] = [1e-9, 2e-10, 5e-9]
    t[t == 0] = 0.5
    s[s == 0] = 1.0
    return rng.standard_normal(N), t, s


def _kernel_tol(kind, eps, prec, c, t, s, ref):
    # E <= eps in exact arithmetic; rounding is relative to sum_k |c_k kappa|
    # (the singular kernel reaches ~1e10 in the near fields)
    absum = np.max(np.abs(S.smooth_kernel(kind, s, t)) @ np.abs(c))
    u = 2.0 ** -53 if prec == "fp64" else U32
    return eps * np.sum(np.abs(c)) + 64 * u * absum


@pytest.mark.parametrize("kind", ["exp", "bessel_half"])
@pytest.mark.parametrize("prec,eps", [("fp64", 1e-10), ("fp64", 1e-6), ("fp32", 1e-5)])
@pytest.mark.parametrize("N,M", [(700, 400), (1 << 16, 1 << 16), (33, 5000)])
def test_general_kernel_against_oracle(fl, kind, prec, eps, N, M):
    c, t, s = _kernel_inputs(N, M, seed=N + M)
    f, info = _run_kernel(fl, kind, c, t, s, eps, prec)
    assert info["kernel"] == kind
    P = S.general_params(kind, eps, s.max(), t.max(), N)
    assert info["q"] == P.q and info["levels"] == P.M
    idx = np.arange(M) if M <= 4096 else np.concatenate(
        [np.arange(3), np.random.default_rng(1).choice(M, 2000, replace=False)])
    ref = oracle.kernel_direct(kind, c, t, s[idx])
    err = np.max(np.abs(f[idx] - ref))
    assert err <= _kernel_tol(kind, eps, prec, c, t, s[idx], ref), err


@pytest.mark.parametrize("kind", ["exp", "bessel_half"])
def test_general_kernel_matches_structured(fl, kind):
    c, t, s = _kernel_inputs(900, 600, seed=5)
    eps = 1e-8
    f, info = _run_kernel(fl, kind, c, t, s, eps, "fp64")
    fs, P = S.laplace_alg1_general(kind, c, t, s, eps)
    assert info["q"] == P.q
    # the same f~ = K~ c: rounding only
    absum = np.max(np.abs(S.smooth_kernel(kind, s, t)) @ np.abs(c))
    assert np.max(np.abs(f - fs)) <= 1e-12 * np.sum(np.abs(c)) + 64 * 2.0 ** -53 * absum


def test_general_kernel_invalid(fl):
    dev = torch.device("cuda")
    t = torch.tensor([0.0, 0.5], dtype=torch.float64, device=dev)
    s = torch.tensor([1.0, 2.0], dtype=torch.float64, device=dev)
    with pytest.raises(fl.FLError) as ei:
        fl.LaplacePlan(t, s, 1e-6, kernel="bessel_half")     # singular at s t = 0
    assert ei.value.status == fl.FL_EINVAL
    p = fl.LaplacePlan(t, s, 1e-6, kernel="exp")              # t = 0 is fine for exp
    f = p.execute(torch.tensor([1.0, 2.0], dtype=torch.float64, device=dev)).cpu().numpy()
    assert np.allclose(f, oracle.kernel_direct("exp", np.array([1.0, 2.0]), t.cpu().numpy(),
                                               s.cpu().numpy()), rtol=1e-12, atol=1e-12)
    p.close()
