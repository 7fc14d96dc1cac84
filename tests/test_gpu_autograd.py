"""Gradients of f = C(w) c through torch.autograd (adjoint and k-weighted transform).

For the loss L = sum_j |f_j - g_j|^2, PyTorch's upstream gradient is
G = 2 (f - g) and the chain rule for the holomorphic map gives
    grad c = C^* G,          grad w_j = G_j conj(f'(w_j)),
with f'(w) = sum_k (2 pi i k) c_k e^{2 pi i k w}.  Checked against
* central finite differences of the oracle loss (small N, FP64 form), and
* the oracle's analytic gradient at the gradient workload's full size
  (N = M = 2^18, disk-uniform nodes, FP32 form) on seeded samples.
The bar is 1e-5 relative (max-norm over the checked entries).
"""
import numpy as np
import pytest

import oracle
from paper_1606_03255_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ag():
    from paper_1606_03255_gb300 import build as libbuild
    libbuild.build()
    from paper_1606_03255_gb300 import autograd
    return autograd


def _rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(np.asarray(b))))


def _loss_oracle(c, w, g):
    f = oracle.flt_direct(c, w)
    return float(np.sum(np.abs(f - g) ** 2))


def test_gradients_against_finite_differences(ag):
    N = M = 256
    c0 = W.coefficients(N, seed=1)
    w0 = W.nodes_disk_uniform(M, seed=2)
    g = W.targets(M, seed=3)
    dev = torch.device("cuda")
    c = torch.from_numpy(c0).to(dev).requires_grad_(True)
    w = torch.from_numpy(w0).to(dev).requires_grad_(True)
    op = ag.FourierLaplace(N, eps=1e-12, precision="fp64")
    f = op(c, w)
    loss = torch.sum(torch.abs(f - torch.from_numpy(g).to(dev)) ** 2)
    loss.backward()
    gc = c.grad.cpu().numpy()
    gw = w.grad.cpu().numpy()
    rng = np.random.default_rng(4)
    # c: L is quadratic in c, so the central difference is exact up to rounding
    h = 1e-4
    ks = rng.choice(N, 8, replace=False)
    fd_c, an_c = [], []
    for k in ks:
        for part, unit in ((0, 1.0), (1, 1j)):
            cp, cm = c0.copy(), c0.copy()
            cp[k] += h * unit
            cm[k] -= h * unit
            fd_c.append((_loss_oracle(cp, w0, g) - _loss_oracle(cm, w0, g)) / (2 * h))
            an_c.append(gc[k].real if part == 0 else gc[k].imag)
    assert _rel(an_c, fd_c) <= 1e-5
    # w: phases move by 2 pi k h, so the step is scaled by 1/(2 pi N)
    hw = 1e-4 / (2 * np.pi * N)
    js = rng.choice(M, 8, replace=False)
    fd_w, an_w = [], []
    for j in js:
        for part in (0, 1):
            wp, wm = w0.copy(), w0.copy()
            wp[j, part] += hw
            wm[j, part] -= hw
            fd_w.append((_loss_oracle(c0, wp, g) - _loss_oracle(c0, wm, g)) / (2 * hw))
            an_w.append(gw[j, part])
    assert _rel(an_w, fd_w) <= 1e-5


@pytest.mark.parametrize("prec,eps,bar", [("fp64", 1e-12, 1e-9), ("fp64ff", 1e-12, 1e-9),
                                          ("fp32", 1e-7, 1e-5)])
def test_gradient_workload_full_size_sampled(ag, prec, eps, bar):
    # N = M = 2^18, disk-uniform nodes, g complex N(0,1), L = sum |f - g|^2
    N = M = 1 << 18
    cdt = torch.complex64 if prec == "fp32" else torch.complex128
    c0 = W.coefficients(N, seed=0).astype(np.complex64 if prec == "fp32" else np.complex128)
    w0 = W.nodes_disk_uniform(M, seed=1)
    g = W.targets(M, seed=2)
    dev = torch.device("cuda")
    c = torch.from_numpy(c0).to(dev).requires_grad_(True)
    w = torch.from_numpy(w0).to(dev).requires_grad_(True)
    f = ag.fourier_laplace(c, w, eps=eps, precision=prec)
    f.retain_grad()
    loss = torch.sum(torch.abs(f - torch.from_numpy(g).to(cdt).to(dev)) ** 2)
    loss.backward()
    G = f.grad.detach().cpu().numpy().astype(np.complex128)   # = 2 (f - g)
    c128 = c0.astype(np.complex128)
    rng = np.random.default_rng(5)
    ks = np.sort(rng.choice(N, 128, replace=False))
    ref_c = oracle.flt_adjoint_at(G, w0, ks)
    assert _rel(c.grad.cpu().numpy()[ks], ref_c) <= bar
    js = np.sort(rng.choice(M, 128, replace=False))
    fprime = oracle.flt_direct(2j * np.pi * np.arange(N) * c128, w0[js])
    ref_w = G[js] * np.conj(fprime)
    got_w = w.grad.cpu().numpy()[js]
    assert _rel(got_w[:, 0] + 1j * got_w[:, 1], ref_w) <= bar


def test_plan_reused_until_nodes_change(ag):
    N = M = 300
    dev = torch.device("cuda")
    c = torch.from_numpy(W.coefficients(N, 0)).to(torch.complex64).to(dev)
    w = torch.from_numpy(W.nodes_disk_uniform(M, 1)).to(dev)
    op = ag.FourierLaplace(N, eps=1e-6)
    op(c, w)
    p1 = op._plan
    op(c, w)
    assert op._plan is p1
    with torch.no_grad():
        w[0, 0] += 0.1
    f = op(c, w)
    assert op._plan is not p1
    ref = oracle.flt_direct(c.cpu().numpy(), w.cpu().numpy())
    assert oracle.error_E(ref, f.cpu().numpy(), c.cpu().numpy()) <= 1e-6
