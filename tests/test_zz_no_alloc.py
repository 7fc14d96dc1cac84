"""The allocation-free Laplace transform, fl_laplace_real_noalloc, through the C ABI.

Some callers cannot allocate device memory at the point where they need the
transform: code running inside another framework's memory pool that forbids
outside allocations, real-time loops where cudaMalloc (which can synchronise
the whole device) is not allowed, or a GPU that is already full.
fl_laplace_real_noalloc serves them from one fixed static device array instead
of a plan's buffers.  This file checks that it returns what the planned path
(fl_plan_laplace + fl_laplace_real) returns, within the tolerance the other
Laplace tests use, on calls made one after another with different problems --
so that anything the shared scratch kept from the previous call would show --;
that it meets the accuracy of Theorem A.3 against the plain FP64 oracle on its
own; that the degenerate problems (no frequencies, no nodes, every node at
s = 0) agree with the planned path; and that a problem too large for the
static scratch is refused with a clear error rather than run, whatever N is.

It is kept in a file of its own that pytest collects last; it passes both on
its own in a fresh process (where its first call does the one-time set-up)
and after the rest of the suite.
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


def _problem(N, M, seed, prec):
    c, t, s = W.laplace_inputs(N, M, seed)
    rdt = torch.float64 if prec == "fp64" else torch.float32
    dev = torch.device("cuda")
    return (torch.from_numpy(c).to(rdt).to(dev), torch.from_numpy(t).to(dev),
            torch.from_numpy(s).to(dev))


def _planned(fl, c, t, s, eps, prec, q=0):
    plan = fl.LaplacePlan(t, s, eps, precision=prec, q=q)
    f = plan.execute(c)
    torch.cuda.synchronize()
    plan.close()
    return f.cpu().numpy().astype(np.float64)


def _noalloc(fl, c, t, s, eps, prec, q=0):
    f = torch.empty(s.numel(), dtype=c.dtype, device=c.device)
    st = fl.fl_laplace_real_noalloc(t.numel(), s.numel(), t.data_ptr(), s.data_ptr(),
                                    c.data_ptr(), f.data_ptr(), q, eps,
                                    fl.FL_FP64 if prec == "fp64" else fl.FL_FP32,
                                    torch.cuda.current_stream().cuda_stream)
    fl.check(st, "fl_laplace_real_noalloc")
    torch.cuda.synchronize()
    return f.cpu().numpy().astype(np.float64)


def _status(fl, N, M, t, s, c, f, q, eps, prec):
    return fl.fl_laplace_real_noalloc(N, M, t.data_ptr(), s.data_ptr(), c.data_ptr(),
                                      f.data_ptr(), q, eps,
                                      fl.FL_FP64 if prec == "fp64" else fl.FL_FP32,
                                      torch.cuda.current_stream().cuda_stream)


def _oracle_tol(eps, prec, ref, c):
    # Theorem A.3 (E <= eps), plus the float rounding term of the FP32 form
    if prec == "fp64":
        return eps
    return eps + 32 * U32 * max(float(np.max(np.abs(ref))), 1.0) / max(float(np.sum(np.abs(c))), 1e-300)


def _bound(prec, ref, c):
    # the Laplace tests' tolerance between two GPU results of the same f~
    csum = float(torch.sum(torch.abs(c.double())).item())
    if prec == "fp64":
        return 1e-12 * csum
    return 32 * U32 * max(float(np.max(np.abs(ref))), 1.0)


def test_noalloc_matches_planned_path_on_consecutive_calls(fl):
    cases = [
        (1 << 16, 1 << 16, 0, "fp64", 1e-6),   # the 2^16 Laplace workload
        (5000, 3000, 1, "fp32", 1e-4),         # fewer levels, float data
        (777, 12345, 2, "fp64", 1e-10),        # more levels than the first
    ]
    for N, M, seed, prec, eps in cases:
        c, t, s = _problem(N, M, seed, prec)
        ref = _planned(fl, c, t, s, eps, prec)
        got = _noalloc(fl, c, t, s, eps, prec)
        assert np.max(np.abs(got - ref)) <= _bound(prec, ref, c), (N, M, prec)
        # and on its own against the plain FP64 sum (same c bits as the GPU)
        ch = c.double().cpu().numpy()
        exact = oracle.laplace_direct(ch, t.cpu().numpy(), s.cpu().numpy())
        assert oracle.error_E(exact, got, ch) <= _oracle_tol(eps, prec, exact, ch), (N, M, prec)
    # the first problem again, after the scratch held the others' tables
    N, M, seed, prec, eps = cases[0]
    c, t, s = _problem(N, M, seed, prec)
    ref = _planned(fl, c, t, s, eps, prec)
    again = _noalloc(fl, c, t, s, eps, prec)
    assert np.max(np.abs(again - ref)) <= _bound(prec, ref, c)


def test_noalloc_degenerate_problems(fl):
    # N = 0 (no moments: the sums start from zero), M = 0 (nothing to evaluate)
    # and every s_j = 0 (a single level: f_j = sum_k c_k), in both precisions,
    # one call after another
    for prec in ("fp64", "fp32"):
        for N, M, zero_s in ((0, 17, False), (300, 0, False), (500, 40, True), (1, 1, False)):
            c, t, s = _problem(N, M, 20 + N + M, prec)
            if zero_s:
                s = torch.zeros_like(s)
            eps = 1e-8 if prec == "fp64" else 1e-5
            got = _noalloc(fl, c, t, s, eps, prec)
            ref = _planned(fl, c, t, s, eps, prec)
            assert got.shape == ref.shape == (M,)
            if M == 0:
                continue
            if N == 0:
                assert np.all(got == 0)
                continue
            if zero_s:
                # f_j = sum_k c_k: two summation orders differ at the scale
                # u sum_k |c_k| of a rounded sum, not at the scale of |f_j|
                u = 2.0 ** -53 if prec == "fp64" else U32
                tol = 32 * u * float(torch.sum(torch.abs(c.double())).item())
                total = float(torch.sum(c.double()).item())
                assert np.max(np.abs(got - ref)) <= tol, (prec, N, M)
                assert np.max(np.abs(got - total)) <= tol, (prec, N, M)
                continue
            assert np.max(np.abs(got - ref)) <= _bound(prec, ref, c), (prec, N, M)


def _wide_problem(N, M, smax, seed, prec):
    # t in [0, 1] with max t = 1 and s in [0, smax] with max s = smax: the
    # number of levels, ceil(log2(smax / eps)) + 1, does not depend on N
    c, t, s = _problem(N, M, seed, prec)
    t[0] = 1.0
    s = s / s.max() * smax
    s[0] = smax
    return c, t, s


def test_noalloc_refuses_problems_beyond_its_scratch(fl):
    # q = 40 with ~62 levels needs ~10 MB of moment tables: above the 2 MiB array
    N, M = 40000, 100
    c, t, s = _problem(N, M, 3, "fp64")
    s = s * 1e3
    f = torch.empty(M, dtype=torch.float64, device="cuda")
    st = fl.fl_laplace_real_noalloc(N, M, t.data_ptr(), s.data_ptr(), c.data_ptr(),
                                    f.data_ptr(), 40, 1e-12, fl.FL_FP64,
                                    torch.cuda.current_stream().cuda_stream)
    assert st == fl.FL_EUNSUPPORTED
    msg = fl.fl_last_error()
    assert "bytes" in msg and "static maximum" in msg
    # and it still works for a problem that fits
    c2, t2, s2 = _problem(2000, 500, 4, "fp64")
    ref = _planned(fl, c2, t2, s2, 1e-8, "fp64")
    assert np.max(np.abs(_noalloc(fl, c2, t2, s2, 1e-8, "fp64") - ref)) <= _bound("fp64", ref, c2)


def test_noalloc_limit_does_not_depend_on_n(fl):
    # 70 levels (eps = 1e-12, max s max t = 4e8): q = 30 needs more than the
    # 2 MiB array and is refused at N = 300 as at N = 40000; q = 20 fits at both
    eps, smax = 1e-12, 4e8
    for N in (300, 40000):
        c, t, s = _wide_problem(N, 64, smax, 30 + N, "fp64")
        f = torch.empty(64, dtype=torch.float64, device="cuda")
        assert _status(fl, N, 64, t, s, c, f, 30, eps, "fp64") == fl.FL_EUNSUPPORTED, N
        assert "static maximum" in fl.fl_last_error()
        got = _noalloc(fl, c, t, s, eps, "fp64", q=20)
        ref = _planned(fl, c, t, s, eps, "fp64", q=20)
        assert np.max(np.abs(got - ref)) <= _bound("fp64", ref, c), N
    # FP32 data: 101 levels (eps = 1e-10, max s max t = 2^66) at q = 40 is
    # refused at a small N too, with the array unchanged for the next call
    N, M = 300, 32
    c, t, s = _wide_problem(N, M, 2.0 ** 66, 5, "fp32")
    f = torch.empty(M, dtype=torch.float32, device="cuda")
    assert _status(fl, N, M, t, s, c, f, 40, 1e-10, "fp32") == fl.FL_EUNSUPPORTED
    assert "static maximum" in fl.fl_last_error()
    c2, t2, s2 = _problem(3000, 200, 6, "fp32")
    ref = _planned(fl, c2, t2, s2, 1e-5, "fp32")
    assert np.max(np.abs(_noalloc(fl, c2, t2, s2, 1e-5, "fp32") - ref)) <= _bound("fp32", ref, c2)
