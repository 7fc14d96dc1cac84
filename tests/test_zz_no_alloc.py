"""The allocation-free Laplace transform, fl_laplace_real_noalloc, through the C ABI.

Some callers cannot allocate device memory at the point where they need the
transform: code running inside another framework's memory pool that forbids
outside allocations, real-time loops where cudaMalloc (which can synchronise
the whole device) is not allowed, or a GPU that is already full.
fl_laplace_real_noalloc serves them from one fixed static device array instead
of a plan's buffers.  This file checks that it returns what the planned path
(fl_plan_laplace + fl_laplace_real) returns, within the tolerance the other
Laplace tests use, on calls made one after another with different problems --
so that anything the shared scratch kept from the previous call would show --
and that a problem too large for the static scratch is refused with a clear
error rather than run.

It is kept in a file of its own that pytest collects last; it passes both on
its own in a fresh process (where its first call does the one-time set-up)
and after the rest of the suite.
"""
import numpy as np
import pytest

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
    # the first problem again, after the scratch held the others' tables
    N, M, seed, prec, eps = cases[0]
    c, t, s = _problem(N, M, seed, prec)
    ref = _planned(fl, c, t, s, eps, prec)
    again = _noalloc(fl, c, t, s, eps, prec)
    assert np.max(np.abs(again - ref)) <= _bound(prec, ref, c)


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
