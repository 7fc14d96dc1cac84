"""The C ABI library loads and exports every symbol include/fl.h declares, and
its host-side argument checks work without a GPU."""
import ctypes
import os
import re

import pytest

from paper_1606_03255_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fl():
    libbuild.build()
    from paper_1606_03255_gb300 import fl as flmod
    flmod.load()
    return flmod


def declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(fl_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(fl):
    names = declared_functions()
    assert "fl_plan" in names and "fl_execute" in names and "fl_laplace_real" in names
    lib = ctypes.CDLL(fl.library_path())
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(fl.EXPORTED) == names


def test_version_and_error_string(fl):
    assert "sm_103a" in fl.fl_version()
    assert isinstance(fl.fl_last_error(), str)


@pytest.mark.parametrize("N,M,eps,q,prec", [
    (0, 10, 1e-6, 0, 0),          # N < 1
    (10, -1, 1e-6, 0, 0),         # M < 0
    (10, 10, 0.0, 0, 0),          # eps outside (0, 1)
    (10, 10, 1.5, 0, 0),
    (10, 10, 1e-6, -1, 0),        # q outside [0, 40]
    (10, 10, 1e-6, 41, 0),
    (10, 10, 1e-6, 0, 7),         # unknown precision
    (10, 10, 1e-6, 0, 0),         # NULL nodes with M > 0
])
def test_plan_rejects_bad_arguments_on_host(fl, N, M, eps, q, prec):
    st, h = fl.fl_plan(N, M, None, q, eps, prec, None)
    assert st == fl.FL_EINVAL
    assert not h.value
    assert "fl_plan" in fl.fl_last_error()


def test_plan_rejects_too_large(fl):
    st, h = fl.fl_plan((1 << 23) + 1, 1, None, 0, 1e-6, 0, None)
    assert st == fl.FL_EUNSUPPORTED


def test_null_handles(fl):
    st, _ = fl.fl_get_info(None)
    assert st == fl.FL_EINVAL
    assert fl.fl_execute(None, None, None, None) == fl.FL_EINVAL
    assert fl.fl_adjoint(None, None, None, None) == fl.FL_EINVAL
    assert fl.fl_set_timing(None, 1) == fl.FL_EINVAL
    fl.fl_destroy(None)


def _options(fl, **kw):
    opt = fl.fl_options()
    for k, v in kw.items():
        setattr(opt, k, v)
    return opt


@pytest.mark.parametrize("field,value", [("shared_nodes", 2), ("shared_nodes", -1),
                                         ("oversampling", 3), ("fuse_gather", 3), ("route", 3)])
def test_invalid_options_rejected_on_host(fl, field, value):
    nodes = (ctypes.c_double * 4)()   # never read: the options are checked first
    ptr = ctypes.cast(nodes, ctypes.c_void_p)
    st, h = fl.fl_plan_ex(4, 2, ptr, 0, 1e-6, 0, _options(fl, **{field: value}), None)
    assert st == fl.FL_EINVAL and not h.value
    st, h = fl.fl_plan_batched([4, 4], [2, 2], ptr, 0, 1e-6, 0, _options(fl, **{field: value}), None)
    assert st == fl.FL_EINVAL and not h.value


def test_shared_nodes_need_equal_node_counts(fl):
    nodes = (ctypes.c_double * 8)()
    ptr = ctypes.cast(nodes, ctypes.c_void_p)
    st, h = fl.fl_plan_batched([4, 8, 4], [2, 3, 2], ptr, 0, 1e-6, 0, _options(fl, shared_nodes=1), None)
    assert st == fl.FL_EINVAL and not h.value
    assert "shared nodes" in fl.fl_last_error()


def test_pointer_batched_calls_check_arguments_on_host(fl):
    # a transform with nodes and a NULL node pointer, and a NULL plan
    st, h = fl.fl_plan_batched_ptrs([4, 4], [2, 3], [None, None], 0, 1e-6, 0, None, None)
    assert st == fl.FL_EINVAL and not h.value
    assert "NULL" in fl.fl_last_error()
    st, h = fl.fl_plan_batched_ptrs([4, 4], [-1, 3], [None, None], 0, 1e-6, 0, None, None)
    assert st == fl.FL_EINVAL and not h.value
    assert fl.fl_execute_batched_ptrs(None, [None], [None], None) == fl.FL_EINVAL
