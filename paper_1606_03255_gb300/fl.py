"""ctypes binding of libfl.so with the names of the C ABI in include/fl.h.

Argument marshalling only: every step of the transform runs in the library's
CUDA kernels.  There is no CPU fallback -- if ``_build/libfl.so`` is missing
the import raises, and ``paper_1606_03255_gb300.build.build()`` creates it.

Two layers:

* ``fl_plan``, ``fl_execute``, ``fl_adjoint``, ... -- the C calls, taking raw
  pointers (ints) and sizes, returning ``fl_status`` codes;
* ``Plan`` / ``LaplacePlan`` -- thin owners of a plan handle that take torch
  tensors, check dtype/device/shape and raise ``FLError`` on a non-zero status.
  ``Plan(route=...)``: "auto" (NFFT or direct sum per band by cost), "nfft"
  (every band by NFFT, Algorithm 2 as printed) or "direct".
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

FL_OK, FL_EINVAL, FL_ENOMEM, FL_ECUDA, FL_ETIMEOUT, FL_EUNSUPPORTED = range(6)
FL_FP32, FL_FP64, FL_FP64_FF = 0, 1, 2
# "fp64ff": complex128 in and out, band-grid FFTs in float pairs
PRECISIONS = {"fp32": FL_FP32, "fp64": FL_FP64, "fp64ff": FL_FP64_FF}
FL_MAX_LEVELS = 128
FL_MAX_TIMED_KERNELS = 16

STATUS_NAMES = {FL_OK: "FL_OK", FL_EINVAL: "FL_EINVAL", FL_ENOMEM: "FL_ENOMEM",
                FL_ECUDA: "FL_ECUDA", FL_ETIMEOUT: "FL_ETIMEOUT",
                FL_EUNSUPPORTED: "FL_EUNSUPPORTED"}

# Every symbol include/fl.h declares.
EXPORTED = ["fl_plan", "fl_plan_ex", "fl_plan_batched", "fl_execute_batched", "fl_plan_batched_ptrs",
            "fl_execute_batched_ptrs", "fl_execute", "fl_execute_deriv", "fl_grad_w", "fl_execute_host",
            "fl_adjoint", "fl_transposed", "fl_plan_xi",
            "fl_plan_laplace", "fl_plan_kernel", "fl_laplace_real", "fl_laplace_real_noalloc", "fl_get_info",
            "fl_set_timing", "fl_get_timing", "fl_destroy", "fl_last_error", "fl_version"]


class fl_info(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int), ("precision", ctypes.c_int),
        ("N", ctypes.c_int64), ("M", ctypes.c_int64),
        ("eps", ctypes.c_double), ("eps_laplace", ctypes.c_double),
        ("eps_fourier", ctypes.c_double),
        ("q", ctypes.c_int), ("levels", ctypes.c_int), ("m_w", ctypes.c_int),
        ("sigma", ctypes.c_int),
        ("y1", ctypes.c_double), ("xi1", ctypes.c_double),
        ("z0_nodes", ctypes.c_int64), ("batch", ctypes.c_int),
        ("n_bands_fft", ctypes.c_int), ("n_bands_direct", ctypes.c_int),
        ("band_ell", ctypes.c_int * FL_MAX_LEVELS),
        ("band_route", ctypes.c_int * FL_MAX_LEVELS),
        ("band_nodes", ctypes.c_int64 * FL_MAX_LEVELS),
        ("band_K", ctypes.c_int64 * FL_MAX_LEVELS),
        ("band_n", ctypes.c_int64 * FL_MAX_LEVELS),
        ("model_bytes", ctypes.c_double), ("direct_bias", ctypes.c_double),
        ("scratch_bytes", ctypes.c_double), ("variant", ctypes.c_int), ("kernel", ctypes.c_int),
        ("n_bands_fused", ctypes.c_int), ("fused_entries", ctypes.c_int64),
        ("sigma_min", ctypes.c_double), ("band_parts", ctypes.c_int * FL_MAX_LEVELS),
        ("rhs_per_launch", ctypes.c_int), ("oversampling", ctypes.c_int),
        ("fuse_gather", ctypes.c_int), ("autotuned", ctypes.c_int)]


class fl_options(ctypes.Structure):
    _fields_ = [("route", ctypes.c_int), ("direct_bias", ctypes.c_double),
                ("rhs_per_launch", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("autotune", ctypes.c_int), ("variant", ctypes.c_int),
                ("fuse_gather", ctypes.c_int), ("oversampling", ctypes.c_int),
                ("shared_nodes", ctypes.c_int)]


ROUTES = {"auto": 0, "nfft": 1, "direct": 2}
# window gather inside the FFT's second pass (FP32 forward): by cost, never, always
FUSE = {"auto": 0, "off": 1, "on": 2}
# oversampling of the band grids: by cost, 2 everywhere, sub-bands wherever allowed
SIGMA = {"auto": 0, "2": 1, "min": 2}
# band weights: Algorithm 2 (two-sided interpolation) or the one-sided variant
VARIANTS = {"alg2": 0, "onesided": 1}
# kernels of fl_plan_kernel (generalised Algorithm 1)
KERNELS = {"laplace": 0, "exp": 1, "bessel_half": 2}


class fl_timing(ctypes.Structure):
    _fields_ = [
        ("n_kernels", ctypes.c_int),
        ("name", (ctypes.c_char * 32) * FL_MAX_TIMED_KERNELS),
        ("launches", ctypes.c_int64 * FL_MAX_TIMED_KERNELS),
        ("total_ms", ctypes.c_double * FL_MAX_TIMED_KERNELS),
        ("bytes", ctypes.c_double * FL_MAX_TIMED_KERNELS),
        ("total_launches", ctypes.c_int64),
    ]


class FLError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libfl.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise OSError(f"libfl.so not built at {path}; run paper_1606_03255_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i64, ci, cd = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    pp = ctypes.POINTER(vp)
    sig = {
        "fl_plan": [pp, i64, i64, vp, ci, cd, ci, vp],
        "fl_plan_ex": [pp, i64, i64, vp, ci, cd, ci, ctypes.POINTER(fl_options), vp],
        "fl_plan_batched": [pp, ci, ctypes.POINTER(i64), ctypes.POINTER(i64), vp, ci, cd, ci,
                            ctypes.POINTER(fl_options), vp],
        "fl_execute_batched": [vp, vp, vp, vp],
        "fl_plan_batched_ptrs": [pp, ci, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(vp), ci, cd,
                                 ci, ctypes.POINTER(fl_options), vp],
        "fl_execute_batched_ptrs": [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp],
        "fl_execute": [vp, vp, vp, vp],
        "fl_execute_deriv": [vp, vp, vp, vp],
        "fl_grad_w": [vp, vp, vp, vp, vp],
        "fl_execute_host": [vp, vp, vp, vp],
        "fl_adjoint": [vp, vp, vp, vp],
        "fl_transposed": [vp, vp, vp, vp],
        "fl_plan_xi": [pp, i64, vp, i64, vp, ci, cd, ci, vp],
        "fl_plan_laplace": [pp, i64, i64, vp, vp, ci, cd, ci, vp],
        "fl_plan_kernel": [pp, ci, i64, i64, vp, vp, ci, cd, ci, vp],
        "fl_laplace_real": [vp, vp, vp, vp],
        "fl_laplace_real_noalloc": [i64, i64, vp, vp, vp, vp, ci, cd, ci, vp],
        "fl_get_info": [vp, ctypes.POINTER(fl_info)],
        "fl_set_timing": [vp, ci],
        "fl_get_timing": [vp, ctypes.POINTER(fl_timing)],
        "fl_destroy": [vp],
        "fl_last_error": [],
        "fl_version": [],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ci
    lib.fl_destroy.restype = None
    lib.fl_last_error.restype = ctypes.c_char_p
    lib.fl_version.restype = ctypes.c_char_p
    _lib = lib
    return lib


# ---------------------------------------------------------------------------
# The C calls, same names and argument order as include/fl.h.

def fl_plan(N, M, nodes_ptr, q, eps, prec, stream):
    h = ctypes.c_void_p()
    st = load().fl_plan(ctypes.byref(h), int(N), int(M), nodes_ptr, int(q), float(eps),
                        int(prec), stream)
    return st, h


def fl_plan_ex(N, M, nodes_ptr, q, eps, prec, options, stream):
    h = ctypes.c_void_p()
    opt = ctypes.byref(options) if options is not None else None
    st = load().fl_plan_ex(ctypes.byref(h), int(N), int(M), nodes_ptr, int(q), float(eps),
                           int(prec), opt, stream)
    return st, h


def fl_plan_batched(Ns, Ms, nodes_ptr, q, eps, prec, options, stream):
    h = ctypes.c_void_p()
    B = len(Ns)
    na = (ctypes.c_int64 * B)(*[int(x) for x in Ns])
    ma = (ctypes.c_int64 * B)(*[int(x) for x in Ms])
    opt = ctypes.byref(options) if options is not None else None
    st = load().fl_plan_batched(ctypes.byref(h), B, na, ma, nodes_ptr, int(q), float(eps),
                                int(prec), opt, stream)
    return st, h


def fl_execute_batched(plan, c_ptr, f_ptr, stream):
    return load().fl_execute_batched(plan, c_ptr, f_ptr, stream)


def fl_plan_batched_ptrs(Ns, Ms, node_ptrs, q, eps, prec, options, stream):
    h = ctypes.c_void_p()
    B = len(Ns)
    na = (ctypes.c_int64 * B)(*[int(x) for x in Ns])
    ma = (ctypes.c_int64 * B)(*[int(x) for x in Ms])
    pa = (ctypes.c_void_p * B)(*node_ptrs)
    opt = ctypes.byref(options) if options is not None else None
    st = load().fl_plan_batched_ptrs(ctypes.byref(h), B, na, ma, pa, int(q), float(eps), int(prec), opt, stream)
    return st, h


def fl_execute_batched_ptrs(plan, c_ptrs, f_ptrs, stream):
    B = len(c_ptrs)
    ca = (ctypes.c_void_p * B)(*c_ptrs)
    fa = (ctypes.c_void_p * B)(*f_ptrs)
    return load().fl_execute_batched_ptrs(plan, ca, fa, stream)


def fl_execute(plan, c_ptr, f_ptr, stream):
    return load().fl_execute(plan, c_ptr, f_ptr, stream)


def fl_execute_deriv(plan, c_ptr, f_ptr, stream):
    return load().fl_execute_deriv(plan, c_ptr, f_ptr, stream)


def fl_grad_w(plan, c_ptr, r_ptr, gw_ptr, stream):
    return load().fl_grad_w(plan, c_ptr, r_ptr, gw_ptr, stream)


def fl_execute_host(plan, c_ptr, f_ptr, stream):
    return load().fl_execute_host(plan, c_ptr, f_ptr, stream)


def fl_adjoint(plan, r_ptr, c_out_ptr, stream):
    return load().fl_adjoint(plan, r_ptr, c_out_ptr, stream)


def fl_transposed(plan, g_ptr, out_ptr, stream):
    return load().fl_transposed(plan, g_ptr, out_ptr, stream)


def fl_plan_xi(N, xi_ptr, M, nodes_ptr, q, eps, prec, stream):
    h = ctypes.c_void_p()
    st = load().fl_plan_xi(ctypes.byref(h), int(N), xi_ptr, int(M), nodes_ptr, int(q), float(eps),
                           int(prec), stream)
    return st, h


def fl_plan_laplace(N, M, t_ptr, s_ptr, q, eps, prec, stream):
    h = ctypes.c_void_p()
    st = load().fl_plan_laplace(ctypes.byref(h), int(N), int(M), t_ptr, s_ptr, int(q),
                                float(eps), int(prec), stream)
    return st, h


def fl_plan_kernel(kernel, N, M, t_ptr, s_ptr, q, eps, prec, stream):
    h = ctypes.c_void_p()
    st = load().fl_plan_kernel(ctypes.byref(h), int(kernel), int(N), int(M), t_ptr, s_ptr, int(q),
                               float(eps), int(prec), stream)
    return st, h


def fl_laplace_real(plan, c_ptr, f_ptr, stream):
    return load().fl_laplace_real(plan, c_ptr, f_ptr, stream)


def fl_laplace_real_noalloc(N, M, t_ptr, s_ptr, c_ptr, f_ptr, q, eps, prec, stream):
    """Laplace transform without any device allocation (static 2 MiB scratch).

    For callers that cannot allocate device memory where they need the
    transform; see include/fl.h for the limits and the one-time set-up.
    """
    return load().fl_laplace_real_noalloc(int(N), int(M), t_ptr, s_ptr, c_ptr, f_ptr, int(q),
                                          float(eps), int(prec), stream)


def fl_get_info(plan):
    info = fl_info()
    st = load().fl_get_info(plan, ctypes.byref(info))
    return st, info


def fl_set_timing(plan, enable):
    return load().fl_set_timing(plan, int(bool(enable)))


def fl_get_timing(plan):
    t = fl_timing()
    st = load().fl_get_timing(plan, ctypes.byref(t))
    return st, t


def fl_destroy(plan):
    load().fl_destroy(plan)


def fl_last_error() -> str:
    return load().fl_last_error().decode()


def fl_version() -> str:
    return load().fl_version().decode()


def check(status: int, what: str = "") -> None:
    if status != FL_OK:
        raise FLError(status, f"{what}: {fl_last_error()}" if what else fl_last_error())


# ---------------------------------------------------------------------------
# Tensor-level helpers.

def _precision(name: str) -> int:
    if name not in PRECISIONS:
        raise ValueError(f"precision must be one of {sorted(PRECISIONS)}, not {name!r}")
    return PRECISIONS[name]


def _torch():
    import torch
    return torch


def _stream_handle(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t) -> int:
    return int(t.data_ptr())


def _require(t, dtype, numel: int, name: str):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if t.numel() != numel or not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous with {numel} elements")


def info_dict(info: fl_info) -> dict:
    nb = info.levels + 1
    return {
        "kind": info.kind, "precision": info.precision, "N": info.N, "M": info.M,
        "eps": info.eps, "eps_laplace": info.eps_laplace, "eps_fourier": info.eps_fourier,
        "q": info.q, "levels": info.levels, "m_w": info.m_w, "sigma": info.sigma,
        "y1": info.y1, "xi1": info.xi1, "z0_nodes": info.z0_nodes, "batch": info.batch,
        "n_bands_fft": info.n_bands_fft, "n_bands_direct": info.n_bands_direct,
        "band_ell": list(info.band_ell[:nb]), "band_route": list(info.band_route[:nb]),
        "band_nodes": list(info.band_nodes[:nb]), "band_K": list(info.band_K[:nb]),
        "band_n": list(info.band_n[:nb]),
        "model_bytes": info.model_bytes, "direct_bias": info.direct_bias,
        "scratch_bytes": info.scratch_bytes,
        "variant": {v: k for k, v in VARIANTS.items()}.get(info.variant, info.variant),
        "kernel": {v: k for k, v in KERNELS.items()}.get(info.kernel, info.kernel),
        "n_bands_fused": info.n_bands_fused, "fused_entries": info.fused_entries,
        "sigma_min": info.sigma_min, "band_parts": list(info.band_parts[:nb]),
        "rhs_per_launch": info.rhs_per_launch,
        "oversampling": {v: k for k, v in SIGMA.items()}.get(info.oversampling, info.oversampling),
        "fuse_gather": {v: k for k, v in FUSE.items()}.get(info.fuse_gather, info.fuse_gather),
        "autotuned": bool(info.autotuned),
    }


def timing_dict(t: fl_timing) -> dict:
    out = {}
    for i in range(t.n_kernels):
        name = bytes(t.name[i]).split(b"\0", 1)[0].decode()
        out[name] = {"launches": int(t.launches[i]), "total_ms": float(t.total_ms[i]),
                     "bytes": float(t.bytes[i])}
    return {"kernels": out, "total_launches": int(t.total_launches)}


class Plan:
    """Owner of an Algorithm-2 plan: f = sum_k c_k exp(2 pi i k w_j).

    nodes: CUDA float64 tensor (M, 2) of (Re w, Im w), or complex128 (M,).
    precision: "fp32" (complex64 c/f), "fp64" (complex128 c/f) or "fp64ff"
    (complex128 c/f, band-grid FFTs in float pairs; batched plans forward only).
    """

    def __init__(self, N: int, nodes, eps: float, precision: str = "fp32", q: int = 0,
                 stream=None, route: str = "auto", direct_bias: float = 1.0,
                 rhs_per_launch: int = 0, use_graph: bool = False, autotune: bool = False,
                 variant: str = "alg2", fuse: str = "auto", sigma: str = "auto"):
        torch = _torch()
        if nodes.is_complex():
            nodes = torch.view_as_real(nodes.to(torch.complex128))
        nodes = nodes.to(torch.float64).contiguous()
        self.N = int(N)
        self.M = int(nodes.shape[0]) if nodes.dim() else 0
        self.prec = _precision(precision)
        self.cdtype = torch.complex64 if self.prec == FL_FP32 else torch.complex128
        self._handle = None
        opt = fl_options(ROUTES[route], float(direct_bias), int(rhs_per_launch), int(bool(use_graph)),
                         int(bool(autotune)), VARIANTS[variant], FUSE[fuse], SIGMA[str(sigma)])
        st, h = fl_plan_ex(self.N, self.M, _ptr(nodes) if self.M else None, q, eps, self.prec,
                           opt, _stream_handle(stream))
        check(st, "fl_plan")
        self._handle = h

    @property
    def handle(self):
        return self._handle

    def execute(self, c, out=None, stream=None, deriv: bool = False):
        torch = _torch()
        _require(c, self.cdtype, self.N, "c")
        if out is None:
            out = torch.empty(self.M, dtype=self.cdtype, device=c.device)
        _require(out, self.cdtype, self.M, "out")
        fn = fl_execute_deriv if deriv else fl_execute
        check(fn(self._handle, _ptr(c), _ptr(out) if self.M else None, _stream_handle(stream)),
              "fl_execute")
        return out

    def grad_w(self, c, r, out=None, stream=None):
        """gw_j = r_j conj(df/dw (w_j)): node gradient for upstream gradient r."""
        torch = _torch()
        _require(c, self.cdtype, self.N, "c")
        _require(r, self.cdtype, self.M, "r")
        if out is None:
            out = torch.empty(self.M, dtype=self.cdtype, device=c.device)
        _require(out, self.cdtype, self.M, "out")
        check(fl_grad_w(self._handle, _ptr(c), _ptr(r) if self.M else None,
                        _ptr(out) if self.M else None, _stream_handle(stream)), "fl_grad_w")
        return out

    def adjoint(self, r, out=None, stream=None):
        torch = _torch()
        _require(r, self.cdtype, self.M, "r")
        if out is None:
            out = torch.empty(self.N, dtype=self.cdtype, device=r.device)
        _require(out, self.cdtype, self.N, "out")
        check(fl_adjoint(self._handle, _ptr(r) if self.M else None, _ptr(out),
                         _stream_handle(stream)), "fl_adjoint")
        return out

    def transposed(self, g, out=None, stream=None):
        """out_k = sum_j g_j z_j^k, k < N (C^T g)."""
        torch = _torch()
        _require(g, self.cdtype, self.M, "g")
        if out is None:
            out = torch.empty(self.N, dtype=self.cdtype, device=g.device)
        _require(out, self.cdtype, self.N, "out")
        check(fl_transposed(self._handle, _ptr(g) if self.M else None, _ptr(out),
                            _stream_handle(stream)), "fl_transposed")
        return out

    def execute_host(self, c_host, f_host, stream=None):
        """c_host, f_host: CPU tensors (ideally pinned) of the plan's complex dtype."""
        check(fl_execute_host(self._handle, _ptr(c_host), _ptr(f_host), _stream_handle(stream)),
              "fl_execute_host")
        return f_host

    def info(self) -> dict:
        st, inf = fl_get_info(self._handle)
        check(st, "fl_get_info")
        return info_dict(inf)

    def set_timing(self, enable: bool):
        check(fl_set_timing(self._handle, enable), "fl_set_timing")

    def timing(self) -> dict:
        st, t = fl_get_timing(self._handle)
        check(st, "fl_get_timing")
        return timing_dict(t)

    def close(self):
        if self._handle is not None and self._handle.value:
            fl_destroy(self._handle)
        self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchedPlan:
    """B independent transforms f_i = C_i c_i in one plan (fl_plan_batched).

    Ns, Ms: sizes per transform; nodes: CUDA float64 (sum Ms, 2), the nodes of
    transform 0, 1, ... in order, or with shared_nodes=True the (M, 2) node
    set of every transform (Ms may then be omitted: M for each).  execute(c)
    takes the coefficients of all transforms concatenated (sum Ns) and returns
    the results concatenated.
    """

    def __init__(self, Ns, Ms, nodes, eps: float, precision: str = "fp32", q: int = 0,
                 stream=None, route: str = "auto", direct_bias: float = 1.0,
                 rhs_per_launch: int = 0, use_graph: bool = True, autotune: bool = False,
                 variant: str = "alg2", fuse: str = "auto", sigma: str = "auto",
                 shared_nodes: bool = False):
        torch = _torch()
        per_transform = isinstance(nodes, (list, tuple))
        if per_transform:
            nodes = [w.to(torch.float64).contiguous() for w in nodes]
        else:
            nodes = nodes.to(torch.float64).contiguous()
        self.Ns = [int(x) for x in Ns]
        if shared_nodes and Ms is None:
            Ms = [int((nodes[0] if per_transform else nodes).shape[0])] * len(self.Ns)
        self.Ms = [int(x) for x in Ms]
        self.N, self.M = sum(self.Ns), sum(self.Ms)
        self.prec = _precision(precision)
        self.cdtype = torch.complex64 if self.prec == FL_FP32 else torch.complex128
        self._handle = None
        opt = fl_options(ROUTES[route], float(direct_bias), int(rhs_per_launch),
                         1 if use_graph else -1, int(bool(autotune)), VARIANTS[variant], FUSE[fuse],
                         SIGMA[str(sigma)], int(bool(shared_nodes)))
        if per_transform:   # one node tensor per transform (fl_plan_batched_ptrs)
            st, h = fl_plan_batched_ptrs(self.Ns, self.Ms, [_ptr(w) if w.numel() else None for w in nodes],
                                         q, eps, self.prec, opt, _stream_handle(stream))
            check(st, "fl_plan_batched_ptrs")
        else:
            st, h = fl_plan_batched(self.Ns, self.Ms, _ptr(nodes) if self.M else None, q, eps,
                                    self.prec, opt, _stream_handle(stream))
            check(st, "fl_plan_batched")
        self._handle = h

    @property
    def handle(self):
        return self._handle

    def execute(self, c, out=None, stream=None):
        torch = _torch()
        _require(c, self.cdtype, self.N, "c")
        if out is None:
            out = torch.empty(self.M, dtype=self.cdtype, device=c.device)
        _require(out, self.cdtype, self.M, "out")
        check(fl_execute_batched(self._handle, _ptr(c), _ptr(out) if self.M else None,
                                 _stream_handle(stream)), "fl_execute_batched")
        return out

    def execute_list(self, cs, outs=None, stream=None):
        """The batch on per-transform tensors (fl_execute_batched_ptrs): cs[i]
        holds N_i coefficients; returns (or fills) one result tensor per
        transform."""
        torch = _torch()
        if len(cs) != len(self.Ns):
            raise ValueError("execute_list: one coefficient tensor per transform")
        for c, n in zip(cs, self.Ns):
            _require(c, self.cdtype, n, "c")
        if outs is None:
            outs = [torch.empty(m, dtype=self.cdtype, device=cs[0].device) for m in self.Ms]
        for o, m in zip(outs, self.Ms):
            _require(o, self.cdtype, m, "out")
        check(fl_execute_batched_ptrs(self._handle, [_ptr(c) for c in cs],
                                      [_ptr(o) if o.numel() else None for o in outs],
                                      _stream_handle(stream)), "fl_execute_batched_ptrs")
        return outs

    def info(self) -> dict:
        st, inf = fl_get_info(self._handle)
        check(st, "fl_get_info")
        return info_dict(inf)

    def set_timing(self, enable: bool):
        check(fl_set_timing(self._handle, enable), "fl_set_timing")

    def timing(self) -> dict:
        st, t = fl_get_timing(self._handle)
        check(st, "fl_get_timing")
        return timing_dict(t)

    def close(self):
        if self._handle is not None and self._handle.value:
            fl_destroy(self._handle)
        self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class XiPlan:
    """Owner of a real-exponent plan: f_j = sum_k c_k exp(2 pi i xi_k w_j), xi_k >= 1.

    xi: CUDA float64 tensor (N,); nodes: CUDA float64 (M, 2) with |Re w| <= 1/2.
    """

    def __init__(self, xi, nodes, eps: float, precision: str = "fp32", q: int = 0, stream=None):
        torch = _torch()
        xi = xi.to(torch.float64).contiguous()
        nodes = nodes.to(torch.float64).contiguous()
        self.N = int(xi.numel())
        self.M = int(nodes.shape[0]) if nodes.dim() else 0
        self.prec = _precision(precision)
        self.cdtype = torch.complex64 if self.prec == FL_FP32 else torch.complex128
        self._handle = None
        st, h = fl_plan_xi(self.N, _ptr(xi), self.M, _ptr(nodes) if self.M else None, q, eps,
                           self.prec, _stream_handle(stream))
        check(st, "fl_plan_xi")
        self._handle = h

    @property
    def handle(self):
        return self._handle

    def execute(self, c, out=None, stream=None):
        torch = _torch()
        _require(c, self.cdtype, self.N, "c")
        if out is None:
            out = torch.empty(self.M, dtype=self.cdtype, device=c.device)
        _require(out, self.cdtype, self.M, "out")
        check(fl_execute(self._handle, _ptr(c), _ptr(out) if self.M else None,
                         _stream_handle(stream)), "fl_execute")
        return out

    def adjoint(self, r, out=None, stream=None):
        """out_k = sum_j conj(z_j^{xi_k}) r_j (C^* r), in the order of xi."""
        torch = _torch()
        _require(r, self.cdtype, self.M, "r")
        if out is None:
            out = torch.empty(self.N, dtype=self.cdtype, device=r.device)
        _require(out, self.cdtype, self.N, "out")
        check(fl_adjoint(self._handle, _ptr(r) if self.M else None, _ptr(out),
                         _stream_handle(stream)), "fl_adjoint")
        return out

    def transposed(self, g, out=None, stream=None):
        """out_k = sum_j g_j z_j^{xi_k} (C^T g), in the order of xi."""
        torch = _torch()
        _require(g, self.cdtype, self.M, "g")
        if out is None:
            out = torch.empty(self.N, dtype=self.cdtype, device=g.device)
        _require(out, self.cdtype, self.N, "out")
        check(fl_transposed(self._handle, _ptr(g) if self.M else None, _ptr(out),
                            _stream_handle(stream)), "fl_transposed")
        return out

    def info(self) -> dict:
        st, inf = fl_get_info(self._handle)
        check(st, "fl_get_info")
        return info_dict(inf)

    def set_timing(self, enable: bool):
        check(fl_set_timing(self._handle, enable), "fl_set_timing")

    def timing(self) -> dict:
        st, t = fl_get_timing(self._handle)
        check(st, "fl_get_timing")
        return timing_dict(t)

    def close(self):
        if self._handle is not None:
            fl_destroy(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LaplacePlan:
    """Owner of an Algorithm-1 plan: f_j = sum_k c_k kappa(s_j, t_k) (real data).

    kernel: "laplace" (exp(-s t) by Algorithm 1, the default), or a kernel of
    the generalised Algorithm 1: "exp" (exp(-s t)) or "bessel_half"
    (K_{1/2}(s t) = sqrt(pi / (2 s t)) exp(-s t), s, t > 0).
    """

    def __init__(self, t, s, eps: float, precision: str = "fp64", q: int = 0, stream=None,
                 kernel: str = "laplace"):
        torch = _torch()
        t = t.to(torch.float64).contiguous()
        s = s.to(torch.float64).contiguous()
        self.N, self.M = int(t.numel()), int(s.numel())
        self.prec = _precision(precision)
        self.rdtype = torch.float32 if self.prec == FL_FP32 else torch.float64
        self._handle = None
        if kernel == "laplace":
            st, h = fl_plan_laplace(self.N, self.M, _ptr(t), _ptr(s), q, eps, self.prec,
                                    _stream_handle(stream))
        else:
            st, h = fl_plan_kernel(KERNELS[kernel], self.N, self.M, _ptr(t), _ptr(s), q, eps,
                                   self.prec, _stream_handle(stream))
        check(st, "fl_plan_laplace" if kernel == "laplace" else "fl_plan_kernel")
        self._handle = h

    @property
    def handle(self):
        return self._handle

    def execute(self, c, out=None, stream=None):
        torch = _torch()
        _require(c, self.rdtype, self.N, "c")
        if out is None:
            out = torch.empty(self.M, dtype=self.rdtype, device=c.device)
        _require(out, self.rdtype, self.M, "out")
        check(fl_laplace_real(self._handle, _ptr(c), _ptr(out), _stream_handle(stream)),
              "fl_laplace_real")
        return out

    def info(self) -> dict:
        st, inf = fl_get_info(self._handle)
        check(st, "fl_get_info")
        return info_dict(inf)

    def set_timing(self, enable: bool):
        check(fl_set_timing(self._handle, enable), "fl_set_timing")

    def timing(self) -> dict:
        st, t = fl_get_timing(self._handle)
        check(st, "fl_get_timing")
        return timing_dict(t)

    def close(self):
        if self._handle is not None and self._handle.value:
            fl_destroy(self._handle)
        self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
