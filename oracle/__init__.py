"""CPU oracle for the fast Fourier-Laplace transform (Kunis & Melzer).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the library in
``paper_1606_03255_gb300`` never does, and this package never imports it.

Two layers:

* ``fl_oracle.c`` (loaded through ctypes): the plain definitions, term by term,
  in FP64 with compensated summation -- the forward sum of eq. (4.1) with
  xi_k = k, its adjoint, the real Laplace sum of eq. (3.2), and a long-double
  brute force for tiny N.
* ``structured.py``: the matrices Algorithms 1 and 2 of the paper apply,
  assembled block by block from Definition 3.2 and eq. (A.1) in numpy (the
  Hadamard product A o K~ of Lemma 4.1 for Algorithm 2, with the Fourier
  matrix A formed exactly in place of the NFFT), for tiny N.  It isolates the
  error of the hierarchical Laplace factorisation from that of the NFFT.

Index convention: the paper sums k = 1..N; this library sums k = 0..N-1, so
xi_k = k and xi_1 (the largest frequency) is N - 1.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fl_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``fl_oracle.c`` into ``_build/liboracle.so`` (gcc, no -ffast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    flags = ["-O2", "-ffp-contract=off", "-fPIC", "-shared", "-Wall"]
    if platform.machine() in ("x86_64", "AMD64"):
        # fma() is correctly rounded either way; this only avoids a libm call.
        try:
            with open("/proc/cpuinfo") as fh:
                if " fma " in fh.read():
                    flags.append("-mfma")
        except OSError:
            pass
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.run(["gcc", *flags, "-o", tmp, _SRC, "-lm", "-lpthread"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, dp, ci = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int
            lib.oracle_flt_direct.argtypes = [i64, dp, i64, dp, dp, ci]
            lib.oracle_flt_adjoint.argtypes = [i64, dp, i64, dp, dp, ci]
            lib.oracle_flt_adjoint_at.argtypes = [i64, dp, dp, i64, dp, dp, ci]
            lib.oracle_laplace_direct.argtypes = [i64, dp, dp, i64, dp, dp, ci]
            lib.oracle_kernel_direct.argtypes = [ci, i64, dp, dp, i64, dp, dp, ci]
            lib.oracle_xi_direct.argtypes = [i64, dp, dp, i64, dp, dp, ci]
            lib.oracle_xi_transposed.argtypes = [i64, dp, i64, dp, dp, dp, ci]
            lib.oracle_flt_brute_ld.argtypes = [i64, dp, i64, dp, dp]
            for fn in (lib.oracle_flt_direct, lib.oracle_flt_adjoint, lib.oracle_flt_adjoint_at,
                       lib.oracle_laplace_direct, lib.oracle_kernel_direct, lib.oracle_xi_direct,
                       lib.oracle_xi_transposed, lib.oracle_flt_brute_ld):
                fn.restype = ci
            lib.oracle_default_threads.restype = ci
            _lib = lib
    return _lib


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def _nodes(w) -> np.ndarray:
    """Nodes as an (M, 2) float64 array of (Re w, Im w)."""
    w = np.asarray(w)
    if np.iscomplexobj(w):
        w = np.stack([w.real, w.imag], axis=-1)
    return np.ascontiguousarray(w, dtype=np.float64).reshape(-1, 2)


def default_threads() -> int:
    return int(_load().oracle_default_threads())


def flt_direct(c, w, threads: int = 0) -> np.ndarray:
    """f_j = sum_{k<N} c_k exp(2 pi i k w_j) (eq. 4.1, xi_k = k), FP64, term by term."""
    c, w = _c128(c), _nodes(w)
    f = np.empty(w.shape[0], dtype=np.complex128)
    rc = _load().oracle_flt_direct(c.size, c.ctypes.data, w.shape[0], w.ctypes.data,
                                   f.ctypes.data, threads)
    if rc != 0:
        raise ValueError("oracle_flt_direct: invalid arguments (Im w < 0 or non-finite?)")
    return f


def flt_adjoint(r, w, N: int, threads: int = 0) -> np.ndarray:
    """g_k = sum_j conj(z_j)^k r_j for k < N: the adjoint C^* of eq. (4.1)'s matrix."""
    r, w = _c128(r), _nodes(w)
    g = np.empty(int(N), dtype=np.complex128)
    rc = _load().oracle_flt_adjoint(int(N), r.ctypes.data, w.shape[0], w.ctypes.data,
                                    g.ctypes.data, threads)
    if rc != 0:
        raise ValueError("oracle_flt_adjoint: invalid arguments")
    return g


def flt_adjoint_at(r, w, ks, threads: int = 0) -> np.ndarray:
    """g_i = sum_j conj(z_j)^{ks[i]} r_j: the adjoint C^* r at selected frequencies."""
    r, w = _c128(r), _nodes(w)
    ks = np.ascontiguousarray(ks, dtype=np.int64)
    g = np.empty(ks.size, dtype=np.complex128)
    rc = _load().oracle_flt_adjoint_at(ks.size, ks.ctypes.data, r.ctypes.data, w.shape[0],
                                       w.ctypes.data, g.ctypes.data, threads)
    if rc != 0:
        raise ValueError("oracle_flt_adjoint_at: invalid arguments")
    return g


def laplace_direct(c, t, s, threads: int = 0) -> np.ndarray:
    """f_j = sum_k c_k exp(-s_j t_k) (eq. 3.2), FP64, term by term."""
    c = np.ascontiguousarray(c, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.float64)
    f = np.empty(s.size, dtype=np.float64)
    rc = _load().oracle_laplace_direct(c.size, c.ctypes.data, t.ctypes.data, s.size,
                                       s.ctypes.data, f.ctypes.data, threads)
    if rc != 0:
        raise ValueError("oracle_laplace_direct: invalid arguments")
    return f


def xi_direct(c, xi, w, threads: int = 0) -> np.ndarray:
    """f_j = sum_k c_k exp(2 pi i xi_k w_j) for real exponents xi_k >= 0 (eq. 4.1
    with general xi_k), FP64 term by term."""
    c, w = _c128(c), _nodes(w)
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    f = np.empty(w.shape[0], dtype=np.complex128)
    rc = _load().oracle_xi_direct(c.size, c.ctypes.data, xi.ctypes.data, w.shape[0], w.ctypes.data,
                                  f.ctypes.data, threads)
    if rc != 0:
        raise ValueError("oracle_xi_direct: invalid arguments")
    return f


def xi_transposed(h, xi, w, threads: int = 0) -> np.ndarray:
    """g_k = sum_j h_j exp(2 pi i xi_k w_j): the transposed evaluation at real
    exponents (remark after Algorithm 2), FP64 term by term."""
    h, w = _c128(h), _nodes(w)
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    if h.size != w.shape[0]:
        raise ValueError("xi_transposed: one value per node")
    g = np.empty(xi.size, dtype=np.complex128)
    rc = _load().oracle_xi_transposed(xi.size, xi.ctypes.data, w.shape[0], w.ctypes.data,
                                      h.ctypes.data, g.ctypes.data, threads)
    if rc != 0:
        raise ValueError("oracle_xi_transposed: invalid arguments")
    return g


KERNELS = {"exp": 1, "bessel_half": 2}


def kernel_direct(kind: str, c, t, s, threads: int = 0) -> np.ndarray:
    """f_j = sum_k c_k kappa(s_j, t_k), FP64 term by term, for the kernels of the
    generalised Algorithm 1: "exp" exp(-s t), "bessel_half" K_{1/2}(s t) =
    sqrt(pi/(2 s t)) exp(-s t) (s, t > 0)."""
    c = np.ascontiguousarray(c, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.float64)
    f = np.empty(s.size, dtype=np.float64)
    rc = _load().oracle_kernel_direct(KERNELS[kind], c.size, c.ctypes.data, t.ctypes.data, s.size,
                                      s.ctypes.data, f.ctypes.data, threads)
    if rc != 0:
        raise ValueError("oracle_kernel_direct: invalid arguments")
    return f


def flt_brute_ld(c, w) -> np.ndarray:
    """Same sum as ``flt_direct`` in long double (tiny N only, N <= 65536)."""
    c, w = _c128(c), _nodes(w)
    f = np.empty(w.shape[0], dtype=np.complex128)
    rc = _load().oracle_flt_brute_ld(c.size, c.ctypes.data, w.shape[0], w.ctypes.data,
                                     f.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_flt_brute_ld: invalid arguments")
    return f


def error_E(f_exact, f_approx, c) -> float:
    """E = ||f - f~||_inf / ||c||_1, the paper's error measure (eq. 5.1)."""
    f_exact = np.asarray(f_exact)
    f_approx = np.asarray(f_approx)
    denom = np.sum(np.abs(np.asarray(c, dtype=np.complex128)))
    if f_exact.size == 0:
        return 0.0
    return float(np.max(np.abs(f_exact - f_approx)) / denom)
