"""GB300-native fast Fourier-Laplace transform (Kunis & Melzer, arXiv 1606.03255).

Evaluates f(w_j) = sum_{k<N} c_k exp(2 pi i k w_j) at nodes with Im w_j >= 0
(a degree-N polynomial at nodes in the closed unit disk, Algorithm 2 of the
paper) and the real discrete Laplace transform sum_k c_k exp(-s_j t_k)
(Algorithm 1), on one GPU, through the C ABI declared in ``include/fl.h``.

Submodules are imported lazily so that ``workloads`` (input generators) can be
used on machines without the compiled library:

* ``fl``        -- ctypes binding with the C ABI's names (fl_plan, fl_execute, ...)
* ``autograd``  -- torch.autograd.Function with the adjoint as backward
* ``workloads`` -- seeded synthetic inputs
"""
__all__ = ["fl", "autograd", "workloads", "build"]


def __getattr__(name):
    if name in ("fl", "autograd", "workloads", "build"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
