"""GB300-native solvers for the 2D Laplace equation (5-point stencil) compared in
"A Comparison of SOR, ADI and Multigrid Methods for Solving Partial Differential
Equations" (arXiv 2208.02427): Jacobi, red-black Gauss-Seidel / SOR, ADI line
relaxation and the multigrid V-cycle, as hand-written sm_103a CUDA kernels behind the
C ABI of include/laplace.h.

``paper_2208_02427_gb300.workloads`` (seeded inputs) imports numpy only; the CUDA
binding (``binding``: Laplace, field, smooth, ...) is loaded on first use.
"""
from __future__ import annotations

__all__ = ["Laplace", "LapError", "field", "to_field", "smooth", "jacobi_sweep", "restrict",
           "prolong_add", "kernel_launches", "load", "library_path", "workloads"]


def __getattr__(name):
    import importlib
    if name == "workloads":
        return importlib.import_module(__name__ + ".workloads")
    if name in __all__:
        return getattr(importlib.import_module(__name__ + ".binding"), name)
    raise AttributeError(name)
