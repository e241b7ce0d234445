"""GB300-native reverse-mode ("adjoint") gradients for variational circuits.

Jones & Gacon, "Efficient calculation of gradients in classical simulations of
variational quantum algorithms" (arXiv:2009.02823): Algorithm 1 evaluates the full
energy gradient in O(P) gate passes.  This package is a thin Python layer over the
C ABI of libvqg.so (include/vqg.h), whose CUDA kernels for sm_103a do all the work.

Submodules are imported lazily so that ``workloads`` (seeded input descriptions)
can be used without loading the CUDA library.
"""
import importlib

__all__ = ["Circuit", "VqgError", "binding", "workloads", "autograd", "build", "batch"]


def __getattr__(name):
    if name in ("Circuit", "VqgError"):
        return getattr(importlib.import_module(".binding", __name__), name)
    if name in ("binding", "workloads", "autograd", "build", "batch"):
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
