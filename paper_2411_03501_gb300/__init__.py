"""GB300-native explicit Hamilton-Jacobi level-set integrator (LevelSetPy,
arXiv 2411.03501): fused sm_103a CUDA stage kernels behind a C ABI
(``include/lsp.h``), with a thin ctypes binding.

The CUDA library is loaded on first use; if it has not been built the call
fails with an error (there is no CPU fallback).
"""
from . import workloads  # noqa: F401  (seeded inputs; no method arithmetic)

__all__ = ["workloads"]


def __getattr__(name):
    # Load the binding lazily so that importing the package (e.g. for the
    # input generators) does not require the compiled library.
    if name in ("lsp", "binding"):
        from . import binding
        return binding
    raise AttributeError(name)
