"""GB300-native batched GEMM for many small matrices (arXiv 1304.7053).

``C_p = alpha * op(A_p) * op(B_p) + beta * C_p`` for p = 1..N with m, n, k <= 16,
on the uniform 3-D batch layout (second-level leading dimension) of Section 4,
computed by hand-written sm_103a CUDA kernels behind the C ABI declared in
``include/sbgemm.h``.

Importing the package is cheap; the CUDA library is loaded on first use of
the binding (``paper_1304_7053_gb300.sbgemm``), which raises if it has not
been built.  There is no CPU fallback.
"""
import importlib

__all__ = ["sbgemm", "inputs"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
