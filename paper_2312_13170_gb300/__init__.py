"""libloopnest: GB300-native (sm_103a) kernels for the loop nests that loop
internalization and array-reduction detection speed up (arXiv 2312.13170,
Sec. VI-B and VI-C): GEMM, a chain of two GEMMs, covariance, correlation,
SYRK and SYR2K, each in a plain and an internalized form.

The compute runs in ``libloopnest.so`` (CUDA C++ behind a C ABI declared in
``include/loopnest.h``). ``paper_2312_13170_gb300.api`` is the thin Python
binding; importing this package does not load the shared library.
"""

__all__ = ["api", "inputs"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
