"""GB300 (sm_103a) CRS sparse matrix-vector multiply after Schubert, Fehske, Hager
and Wellein (2011): plain and local/nonlocal split spMVM, block vectors, a
reverse pass, FP32-storage iterative-refinement CG and a batched persistent
launch, behind the C ABI of ``include/spmv.h``.

``workloads`` (input generators) and ``model`` (code-balance model) import
without the CUDA library; the torch wrappers in ``torch_api`` load ``libspmv.so``.
"""
__all__ = ["Matrix", "Split", "Batch", "SpMVFunction", "spmv", "ir_cg", "cg"]


def __getattr__(name):
    if name in __all__:
        from . import torch_api as _api
        return getattr(_api, name)
    raise AttributeError(name)
