"""GB300-native compressed matrix multiplication in the Fast Walsh-Hadamard
Transform form (Pagh's sketch with XOR buckets; Andersson & Karppa,
arXiv 2601.09477).

The compute path is hand-written sm_103a CUDA behind the C-ABI library
``libcmm.so`` (declared in ``include/cmm.h``); this package is its thin Python
binding.  PyTorch is used for device memory and streams only.
"""
__all__ = ["cmm", "workloads"]


def __getattr__(name):
    if name in ("cmm", "workloads", "autotune", "autograd_fn"):
        import importlib
        return importlib.import_module(__name__ + "." + name)
    raise AttributeError(name)
