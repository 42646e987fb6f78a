"""GB300-native on-the-fly RNG + Langevin dynamics (sm_103a CUDA library).

The compute lives in libgbrng.so (C ABI: include/gbrng.h); ``gbrng`` is its
ctypes binding and ``autograd`` wraps the adjoint as a torch.autograd.Function.
"""

__all__ = ["build", "gbrng", "autograd", "workloads"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
