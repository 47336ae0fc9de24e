"""GB300-native axion Monte-Carlo operators for particle-in-cell plasmas.

The compute path is libaxpic.so (CUDA for sm_103a behind the C ABI in
include/axpic.h); ``_lib`` is its ctypes binding and ``AxionPlasma`` a front
end that keeps the particle slabs in torch CUDA tensors. There is no CPU
fallback: without the built library every operator raises.
"""
from . import _lib, workloads  # noqa: F401

__all__ = ["AxionPlasma", "_lib", "workloads"]


def __getattr__(name):
    if name == "AxionPlasma":
        from .plasma import AxionPlasma
        return AxionPlasma
    raise AttributeError(name)
