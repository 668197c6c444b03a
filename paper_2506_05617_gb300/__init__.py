"""GB300 (sm_103a) library for the SVD of stride-1 periodic multi-channel 2-D
convolutions by local Fourier analysis (arXiv 2506.05617).

The computation runs in the CUDA library ``lib/liblfa.so`` (C ABI in
``include/lfa.h``); ``lfa`` is its ctypes binding and ``torch_api`` the PyTorch
wrapper (memory, streams and an autograd Function).
"""
from . import lfa  # noqa: F401

__all__ = ["lfa", "build", "torch_api"]
