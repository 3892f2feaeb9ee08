"""PTSBE on GB300: pre-trajectory sampling with batched execution behind the libptsbe C ABI.

``capi`` is the ctypes binding with the C names; ``runtime`` marshals circuits, Kraus sets and
PyTorch device buffers into those calls. Every computation runs in libptsbe (host C++ for
registration and pre-trajectory sampling, CUDA kernels for state preparation and sampling).
"""
from . import capi  # noqa: F401
from .build import build  # noqa: F401
