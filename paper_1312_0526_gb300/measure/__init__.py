"""Measurement helpers of the benchmark (not part of the peeling library).

``random_access`` runs the random-access ceiling probe of ``probe.cu``
(library ``_build/libhpeel_measure.so``, built beside ``libhpeel.so``): the
rate at which the memory system serves the access pattern of the peeling
rounds, against which the rounds' own rate is reported.
"""
from __future__ import annotations

import ctypes
import os
import threading

from .. import build as _build

LIB_PATH = _build.MEASURE_LIB
_lib = None
_lock = threading.Lock()


def lib():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: build it with "
                                  "`python -m paper_1312_0526_gb300.build`")
            L = ctypes.CDLL(LIB_PATH)
            L.hpeel_measure_random_access.restype = ctypes.c_int
            L.hpeel_measure_random_access.argtypes = [
                ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_size_t,
                ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64, ctypes.c_void_p]
            _lib = L
        return _lib


def random_access(kind: int, n_ops: int, a, b=None, seed: int = 1) -> None:
    """Enqueue the probe on the current stream: kind 0 random 64-bit atomicAdd
    into a, 1 random 8-byte load from a, 2 one peeled edge (record claim in a,
    two vertex updates in b).  a and b are CUDA tensors used as raw memory."""
    import torch
    for t in (a,) + ((b,) if b is not None else ()):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
            raise ValueError("probe buffers must be contiguous CUDA tensors")
    rc = lib().hpeel_measure_random_access(
        kind, n_ops, ctypes.c_void_p(a.data_ptr()), a.numel() * a.element_size(),
        ctypes.c_void_p(b.data_ptr()) if b is not None else None,
        0 if b is None else b.numel() * b.element_size(), seed,
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if rc != 0:
        raise ValueError(f"random-access probe refused its arguments (code {rc})")
