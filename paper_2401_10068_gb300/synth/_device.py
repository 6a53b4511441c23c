"""ctypes binding of ``libvbh_synth.so`` (C ABI in ``include/vbh_synth.h``)."""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .. import _build

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.lib_path("vbh_synth")
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it first (__graft_entry__.build())")
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.vbh_synth_generate.restype = ctypes.c_int
        lib.vbh_synth_generate.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                           ctypes.c_int64, ctypes.c_uint64, dp, dp, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_void_p]
        _LIB = lib
    return _LIB


def generate(r, d, V: int, S: int, start: int, seed: int, truth: dict, p_const: float, stream=None):
    """Fill device tensors r [V] and d [V, S] (float32) on ``stream``."""
    import torch
    dp = ctypes.POINTER(ctypes.c_double)
    K = np.ascontiguousarray(truth["K_true"], dtype=np.float64)
    L = np.ascontiguousarray(truth["L_beta"], dtype=np.float64)
    if stream is None:
        stream = torch.cuda.current_stream(r.device)
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    rc = _lib().vbh_synth_generate(ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(d.data_ptr()), int(V), int(S),
                                   int(start), int(seed) & ((1 << 64) - 1),
                                   K.ctypes.data_as(dp) if K.size else None,
                                   L.ctypes.data_as(dp) if L.size else None,
                                   float(truth["rho"]), float(p_const), ctypes.c_void_p(s) if s else None)
    if rc != 0:
        raise RuntimeError(f"vbh_synth_generate failed with status {rc}")
