"""Binding of the device half of the input generator (csrc/philox_fill.cu)."""

import ctypes
import os

_LIB = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libcosma_inputs.so")
_lib = None
KIND = {"uniform": 0, "integer": 1, "loguniform": 2}
DTYPE = {"f64": 0, "f32": 1, "bf16": 2}


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB):
            raise RuntimeError(f"input generator library not built: {_LIB}")
        lib = ctypes.CDLL(_LIB)
        lib.cosma_inputs_fill.restype = ctypes.c_int
        lib.cosma_inputs_fill.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p]
        _lib = lib
    return _lib


def fill(t, kind="uniform", dtype="f64", seed=0, stream_id=0, cuda_stream=None):
    """Fill the 2-D row-major CUDA tensor t in place (see the package docstring)."""
    import torch
    rows, cols = t.shape
    ld = max(t.stride(0), 1)
    s = (cuda_stream or torch.cuda.current_stream()).cuda_stream
    rc = _load().cosma_inputs_fill(t.data_ptr(), rows, cols, ld, KIND[kind], DTYPE[dtype],
                                   seed, stream_id, s)
    if rc != 0:
        raise RuntimeError(f"cosma_inputs_fill failed: cudaError {rc}")
    return t


def new(rows, cols, kind="uniform", dtype="f64", seed=0, stream_id=0, device="cuda"):
    import torch
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dtype]
    t = torch.empty((rows, cols), dtype=tdt, device=device)
    return fill(t, kind, dtype, seed, stream_id)
