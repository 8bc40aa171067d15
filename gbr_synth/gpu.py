"""GPU twin of the seeded generator (see ``synth_gpu.cu``): fills torch CUDA
tensors with exactly the draws of :mod:`gbr_synth`."""
from __future__ import annotations

import ctypes as C
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth_gpu.cu")
_LIB = os.path.join(_HERE, "_build", "libgbrsynth.so")
_lib = None

ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["nvcc", ARCH, "-O3", "-shared", "-Xcompiler", "-fPIC", "-cudart", "shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB):
            raise RuntimeError(f"{_LIB} is missing: run __graft_entry__.build() first")
        L = C.CDLL(_LIB)
        u64, i64, vp, dbl = C.c_uint64, C.c_int64, C.c_void_p, C.c_double
        L.synth_u64.argtypes = [u64, u64, i64, u64, vp, vp]
        L.synth_bounded.argtypes = [u64, u64, i64, u64, vp, vp]
        L.synth_uniform.argtypes = [u64, u64, i64, dbl, dbl, vp, vp]
        for f in (L.synth_u64, L.synth_bounded, L.synth_uniform):
            f.restype = C.c_int
        _lib = L
    return _lib


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _chk(rc):
    if rc:
        raise RuntimeError(f"synth kernel launch failed: cudaError {rc}")


def u64(seed: int, n: int, offset: int = 0, mask: int = (1 << 64) - 1, device="cuda"):
    import torch
    out = torch.empty(n, dtype=torch.int64, device=device)
    _chk(lib().synth_u64(seed, offset, n, mask, C.c_void_p(out.data_ptr()), _stream()))
    return out


def bounded(seed: int, n: int, bound: int, offset: int = 0, device="cuda"):
    import torch
    out = torch.empty(n, dtype=torch.int64, device=device)
    _chk(lib().synth_bounded(seed, offset, n, bound, C.c_void_p(out.data_ptr()), _stream()))
    return out


def uniform(seed: int, n: int, lo: float = -1.0, hi: float = 1.0, offset: int = 0, device="cuda"):
    import torch
    out = torch.empty(n, dtype=torch.float64, device=device)
    _chk(lib().synth_uniform(seed, offset, n, lo, hi, C.c_void_p(out.data_ptr()), _stream()))
    return out
