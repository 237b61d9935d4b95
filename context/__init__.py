"""Context measurements beside the path (not part of it): the vendor global
block-ILU0 baseline (cuSPARSE bsrilu02 + bsrsv2 + bsrmv) and the GPU's FP64
FMA rate. Built in-tree as ``libilu0dd_context.so``; bench.py and the GPU tests
load it through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "context.cu")
LIB = os.path.join(HERE, "libilu0dd_context.so")
CUDA_LIB = "/usr/local/cuda/lib64"

_lib = None


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC),
                                                                         os.path.getmtime(__file__)):
        return LIB
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-shared",
           "-Xcompiler", "-fPIC", "-cudart", "static", SRC, "-o", tmp, "-L", CUDA_LIB, "-lcusparse",
           "-Xlinker", "-rpath=" + CUDA_LIB]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on context.cu:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            build()
        lib = ctypes.CDLL(LIB)
        P, I, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        lib.ctx_vendor_ilu0_create.argtypes = [ctypes.c_int32, I64, P, P, P, ctypes.POINTER(P),
                                               ctypes.POINTER(ctypes.c_double)]
        lib.ctx_vendor_ilu0_apply.argtypes = [P, P, P, P]
        lib.ctx_vendor_spmv.argtypes = [P, P, P, P]
        lib.ctx_vendor_ilu0_factors.argtypes = [P, P]
        lib.ctx_vendor_ilu0_destroy.argtypes = [P]
        lib.ctx_fp64_fma_rate.argtypes = [I, ctypes.POINTER(ctypes.c_double)]
        for f in ("ctx_vendor_ilu0_create", "ctx_vendor_ilu0_apply", "ctx_vendor_spmv", "ctx_vendor_ilu0_factors",
                  "ctx_vendor_ilu0_destroy", "ctx_fp64_fma_rate"):
            getattr(lib, f).restype = I
        _lib = lib
    return _lib


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"{what} failed with code {rc} (1 CUDA, 2 cuSPARSE, 3 zero pivot, 4 invalid)")


def fp64_fma_gflops(iters: int = 2048) -> float:
    out = ctypes.c_double()
    _check(load().ctx_fp64_fma_rate(iters, ctypes.byref(out)), "ctx_fp64_fma_rate")
    return out.value


class VendorIlu0:
    """cuSPARSE global block ILU0 of a 3x3 BSR matrix in natural order."""

    def __init__(self, row_ptr, col, val):
        import numpy as np
        self._keep = [np.ascontiguousarray(row_ptr, np.int32), np.ascontiguousarray(col, np.int32),
                      np.ascontiguousarray(val, np.float64)]
        rp, cl, vl = self._keep
        self.mb = len(rp) - 1
        self.nnzb = len(cl)
        h = ctypes.c_void_p()
        ms = ctypes.c_double()
        _check(load().ctx_vendor_ilu0_create(self.mb, self.nnzb, rp.ctypes.data, cl.ctypes.data, vl.ctypes.data,
                                             ctypes.byref(h), ctypes.byref(ms)), "ctx_vendor_ilu0_create")
        self._h = h
        self.setup_ms = ms.value
        self._keep = None

    def apply(self, r, z, stream=None):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        _check(load().ctx_vendor_ilu0_apply(self._h, r.data_ptr(), z.data_ptr(), s), "ctx_vendor_ilu0_apply")

    def spmv(self, x, y, stream=None):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        _check(load().ctx_vendor_spmv(self._h, x.data_ptr(), y.data_ptr(), s), "ctx_vendor_spmv")

    def factors(self):
        import numpy as np
        out = np.empty(9 * self.nnzb, np.float64)
        _check(load().ctx_vendor_ilu0_factors(self._h, out.ctypes.data), "ctx_vendor_ilu0_factors")
        return out

    def close(self):
        if self._h:
            load().ctx_vendor_ilu0_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
