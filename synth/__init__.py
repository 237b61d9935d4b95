"""Seeded synthetic 3x3-block 7-point-stencil systems (the common input source).

The paper evaluates on 3x3 BSR discretisations of 3D Laplacians (Table 2,
"Laplacian1/2") and on reservoir matrices with strongly layered permeability
(spe10, Section 5).  Neither the Laplacian values nor the reservoir data are
published, so the workloads here are seeded stand-ins with the same shape:

* ``laplace``: off-diagonal blocks -I + U(-0.1, 0.1), diagonal blocks
  6.5 I + U(-0.1, 0.1) (nonsymmetric, block diagonally dominant in mean).
* ``layered``: log-normal cell coefficient exp(2 g), g ~ N(0, 1), constant
  through 8-cell-thick z-layers of each column; faces couple with the harmonic
  mean times (I + 3x3 U(-0.1, 0.1)); diagonal = sum of couplings + 0.01 I.

This module computes nothing of the method itself; both the CPU oracle and the
CUDA library consume the arrays it returns.  The C source (``synth.c``) is
compiled on first use with the system C compiler.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

MODEL_LAPLACE = 0
MODEL_LAYERED = 1


def build(force: bool = False) -> str:
    """Compile ``libsynth.so`` next to its source (no fast-math, no contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
            f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
            lib.synth_bits.restype = ctypes.c_uint64
            lib.synth_bits.argtypes = [ctypes.c_uint64] * 3
            lib.synth_unit.restype = ctypes.c_double
            lib.synth_unit.argtypes = [ctypes.c_uint64] * 3
            lib.synth_nnzb.restype = ctypes.c_int64
            lib.synth_nnzb.argtypes = [ctypes.c_int] * 3
            lib.synth_pattern.restype = None
            lib.synth_pattern.argtypes = [ctypes.c_int] * 3 + [i32p, i32p]
            lib.synth_system.restype = ctypes.c_int64
            lib.synth_system.argtypes = ([ctypes.c_int] * 4 + [ctypes.c_uint64, i32p, i32p, f64p,
                                                                f64p, f64p])
            lib.synth_system_bs.restype = ctypes.c_int64
            lib.synth_system_bs.argtypes = ([ctypes.c_int] * 5 + [ctypes.c_uint64, i32p, i32p, f64p, f64p, f64p])
            lib.synth_unstructured_nnzb.restype = ctypes.c_int64
            lib.synth_unstructured_nnzb.argtypes = [ctypes.c_int] * 3 + [ctypes.c_uint64]
            lib.synth_unstructured.restype = ctypes.c_int64
            lib.synth_unstructured.argtypes = ([ctypes.c_int] * 3 + [ctypes.c_uint64, i32p, i32p, f64p, f64p, f64p,
                                                                    i32p])
            lib.synth_sides.restype = None
            lib.synth_sides.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, i32p]
            _lib = lib
    return _lib


@dataclass
class System:
    """A BSR system in natural cell order.  ``val`` has shape (nnzb, 3, 3)."""

    nx: int
    ny: int
    nz: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    xstar: np.ndarray
    b: np.ndarray

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def nnzb(self) -> int:
        return int(self.row_ptr[-1])


def nnzb(nx: int, ny: int, nz: int) -> int:
    return int(_load().synth_nnzb(nx, ny, nz))


def pattern(nx: int, ny: int, nz: int):
    """Row pointers and column indices of the 7-point block pattern (no values)."""
    lib = _load()
    n = nx * ny * nz
    rp = np.empty(n + 1, np.int32)
    col = np.empty(lib.synth_nnzb(nx, ny, nz), np.int32)
    lib.synth_pattern(nx, ny, nz, rp, col)
    return rp, col


def system(nx: int, ny: int, nz: int, seed: int, model: int = MODEL_LAPLACE, bs: int = 3) -> System:
    """The 7-point system with bs x bs blocks: bs = 3 (3 unknowns per cell) or
    bs = 1 (the scalar CSR form, each value the 3x3 model's (0,0) entry)."""
    lib = _load()
    n = nx * ny * nz
    m = lib.synth_nnzb(nx, ny, nz)
    rp = np.empty(n + 1, np.int32)
    col = np.empty(m, np.int32)
    val = np.empty(m * bs * bs, np.float64)
    xs = np.empty(bs * n, np.float64)
    b = np.empty(bs * n, np.float64)
    lib.synth_system_bs(model, bs, nx, ny, nz, seed, rp, col, val, xs, b)
    return System(nx, ny, nz, rp, col, val.reshape(m, bs, bs), xs, b)


def unstructured(nx: int, ny: int, nz: int, seed: int) -> System:
    """The unstructured system (irregular 27-point pattern, cells renumbered at
    random): a stand-in for graph-partitioned matrices. ``nx, ny, nz`` only size
    the underlying cell grid; the row order carries no geometry."""
    lib = _load()
    n = nx * ny * nz
    m = lib.synth_unstructured_nnzb(nx, ny, nz, seed)
    rp = np.empty(n + 1, np.int32)
    col = np.empty(m, np.int32)
    val = np.empty(m * 9, np.float64)
    xs = np.empty(3 * n, np.float64)
    b = np.empty(3 * n, np.float64)
    scratch = np.empty(2 * n, np.int32)
    lib.synth_unstructured(nx, ny, nz, seed, rp, col, val, xs, b, scratch)
    return System(nx, ny, nz, rp, col, val.reshape(m, 3, 3), xs, b)


def unit(seed: int, stream: int, index: int) -> float:
    return float(_load().synth_unit(seed, stream, index))


def bits(seed: int, stream: int, index: int) -> int:
    return int(_load().synth_bits(seed, stream, index))


def ragged_sides(seed: int, lo: int = 24, hi: int = 96):
    s = np.empty(3, np.int32)
    _load().synth_sides(seed, lo, hi, s)
    return tuple(int(v) for v in s)


# Named workloads (grid, subdomain, model, seed).  Seeds are this project's
# choice; the paper publishes none.
WORKLOADS = {
    "laplace16_sub8x8x4": dict(grid=(16, 16, 16), sub=(8, 8, 4), model=MODEL_LAPLACE, seed=1),
    "laplace64_sub4": dict(grid=(64, 64, 64), sub=(4, 4, 4), model=MODEL_LAPLACE, seed=2),
    "laplace64_sub8": dict(grid=(64, 64, 64), sub=(8, 8, 8), model=MODEL_LAPLACE, seed=2),
    "laplace64_sub16x16x8": dict(grid=(64, 64, 64), sub=(16, 16, 8), model=MODEL_LAPLACE, seed=2),
    "layered160_sub16x16x8": dict(grid=(160, 160, 160), sub=(16, 16, 8), model=MODEL_LAYERED, seed=3),
    # smaller case of the same shape (0.48 GB apply, above L2) for profiler captures
    "layered96_sub16x16x8": dict(grid=(96, 96, 96), sub=(16, 16, 8), model=MODEL_LAYERED, seed=3),
    "laplace64_mixed_sub16x16x8": dict(grid=(64, 64, 64), sub=(16, 16, 8), model=MODEL_LAPLACE, seed=4),
}


def ragged_batch(nsys: int = 64, lo: int = 24, hi: int = 96, seed0: int = 5000):
    """Grid sides of the ragged batch: system s uses seed seed0 + s."""
    return [ragged_sides(seed0 + s, lo, hi) for s in range(nsys)]
