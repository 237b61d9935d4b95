"""CPU oracle (plain FP64) for the subdomain-wise ILU0 BiCGSTAB hot path.

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only users.  The CUDA library never
imports, links or calls anything here, and the two share no code; both take
their inputs from :mod:`synth`.

The arithmetic lives in ``oracle.c`` (plain loops, one function per step of
the paper, each citing its passage).  This module compiles it with the system
C compiler on first use and wraps it with numpy arrays.

Paper map:
  partition            Algorithm 2 (geometric cuts)
  permutation/reorder  Section 3.1, Algorithm 3
  drop                 Section 3.2
  ilu0                 Algorithm 7 (ILU0 part), block form
  ildu0                Algorithm 7 with the ILDU0 post-processing (Section 4.3)
  levels_lower/upper   Algorithm 5 (level sets of the subdomain DAGs)
  apply                Section 4.2.2 / 4.4 result: z = U^-1 L^-1 r (ILU0 form)
  apply_ildu0          the same z in the ILDU0 form: z = U~^-1 D^-1 L^-1 r
  spmv, dot            the products inside Algorithm 1
  bicgstab             Algorithm 1 (right-preconditioned reading)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_lock = threading.Lock()
_libs = {}
_threads = 1

OK, ZERO_PIVOT, BREAKDOWN, NOT_CONVERGED = 0, 2, 5, 6
DOT_TILE = 256


def _compile(lib: str, extra: list, force: bool) -> str:
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", *extra,
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, lib)
    return lib


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` (one thread) and ``liboracle_omp.so`` (the same
    source with OpenMP on its independent loops): O2, no fast-math, no FMA
    contraction."""
    _compile(_LIB_OMP, ["-fopenmp"], force)
    return _compile(_LIB, [], force)


def set_threads(k: int) -> None:
    """Run the oracle on k host threads (k = 1: the plain single-thread build;
    k > 1: the OpenMP build, which gives the same bits)."""
    global _threads
    _threads = max(1, int(k))
    if _threads > 1:
        _load().oracle_set_threads(_threads)


def threads() -> int:
    return _threads


class _Precond(ctypes.Structure):
    _fields_ = [("form", ctypes.c_int32), ("nparts", ctypes.c_int32), ("part_ptr", ctypes.c_void_p),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("lu", ctypes.c_void_p),
                ("f", ctypes.c_void_p), ("inv_d", ctypes.c_void_p)]


class _Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("restarts", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("rel_res_recurrence", ctypes.c_double), ("rel_res_true", ctypes.c_double)]


def _load():
    omp = _threads > 1
    with _lock:
        if omp not in _libs:
            build()
            lib = ctypes.CDLL(_LIB_OMP if omp else _LIB)
            i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
            f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
            vp = ctypes.c_void_p
            I, L, D = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
            lib.oracle_partition.argtypes = [ctypes.c_int] * 6 + [i32p]
            lib.oracle_partition.restype = None
            lib.oracle_partition_bfs.argtypes = [I, i32p, i32p, I, i32p]
            lib.oracle_partition_bfs.restype = I
            lib.oracle_permutation.argtypes = [I, I, i32p, i32p, i32p, i32p]
            lib.oracle_permutation.restype = None
            lib.oracle_reorder.argtypes = [I, ctypes.c_int, i32p, i32p, vp, i32p, i32p, i32p, i32p, vp]
            lib.oracle_reorder.restype = None
            lib.oracle_drop.argtypes = [I, ctypes.c_int, i32p, i32p, vp, i32p, vp, vp, vp]
            lib.oracle_drop.restype = L
            lib.oracle_ilu0.argtypes = [I, ctypes.c_int, i32p, i32p, f64p, f64p]
            lib.oracle_ilu0.restype = ctypes.c_int
            lib.oracle_levels_lower.argtypes = [I, i32p, i32p, i32p]
            lib.oracle_levels_lower.restype = I
            lib.oracle_levels_upper.argtypes = [I, i32p, i32p, i32p]
            lib.oracle_levels_upper.restype = I
            lib.oracle_apply.argtypes = [I, ctypes.c_int, i32p, i32p, f64p, f64p, f64p]
            lib.oracle_apply.restype = ctypes.c_int
            lib.oracle_spmv.argtypes = [I, ctypes.c_int, i32p, i32p, f64p, f64p, f64p]
            lib.oracle_spmv.restype = None
            lib.oracle_dot.argtypes = [I, ctypes.c_int, f64p, f64p]
            lib.oracle_dot.restype = D
            lib.oracle_bicgstab.argtypes = [I, ctypes.c_int, i32p, i32p, f64p, i32p, i32p, f64p, f64p, f64p, I, D,
                                            ctypes.POINTER(_Info), vp]
            lib.oracle_bicgstab.restype = ctypes.c_int
            lib.oracle_inverse_gj.argtypes = [ctypes.c_int, f64p, f64p]
            lib.oracle_inverse_gj.restype = ctypes.c_int
            lib.oracle_ildu0.argtypes = [I, ctypes.c_int, i32p, i32p, f64p, I, i32p, f64p, f64p]
            lib.oracle_ildu0.restype = ctypes.c_int
            lib.oracle_apply_ildu0.argtypes = [I, ctypes.c_int, i32p, i32p, f64p, f64p, I, i32p, f64p, f64p]
            lib.oracle_apply_ildu0.restype = None
            lib.oracle_bicgstab_general.argtypes = [I, ctypes.c_int, i32p, i32p, f64p, ctypes.POINTER(_Precond),
                                                    f64p, vp, f64p, I, D, ctypes.POINTER(_Info), vp]
            lib.oracle_bicgstab_general.restype = ctypes.c_int
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            lib.oracle_set_threads.restype = None
            lib.oracle_threads.argtypes = []
            lib.oracle_threads.restype = ctypes.c_int
            _libs[omp] = lib
    return _libs[omp]


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64).reshape(-1)


@dataclass
class BSR:
    """Block sparse rows; ``val`` has shape (nnzb, bs, bs) or is None (pattern
    only). bs = 3 for the BSR inputs, 1 for scalar CSR."""

    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray | None
    block: int = 3  # bs when val is None

    @property
    def bs(self) -> int:
        if self.val is not None:
            if self.val.ndim == 3:
                return int(self.val.shape[1])
            nnzb = int(self.row_ptr[-1])  # flat values: bs*bs per block
            if nnzb > 0:
                b = int(round((self.val.size / nnzb) ** 0.5))
                if b * b * nnzb == self.val.size:
                    return b
        return self.block

    @property
    def n(self) -> int:
        return len(self.row_ptr) - 1

    @property
    def nnzb(self) -> int:
        return int(self.row_ptr[-1])


def partition(grid, sub) -> np.ndarray:
    """Algorithm 2 (ceil-division for ragged grids)."""
    nx, ny, nz = grid
    part = np.empty(nx * ny * nz, np.int32)
    _load().oracle_partition(nx, ny, nz, *sub, part)
    return part


def nparts(grid, sub) -> int:
    return int(np.prod([-(-g // s) for g, s in zip(grid, sub)]))


def partition_bfs(row_ptr, col, part_rows: int):
    """Graph partition into parts of part_rows rows cut from a breadth-first order
    (the stand-in for Section 3.1's METIS partition). Returns (part_id, nparts)."""
    rp = np.ascontiguousarray(row_ptr, np.int32)
    cl = np.ascontiguousarray(col, np.int32)
    n = len(rp) - 1
    part = np.empty(max(n, 1), np.int32)
    k = int(_load().oracle_partition_bfs(n, rp, cl, part_rows, part))
    return part[:n], k


def permutation(part_id: np.ndarray, nparts_: int):
    """Section 3.1: returns perm (new -> old), iperm (old -> new), part_ptr."""
    n = len(part_id)
    perm = np.empty(n, np.int32)
    iperm = np.empty(n, np.int32)
    pp = np.empty(nparts_ + 1, np.int32)
    _load().oracle_permutation(n, nparts_, np.ascontiguousarray(part_id, np.int32), perm, iperm, pp)
    return perm, iperm, pp


def reorder(A: BSR, perm, iperm) -> BSR:
    """Algorithm 3 on BSR."""
    n, bs = A.n, A.bs
    rp = np.empty(n + 1, np.int32)
    col = np.empty(A.nnzb, np.int32)
    val = None if A.val is None else np.empty((A.nnzb, bs, bs), np.float64)
    src = None if A.val is None else np.ascontiguousarray(A.val, np.float64)
    _load().oracle_reorder(n, bs, A.row_ptr, A.col, _ptr(src), perm, iperm, rp, col, _ptr(val))
    return BSR(rp, col, val, bs)


def drop(A: BSR, label: np.ndarray) -> BSR:
    """Section 3.2: keep blocks whose row and column carry the same label."""
    lib = _load()
    bs = A.bs
    label = np.ascontiguousarray(label, np.int32)
    kept = lib.oracle_drop(A.n, bs, A.row_ptr, A.col, None, label, None, None, None)
    rp = np.empty(A.n + 1, np.int32)
    col = np.empty(kept, np.int32)
    val = None if A.val is None else np.empty((kept, bs, bs), np.float64)
    src = None if A.val is None else np.ascontiguousarray(A.val, np.float64)
    lib.oracle_drop(A.n, bs, A.row_ptr, A.col, _ptr(src), label, _ptr(rp), _ptr(col), _ptr(val))
    return BSR(rp, col, val, bs)


def ilu0(Add: BSR):
    """Algorithm 7 (block ILU0).  Returns (lu values, status)."""
    bs = Add.bs
    lu = np.empty((Add.nnzb, bs, bs), np.float64)
    st = _load().oracle_ilu0(Add.n, bs, Add.row_ptr, Add.col, _f64(Add.val), lu.reshape(-1))
    return lu, int(st)


@dataclass
class ILDU:
    """ILDU0 factors (Algorithm 7 with Section 4.3's post-processing): ``F`` holds
    L at strictly-lower and U~ = D^-1 U at strictly-upper positions of the dropped
    pattern (zero on the diagonal), ``inv_d`` the (n, bs, bs) inverses of U's
    diagonal blocks, ``part_ptr`` the subdomain row ranges."""

    F: BSR
    inv_d: np.ndarray
    part_ptr: np.ndarray


def inverse(M: np.ndarray) -> np.ndarray | None:
    """bs x bs inverse by Gauss-Jordan with partial pivoting (None if singular)."""
    M = np.ascontiguousarray(M, np.float64)
    X = np.empty_like(M)
    return None if _load().oracle_inverse_gj(M.shape[0], M.reshape(-1), X.reshape(-1)) else X


def ildu0(Add: BSR, part_ptr: np.ndarray):
    """Algorithm 7 followed by the ILDU0 post-processing.  Returns (ILDU, status)."""
    bs = Add.bs
    pp = np.ascontiguousarray(part_ptr, np.int32)
    f = np.empty((Add.nnzb, bs, bs), np.float64)
    inv_d = np.empty((Add.n, bs, bs), np.float64)
    st = _load().oracle_ildu0(Add.n, bs, Add.row_ptr, Add.col, _f64(Add.val), len(pp) - 1, pp,
                              f.reshape(-1), inv_d.reshape(-1))
    return ILDU(BSR(Add.row_ptr, Add.col, f, bs), inv_d, pp), int(st)


def apply_ildu0(M: ILDU, r: np.ndarray) -> np.ndarray:
    """z = U~^-1 D^-1 L^-1 r (sequential substitution per subdomain, ILDU0 form)."""
    F = M.F
    bs = F.bs
    z = np.empty(bs * F.n, np.float64)
    _load().oracle_apply_ildu0(F.n, bs, F.row_ptr, F.col, _f64(F.val), _f64(M.inv_d), len(M.part_ptr) - 1,
                               M.part_ptr, _f64(r), z)
    return z


def levels_lower(M: BSR):
    lev = np.empty(M.n, np.int32)
    nl = _load().oracle_levels_lower(M.n, M.row_ptr, M.col, lev)
    return lev, int(nl)


def levels_upper(M: BSR):
    lev = np.empty(M.n, np.int32)
    nl = _load().oracle_levels_upper(M.n, M.row_ptr, M.col, lev)
    return lev, int(nl)


def apply(LU: BSR, r: np.ndarray) -> np.ndarray:
    """z = U^-1 L^-1 r (sequential substitution, ILU0 form)."""
    bs = LU.bs
    z = np.empty(bs * LU.n, np.float64)
    st = _load().oracle_apply(LU.n, bs, LU.row_ptr, LU.col, _f64(LU.val), _f64(r), z)
    if st:
        raise ArithmeticError(f"singular pivot block at row {-st - 1}")
    return z


def spmv(A: BSR, x: np.ndarray) -> np.ndarray:
    bs = A.bs
    y = np.empty(bs * A.n, np.float64)
    _load().oracle_spmv(A.n, bs, A.row_ptr, A.col, _f64(A.val), _f64(x), y)
    return y


def dot(x: np.ndarray, y: np.ndarray, bs: int = 3) -> float:
    """Dot product in the project's fixed order (block rows of bs entries,
    256-row tiles, halving sums)."""
    x = _f64(x)
    y = _f64(y)
    assert len(x) == len(y) and len(x) % bs == 0
    return float(_load().oracle_dot(len(x) // bs, bs, x, y))


@dataclass
class SolveResult:
    x: np.ndarray
    status: int
    iterations: int
    restarts: int
    rel_res_recurrence: float
    rel_res_true: float
    history: np.ndarray


def bicgstab(A: BSR, M, b: np.ndarray, maxit: int = 10000, rtol: float = 1e-8, x0=None) -> SolveResult:
    """Algorithm 1 with M = LU; vectors in the reordered numbering.  M is the
    ILU0-form factor matrix (a BSR from ``ilu0``) or an ``ILDU`` (ILDU0 form);
    x0 is the initial guess (None: zero)."""
    bs = A.bs
    x = np.empty(bs * A.n, np.float64)
    hist = np.zeros(maxit + 1, np.float64)
    info = _Info()
    keep = []
    if isinstance(M, ILDU):
        F = M.F
        fv, dv, pp = _f64(F.val), _f64(M.inv_d), np.ascontiguousarray(M.part_ptr, np.int32)
        keep += [fv, dv, pp]
        pc = _Precond(1, len(pp) - 1, _ptr(pp), _ptr(F.row_ptr), _ptr(F.col), None, _ptr(fv), _ptr(dv))
    else:
        lv = _f64(M.val)
        keep.append(lv)
        pc = _Precond(0, 0, None, _ptr(M.row_ptr), _ptr(M.col), _ptr(lv), None, None)
    x0a = None if x0 is None else _f64(x0)
    _load().oracle_bicgstab_general(A.n, bs, A.row_ptr, A.col, _f64(A.val), ctypes.byref(pc), _f64(b),
                                    _ptr(x0a), x, maxit, rtol, ctypes.byref(info), _ptr(hist))
    it = info.iterations
    return SolveResult(x, info.status, it, info.restarts, info.rel_res_recurrence,
                       info.rel_res_true, hist[: it + 1].copy())


@dataclass
class Decomposition:
    """Everything the method derives from A before the solve (Sections 3 and 4.3)."""

    grid: tuple
    sub: tuple
    part_id: np.ndarray
    perm: np.ndarray
    iperm: np.ndarray
    part_ptr: np.ndarray
    Ap: BSR          # reordered full matrix (SpMV operand)
    Add: BSR         # reordered matrix without inter-subdomain blocks
    LU: BSR          # ILU0 factors of Add, same pattern
    status: int

    def ildu(self) -> ILDU:
        """The ILDU0 factors of Add (computed on first use); raises on a zero pivot."""
        if getattr(self, "_ildu", None) is None:
            m, st = ildu0(self.Add, self.part_ptr)
            if st:
                raise ArithmeticError(f"singular pivot block at row {-st - 1}")
            self._ildu = m
        return self._ildu


def decompose(row_ptr, col, val, grid, sub, factor: bool = True) -> Decomposition:
    """Partition (Alg. 2), reorder (Alg. 3), drop (Section 3.2), ILU0 (Alg. 7)."""
    return decompose_labeled(row_ptr, col, val, partition(grid, sub), nparts(grid, sub), factor=factor,
                             grid=grid, sub=sub)


def decompose_labeled(row_ptr, col, val, part, np_, factor: bool = True, grid=None, sub=None,
                      bs: int | None = None) -> Decomposition:
    """Reorder (Alg. 3), drop (Section 3.2) and ILU0 (Alg. 7) for given labels
    (any partition, e.g. partition_bfs for matrices without a grid). bs is
    taken from val (bs*bs entries per block) unless given (pattern only)."""
    part = np.ascontiguousarray(part, np.int32)
    perm, iperm, pp = permutation(part, np_)
    rp = np.ascontiguousarray(row_ptr, np.int32)
    if val is not None and bs is None:
        nnzb = int(rp[-1])
        bs = int(round((np.size(val) / max(nnzb, 1)) ** 0.5)) if nnzb else 3
    bs = 3 if bs is None else bs
    A = BSR(rp, np.ascontiguousarray(col, np.int32),
            None if val is None else np.ascontiguousarray(val, np.float64).reshape(-1, bs, bs), bs)
    Ap = reorder(A, perm, iperm)
    label = part[perm]
    Add = drop(Ap, label)
    LU, st = BSR(Add.row_ptr, Add.col, None, bs), 0
    if factor and Add.val is not None:
        lu, st = ilu0(Add)
        LU = BSR(Add.row_ptr, Add.col, lu, bs)
    return Decomposition(tuple(grid) if grid is not None else None, tuple(sub) if sub is not None else None, part,
                         perm, iperm, pp, Ap, Add, LU, st)
