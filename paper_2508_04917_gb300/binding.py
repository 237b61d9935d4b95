"""Thin ctypes binding of ``libilu0dd.so`` (argument marshalling only).

Every step of the hot path runs in the library's CUDA kernels; PyTorch only
provides device memory (the workspace, the vectors) and the current stream.
There is no CPU fallback: if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

from . import build as _build

_HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "ilu0dd.h")

OK = 0
ERR_INVALID, ERR_ZERO_PIVOT, ERR_SMEM, ERR_CUDA = 1, 2, 3, 4
ERR_BREAKDOWN, ERR_NOT_CONVERGED, ERR_NONFINITE, ERR_WORKSPACE, ERR_DEVICE_WAIT = 5, 6, 7, 8, 9
F64, F32, BF16, DF64 = 0, 1, 2, 3
PRECISIONS = {"f64": F64, "f32": F32, "bf16": BF16, "df64": DF64}

X_PART_ID, X_PERM, X_IPERM, X_PART_PTR, X_LEVEL_L, X_LEVEL_U = 0, 1, 2, 3, 4, 5
X_DD_ROW_PTR, X_DD_COL, X_L, X_UT, X_INVD, X_AP_ROW_PTR, X_AP_COL = 6, 7, 8, 9, 10, 11, 12
X_STREAM, X_SELL_COL, X_SELL_VAL = 13, 14, 15

Q = dict(n=0, nnzb=1, kept=2, nsub=3, nl=4, nu=5, apply_bytes=6, spmv_bytes=7, stream_bytes=8,
         threads=9, smem=10, pieces=11, cuda_error=12, max_levels=13, workspace=14,
         apply_kernels=15, iter_kernels=16, sell_slots=17, block_dim=18, row_thread=19)


class Ilu0DDError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} (code {code})")


class Bsr(ctypes.Structure):
    _fields_ = [("n_brows", ctypes.c_int32), ("block_dim", ctypes.c_int32), ("nnzb", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class Geom(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in ("nx", "ny", "nz", "sx", "sy", "sz")]


class Opts(ctypes.Structure):
    _fields_ = [("factor_prec", ctypes.c_int32), ("threads_per_cta", ctypes.c_int32),
                ("prefetch_bytes", ctypes.c_int32), ("maxit", ctypes.c_int32), ("rtol", ctypes.c_double),
                ("check_every", ctypes.c_int32), ("use_graphs", ctypes.c_int32),
                ("keep_host", ctypes.c_int32), ("trace", ctypes.c_int32), ("traversal", ctypes.c_int32),
                ("apply_mapping", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32), ("restarts", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("rel_res_recurrence", ctypes.c_double),
                ("rel_res_true", ctypes.c_double), ("setup_s", ctypes.c_double), ("solve_s", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load ``libilu0dd.so`` (building it in-tree first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libilu0dd.so not found at {path}; run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        sig = {
            "ilu0dd_default_opts": ([ctypes.POINTER(Opts)], ctypes.c_int),
            "ilu0dd_strerror": ([ctypes.c_int], ctypes.c_char_p),
            "ilu0_dd_workspace_size": ([ctypes.POINTER(Bsr), ctypes.POINTER(Geom), ctypes.POINTER(Opts),
                                        ctypes.POINTER(sz)], ctypes.c_int),
            "ilu0_dd_setup": ([ctypes.POINTER(Bsr), ctypes.POINTER(Geom), ctypes.POINTER(Opts), vp, sz, vp,
                               ctypes.POINTER(vp)], ctypes.c_int),
            "ilu0dd_plan_create": ([ctypes.POINTER(Bsr), ctypes.POINTER(Geom), ctypes.POINTER(Opts),
                                    ctypes.POINTER(vp), ctypes.POINTER(sz), ctypes.POINTER(sz)], ctypes.c_int),
            "ilu0_dd_setup_planned": ([vp, ctypes.POINTER(Bsr), vp, sz, vp, sz, vp, ctypes.POINTER(vp)],
                                      ctypes.c_int),
            "ilu0dd_plan_destroy": ([vp], ctypes.c_int),
            "ilu0dd_plan_create_partitioned": ([ctypes.POINTER(Bsr), vp, i32, ctypes.POINTER(Opts),
                                                ctypes.POINTER(vp), ctypes.POINTER(sz), ctypes.POINTER(sz)],
                                               ctypes.c_int),
            "ilu0dd_partition_bfs": ([ctypes.POINTER(Bsr), i32, vp, ctypes.POINTER(i32)], ctypes.c_int),
            "ilu0_dd_apply": ([vp, vp, vp, vp], ctypes.c_int),
            "ilu0_dd_apply_unfused": ([vp, vp, vp, vp], ctypes.c_int),
            "ilu0_dd_apply_rowsync": ([vp, vp, vp, vp], ctypes.c_int),
            "ilu0_dd_apply_edge": ([vp, vp, vp, vp], ctypes.c_int),
            "ilu0_dd_apply_global_vector": ([vp, vp, vp, vp], ctypes.c_int),
            "ilu0dd_levels_device": ([vp, vp, vp, i32, vp, vp, vp, vp, vp], ctypes.c_int),
            "ilu0_dd_apply_host": ([vp, vp, vp, vp], ctypes.c_int),
            "ilu0_dd_spmv": ([vp, vp, vp, vp], ctypes.c_int),
            "ilu0_dd_dot": ([vp, vp, vp, vp, vp], ctypes.c_int),
            "ilu0_dd_permute": ([vp, vp, vp, ctypes.c_int, vp], ctypes.c_int),
            "ilu0dd_dot_noalloc": ([vp, vp, i64, vp, vp], ctypes.c_int),
            "ilu0dd_batch_workspace_size": ([ctypes.POINTER(vp), i32, ctypes.POINTER(sz)], ctypes.c_int),
            "ilu0dd_batch_create": ([ctypes.POINTER(vp), i32, ctypes.POINTER(Opts), vp, sz, vp, ctypes.POINTER(vp)],
                                    ctypes.c_int),
            "bicgstab_solve_batched": ([vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(Info), vp],
                                       ctypes.c_int),
            "ilu0dd_batch_destroy": ([vp], None),
            "bicgstab_solve": ([vp, vp, vp, ctypes.POINTER(Info), vp], ctypes.c_int),
            "bicgstab_start": ([vp, vp, vp], ctypes.c_int),
            "bicgstab_iterate": ([vp, i32, vp, vp], ctypes.c_int),
            "bicgstab_state": ([vp, ctypes.POINTER(Info), vp], ctypes.c_int),
            "ilu0_dd_history": ([vp, vp, i32], ctypes.c_int),
            "ilu0_dd_export": ([vp, ctypes.c_int, vp, sz], ctypes.c_int),
            "ilu0_dd_query": ([vp, ctypes.c_int, ctypes.POINTER(i64)], ctypes.c_int),
            "ilu0_dd_device_error": ([vp, ctypes.POINTER(i32)], ctypes.c_int),
            "ilu0dd_set_wait_limits": ([vp, ctypes.c_uint32, i32], ctypes.c_int),
            "ilu0_dd_destroy": ([vp], None),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def declared_functions() -> list[str]:
    """Names of the functions declared in include/ilu0dd.h."""
    text = open(_HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?(?:int|void|const char\s*\*)\s*\**\s*(\w+)\s*\(", text, re.M)))


def strerror(code: int) -> str:
    return load().ilu0dd_strerror(code).decode()


def default_opts(**kw) -> Opts:
    o = Opts()
    load().ilu0dd_default_opts(ctypes.byref(o))
    names = {f[0] for f in Opts._fields_}
    for k, v in kw.items():
        if k not in names:
            raise TypeError(f"unknown option {k!r}")
        if k == "factor_prec" and isinstance(v, str):
            v = PRECISIONS[v]
        setattr(o, k, v)
    return o


def _is_cuda(a) -> bool:
    return getattr(a, "is_cuda", False)


def _arr(a, np_dtype, torch_dtype, name):
    """(address, keep-alive, element count) of one matrix array: a numpy-like
    host array, or a contiguous CUDA tensor (device memory, passed by address)."""
    if _is_cuda(a):
        if a.dtype != torch_dtype or not a.is_contiguous():
            raise ValueError(f"{name}: a device array must be a contiguous CUDA tensor of {torch_dtype}")
        return a.data_ptr(), a, int(a.numel())
    h = np.ascontiguousarray(a, np_dtype).reshape(-1)
    return h.ctypes.data, h, int(h.size)


def _bsr(row_ptr, col, val):
    """ilu0dd_bsr of the matrix arrays, each in host memory (numpy) or in device
    memory (a CUDA tensor: int32 row_ptr and col, float64 val)."""
    import_torch = any(_is_cuda(a) for a in (row_ptr, col, val))
    tdt = (None, None)
    if import_torch:
        import torch
        tdt = (torch.int32, torch.float64)
    rp_p, rp_k, n1 = _arr(row_ptr, np.int32, tdt[0], "row_ptr")
    ci_p, ci_k, nnzb = _arr(col, np.int32, tdt[0], "col")
    if val is None:
        va_p, va_k, bs = None, None, 3
    else:
        if not _is_cuda(val) and np.ndim(val) == 3:
            bs = int(np.shape(val)[-1])
        elif nnzb == 0:
            bs = 3
        else:
            nv = int(val.numel()) if _is_cuda(val) else int(np.size(val))
            bs = int(round((nv / nnzb) ** 0.5))
            if bs * bs * nnzb != nv:
                raise ValueError("val must hold bs*bs values per block")
        va_p, va_k, _ = _arr(val, np.float64, tdt[1], "val")
    b = Bsr(n1 - 1, bs, nnzb, rp_p, ci_p, va_p)
    return b, (rp_k, ci_k, va_k)


def partition_bfs(row_ptr, col, part_rows: int):
    """ilu0dd_partition_bfs: (part_id, nparts), parts of part_rows rows cut from a
    breadth-first order of the pattern (for matrices without a grid)."""
    b, keep = _bsr(row_ptr, col, None)
    part = np.empty(max(b.n_brows, 1), np.int32)
    k = ctypes.c_int32(0)
    rc = load().ilu0dd_partition_bfs(ctypes.byref(b), part_rows, part.ctypes.data, ctypes.byref(k))
    del keep
    if rc:
        raise Ilu0DDError(rc, "ilu0dd_partition_bfs")
    return part[:b.n_brows], int(k.value)


def levels_device(row_ptr, col, part_ptr, stream=None):
    """ilu0dd_levels_device: Algorithm 5's level sets of a reordered dropped
    pattern on the GPU. Arguments are arrays (host or device); returns device
    int32 tensors (lev_l, lev_u, nlev_l, nlev_u)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    rp, cl, pp = (torch.as_tensor(np.ascontiguousarray(a, np.int32) if isinstance(a, np.ndarray) else a,
                                  dtype=torch.int32, device=dev).contiguous() for a in (row_ptr, col, part_ptr))
    n, nsub = rp.numel() - 1, pp.numel() - 1
    out = [torch.empty(max(m, 1), dtype=torch.int32, device=dev) for m in (n, n, nsub, nsub)]
    rc = load().ilu0dd_levels_device(*(ctypes.c_void_p(t.data_ptr()) for t in (rp, cl, pp)), nsub,
                                     *(ctypes.c_void_p(t.data_ptr()) for t in out), _stream(stream))
    if rc:
        raise Ilu0DDError(rc, "ilu0dd_levels_device")
    return out[0][:n], out[1][:n], out[2][:nsub], out[3][:nsub]


def workspace_size(row_ptr, col, val, grid, sub, **opts) -> int:
    """Structural query (host only): workspace bytes, or raises Ilu0DDError."""
    b, keep = _bsr(row_ptr, col, val)
    g = Geom(*grid, *sub)
    o = default_opts(**opts)
    n = ctypes.c_size_t(0)
    rc = load().ilu0_dd_workspace_size(ctypes.byref(b), ctypes.byref(g), ctypes.byref(o), ctypes.byref(n))
    del keep
    if rc:
        raise Ilu0DDError(rc, "ilu0_dd_workspace_size")
    return int(n.value)


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t, n=None, what="vector"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{what} must be a contiguous float64 CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"{what} must have {n} entries, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


class Ilu0DD:
    """Subdomain ILU0 preconditioner + BiCGSTAB solver on one GPU.

    ``row_ptr``, ``col``, ``val`` are the natural-order BSR matrix, host
    arrays (``val`` of shape (nnzb, 3, 3) or flat) or CUDA tensors (device
    memory: int32, int32, float64); ``grid`` = (nx, ny, nz),
    ``sub`` = (sx, sy, sz) are the inputs of Algorithm 2. ``device_setup``
    factors and packs on the GPU (ilu0_dd_setup_planned with scratch), else on
    the host; both give the same bits.
    """

    def __init__(self, row_ptr, col, val, grid=None, sub=None, *, part_id=None, nparts=None, device=None,
                 stream=None, device_setup=True, **opts):
        import torch
        lib = load()
        self._lib = lib
        self.grid = tuple(grid) if grid is not None else None
        self.sub = tuple(sub) if sub is not None else None
        if part_id is None and (grid is None or sub is None):
            raise ValueError("give grid and sub (Algorithm 2) or part_id and nparts (a graph partition)")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        b, keep = _bsr(row_ptr, col, val)
        self.opts = default_opts(**opts)
        plan = ctypes.c_void_p()
        n, ns = ctypes.c_size_t(0), ctypes.c_size_t(0)
        if part_id is not None:
            labels = np.ascontiguousarray(part_id, np.int32)
            if labels.shape != (b.n_brows,):
                raise ValueError("part_id must hold one label per block row")
            if nparts is None:
                nparts = int(labels.max()) + 1 if labels.size else 0
            rc = lib.ilu0dd_plan_create_partitioned(ctypes.byref(b), labels.ctypes.data, int(nparts),
                                                    ctypes.byref(self.opts), ctypes.byref(plan), ctypes.byref(n),
                                                    ctypes.byref(ns))
            keep = keep + (labels,)
        else:
            g = Geom(*grid, *sub)
            rc = lib.ilu0dd_plan_create(ctypes.byref(b), ctypes.byref(g), ctypes.byref(self.opts),
                                        ctypes.byref(plan), ctypes.byref(n), ctypes.byref(ns))
        if rc:
            raise Ilu0DDError(rc, "ilu0dd_plan_create")
        try:
            with torch.cuda.device(self.device):
                self.workspace = torch.empty(max(int(n.value), 256), dtype=torch.uint8, device=self.device)
                # device setup: scratch for the factorisation and packing, released after setup
                scratch = (torch.empty(max(int(ns.value), 256), dtype=torch.uint8, device=self.device)
                           if device_setup else None)
                ctx = ctypes.c_void_p()
                rc = lib.ilu0_dd_setup_planned(plan, ctypes.byref(b), ctypes.c_void_p(self.workspace.data_ptr()),
                                               ctypes.c_size_t(self.workspace.numel()),
                                               ctypes.c_void_p(scratch.data_ptr() if scratch is not None else None),
                                               ctypes.c_size_t(scratch.numel() if scratch is not None else 0),
                                               _stream(stream), ctypes.byref(ctx))
                del scratch
        finally:
            lib.ilu0dd_plan_destroy(plan)
        del keep
        if rc:
            raise Ilu0DDError(rc, "ilu0_dd_setup_planned")
        self._ctx = ctx
        self.n = self.query("n")
        self.bs = self.query("block_dim")
        self.size = self.bs * self.n

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.ilu0_dd_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc:
            raise Ilu0DDError(rc, what)

    def _new(self):
        import torch
        return torch.empty(self.size, dtype=torch.float64, device=self.device)

    # -- hot path ---------------------------------------------------------
    def apply(self, r, z=None, stream=None):
        """z = M^-1 r (reordered numbering)."""
        z = self._new() if z is None else z
        self._check(self._lib.ilu0_dd_apply(self._ctx, _dptr(r, self.size, "r"), _dptr(z, self.size, "z"),
                                            _stream(stream)), "ilu0_dd_apply")
        return z

    def apply_host(self, r, z=None, stream=None, sync=True):
        """z = M^-1 r with HOST buffers (CPU tensors or numpy arrays, float64, 3N
        entries, reordered numbering); copies and applies pipelined by chunks of
        subdomains. Pinned CPU tensors let the copies overlap. Returns z once the
        stream has completed."""
        import torch
        def host_ptr(a, what):
            if isinstance(a, torch.Tensor):
                if a.is_cuda or a.dtype != torch.float64 or not a.is_contiguous() or a.numel() != self.size:
                    raise TypeError(f"{what} must be a contiguous float64 CPU tensor of {self.size} entries")
                return a.data_ptr()
            if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous
                    and a.size == self.size):
                raise TypeError(f"{what} must be a contiguous float64 array of {self.size} entries")
            return a.ctypes.data
        if z is None:
            z = np.empty(self.size, np.float64)
        st = _stream(stream)
        self._check(self._lib.ilu0_dd_apply_host(self._ctx, ctypes.c_void_p(host_ptr(r, "r")),
                                                 ctypes.c_void_p(host_ptr(z, "z")), st), "ilu0_dd_apply_host")
        if sync:
            (torch.cuda.current_stream() if stream is None else stream).synchronize()
        return z

    def apply_rowsync(self, r, z=None, stream=None):
        """z = M^-1 r with per-row completion flags (Algorithm 4's
        synchronization) instead of the level order; same bits as apply()."""
        z = self._new() if z is None else z
        self._check(self._lib.ilu0_dd_apply_rowsync(self._ctx, _dptr(r, self.size, "r"), _dptr(z, self.size, "z"),
                                                    _stream(stream)), "ilu0_dd_apply_rowsync")
        return z

    def apply_edge(self, r, z=None, stream=None):
        """z = M^-1 r with the edge-centric traversal (one thread per block,
        shared-memory atomics); equal to apply() to rounding."""
        z = self._new() if z is None else z
        self._check(self._lib.ilu0_dd_apply_edge(self._ctx, _dptr(r, self.size, "r"), _dptr(z, self.size, "z"),
                                                 _stream(stream)), "ilu0_dd_apply_edge")
        return z

    def apply_global_vector(self, r, z=None, stream=None):
        """z = M^-1 r (FP64 factors) with the subdomain vector in global memory
        instead of shared memory; same bits as apply()."""
        z = self._new() if z is None else z
        self._check(self._lib.ilu0_dd_apply_global_vector(self._ctx, _dptr(r, self.size, "r"),
                                                          _dptr(z, self.size, "z"), _stream(stream)),
                    "ilu0_dd_apply_global_vector")
        return z

    def apply_unfused(self, r, z=None, stream=None):
        """z = M^-1 r in two launches (L sweep, then D^-1 and U~ sweep)."""
        z = self._new() if z is None else z
        self._check(self._lib.ilu0_dd_apply_unfused(self._ctx, _dptr(r, self.size, "r"), _dptr(z, self.size, "z"),
                                                    _stream(stream)), "ilu0_dd_apply_unfused")
        return z

    def spmv(self, x, y=None, stream=None):
        """y = A_p x (reordered numbering, full matrix)."""
        y = self._new() if y is None else y
        self._check(self._lib.ilu0_dd_spmv(self._ctx, _dptr(x, self.size, "x"), _dptr(y, self.size, "y"),
                                           _stream(stream)), "ilu0_dd_spmv")
        return y

    def dot(self, x, y, out=None, stream=None):
        """x . y in the library's fixed order; returns a 1-element CUDA tensor."""
        import torch
        out = torch.empty(1, dtype=torch.float64, device=self.device) if out is None else out
        self._check(self._lib.ilu0_dd_dot(self._ctx, _dptr(x, self.size, "x"), _dptr(y, self.size, "y"),
                                          _dptr(out, 1, "out"), _stream(stream)), "ilu0_dd_dot")
        return out

    def permute(self, x, direction: int, out=None, stream=None):
        """direction 0: natural -> reordered; 1: reordered -> natural."""
        out = self._new() if out is None else out
        self._check(self._lib.ilu0_dd_permute(self._ctx, _dptr(x, self.size, "in"), _dptr(out, self.size, "out"),
                                              int(direction), _stream(stream)), "ilu0_dd_permute")
        return out

    def solve(self, b, x=None, stream=None, check=True):
        """BiCGSTAB (Algorithm 1) on natural-order device vectors; returns (x, info dict)."""
        x = self._new() if x is None else x
        info = Info()
        rc = self._lib.bicgstab_solve(self._ctx, _dptr(b, self.size, "b"), _dptr(x, self.size, "x"),
                                      ctypes.byref(info), _stream(stream))
        if rc and check:
            raise Ilu0DDError(rc, "bicgstab_solve")
        d = info.as_dict()
        d["status"] = rc
        return x, d

    def start(self, b, stream=None):
        """bicgstab_start: load b (natural numbering) and set the initial state."""
        self._check(self._lib.bicgstab_start(self._ctx, _dptr(b, self.size, "b"), _stream(stream)),
                    "bicgstab_start")

    def iterate(self, n, timed=False, stream=None):
        """bicgstab_iterate: n iterations; with timed=True returns (n, 5) kernel milliseconds."""
        ms = np.zeros(5 * n, np.float32) if timed else None
        self._check(self._lib.bicgstab_iterate(self._ctx, int(n), None if ms is None else ms.ctypes.data,
                                               _stream(stream)), "bicgstab_iterate")
        return None if ms is None else ms.reshape(n, 5)

    def state(self, stream=None):
        info = Info()
        self._check(self._lib.bicgstab_state(self._ctx, ctypes.byref(info), _stream(stream)), "bicgstab_state")
        return info.as_dict()

    # -- inspection -------------------------------------------------------
    def history(self, n=None):
        n = (self.opts.maxit + 1) if n is None else n
        buf = np.zeros(n, np.float64)
        self._check(self._lib.ilu0_dd_history(self._ctx, buf.ctypes.data, n), "ilu0_dd_history")
        return buf

    def query(self, what):
        v = ctypes.c_int64(0)
        self._check(self._lib.ilu0_dd_query(self._ctx, Q[what] if isinstance(what, str) else what,
                                            ctypes.byref(v)), "ilu0_dd_query")
        return int(v.value)

    def export(self, what):
        n, kept, nsub = self.n, self.query("kept"), self.query("nsub")
        bb = self.bs * self.bs
        spec = {X_PART_ID: (np.int32, n), X_PERM: (np.int32, n), X_IPERM: (np.int32, n),
                X_PART_PTR: (np.int32, nsub + 1), X_LEVEL_L: (np.int32, n), X_LEVEL_U: (np.int32, n),
                X_DD_ROW_PTR: (np.int32, n + 1), X_DD_COL: (np.int32, kept), X_L: (np.float64, bb * kept),
                X_UT: (np.float64, bb * kept), X_INVD: (np.float64, bb * n), X_AP_ROW_PTR: (np.int32, n + 1),
                X_AP_COL: (np.int32, self.query("nnzb")), X_STREAM: (np.uint8, self.query("stream_bytes")),
                X_SELL_COL: (np.int32, 32 * self.query("sell_slots")),
                X_SELL_VAL: (np.float64, bb * 32 * self.query("sell_slots"))}
        dt, cnt = spec[what]
        buf = np.empty(cnt, dt)
        self._check(self._lib.ilu0_dd_export(self._ctx, what, buf.ctypes.data, buf.nbytes), "ilu0_dd_export")
        return buf

    def device_error(self) -> int:
        v = ctypes.c_int32(0)
        self._check(self._lib.ilu0_dd_device_error(self._ctx, ctypes.byref(v)), "ilu0_dd_device_error")
        return int(v.value)

    def set_wait_limits(self, wait_us=0, stuck_piece=-1):
        """Bound of the apply's level waits in microseconds (0: default) and a
        piece whose completion is never reached (-1: none), for failure-path
        tests."""
        self._check(self._lib.ilu0dd_set_wait_limits(self._ctx, int(wait_us), int(stuck_piece)),
                    "ilu0dd_set_wait_limits")


class Batch:
    """Batched BiCGSTAB over several Ilu0DD contexts (one launch per step for all)."""

    def __init__(self, ctxs, stream=None, **opts):
        import torch
        self._lib = load()
        self.ctxs = list(ctxs)
        arr = (ctypes.c_void_p * len(self.ctxs))(*[c._ctx for c in self.ctxs])
        self._arr = arr
        n = ctypes.c_size_t(0)
        rc = self._lib.ilu0dd_batch_workspace_size(arr, len(self.ctxs), ctypes.byref(n))
        if rc:
            raise Ilu0DDError(rc, "ilu0dd_batch_workspace_size")
        self.device = self.ctxs[0].device
        self.workspace = torch.empty(max(int(n.value), 256), dtype=torch.uint8, device=self.device)
        self.opts = default_opts(**opts)
        b = ctypes.c_void_p()
        rc = self._lib.ilu0dd_batch_create(arr, len(self.ctxs), ctypes.byref(self.opts),
                                           ctypes.c_void_p(self.workspace.data_ptr()),
                                           ctypes.c_size_t(self.workspace.numel()), _stream(stream), ctypes.byref(b))
        if rc:
            raise Ilu0DDError(rc, "ilu0dd_batch_create")
        self._b = b

    def solve(self, bs, xs=None, stream=None, check=True):
        """bs: list of natural-order device vectors; returns (xs, [info dicts])."""
        n = len(self.ctxs)
        xs = [c._new() for c in self.ctxs] if xs is None else xs
        pb = (ctypes.c_void_p * n)(*[_dptr(b, c.size, "b").value for b, c in zip(bs, self.ctxs)])
        px = (ctypes.c_void_p * n)(*[_dptr(x, c.size, "x").value for x, c in zip(xs, self.ctxs)])
        infos = (Info * n)()
        rc = self._lib.bicgstab_solve_batched(self._b, pb, px, infos, _stream(stream))
        if rc and check:
            raise Ilu0DDError(rc, "bicgstab_solve_batched")
        return xs, [i.as_dict() for i in infos]

    def close(self):
        if getattr(self, "_b", None):
            self._lib.ilu0dd_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
