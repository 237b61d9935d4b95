"""CPU tests of the C ABI library: it builds, loads, exports every declared symbol,
and its host-side structural logic (workspace query, argument checks) behaves.

No kernel is launched here; the structural query runs the host part of the
setup only (Algorithm 2, Algorithm 3, the drop of Section 3.2, level sets).
"""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

import paper_2508_04917_gb300 as g
import synth


def test_library_exports_every_declared_symbol():
    lib = g.load()
    names = g.declared_functions()
    assert {"ilu0_dd_setup", "ilu0_dd_apply", "bicgstab_solve", "ilu0_dd_workspace_size"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", g.library_path()], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert set(names) <= exported


def test_strerror_and_defaults():
    assert g.strerror(0) == "ok"
    assert "shared memory" in g.strerror(3)
    o = g.default_opts()
    assert o.factor_prec == g.F64 and o.maxit == 10000 and o.rtol == 1e-8 and o.use_graphs == 1


def _sys(grid=(8, 8, 8)):
    return synth.system(*grid, 3)


def test_workspace_size_scales_with_precision():
    s = _sys((16, 16, 16))
    sizes = {p: g.workspace_size(s.row_ptr, s.col, s.val, (16, 16, 16), (8, 8, 4), factor_prec=p)
             for p in ("f64", "f32", "bf16")}
    assert sizes["f64"] > sizes["f32"] > sizes["bf16"] > 0


def test_rejects_bad_patterns():
    s = _sys()
    col = s.col.copy()
    col[[1, 2]] = col[[2, 1]]  # unsorted row 0
    with pytest.raises(g.Ilu0DDError) as e:
        g.workspace_size(s.row_ptr, col, s.val, (8, 8, 8), (4, 4, 4))
    assert e.value.code == 1
    # drop the diagonal block of row 0 (keep the pattern consistent)
    rp = s.row_ptr.copy()
    q = [q for q in range(rp[0], rp[1]) if s.col[q] == 0][0]
    keep = np.ones(len(s.col), bool)
    keep[q] = False
    rp[1:] -= 1
    with pytest.raises(g.Ilu0DDError) as e:
        g.workspace_size(rp, s.col[keep], s.val[keep], (8, 8, 8), (4, 4, 4))
    assert e.value.code == 1
    with pytest.raises(g.Ilu0DDError) as e:
        g.workspace_size(s.row_ptr, s.col, s.val, (8, 8, 9), (4, 4, 4))  # N mismatch
    assert e.value.code == 1
    with pytest.raises(g.Ilu0DDError) as e:
        g.workspace_size(s.row_ptr, s.col, s.val, (8, 8, 8), (4, 4, 4), factor_prec=7)
    assert e.value.code == 1
    with pytest.raises(g.Ilu0DDError) as e:
        g.workspace_size(s.row_ptr, s.col, s.val, (8, 8, 8), (4, 4, 4), threads_per_cta=48)
    assert e.value.code == 1
    with pytest.raises(g.Ilu0DDError) as e:
        g.workspace_size(s.row_ptr, s.col, s.val, (8, 8, 8), (4, 4, 4), apply_mapping=2)
    assert e.value.code == 1
    with pytest.raises(TypeError):
        g.workspace_size(s.row_ptr, s.col, s.val, (8, 8, 8), (4, 4, 4), no_such_option=1)


def test_subdomain_shared_memory_limit():
    """Section 4 sizes subdomains so their vector fits in shared memory. On sm_103a
    (227 KiB per block) an FP64 subdomain of 9472 block rows (16x16x37 cells,
    222 KiB) fits; one more z-layer does not. FP32-factor contexts keep an FP32
    vector (16 bytes a row in the row-thread layout), so more rows fit."""
    grid = (16, 16, 38)
    rp, col = synth.pattern(*grid)
    val = np.zeros((len(col), 3, 3))
    assert g.workspace_size(rp, col, val, grid, (16, 16, 37)) > 0
    with pytest.raises(g.Ilu0DDError) as e:
        g.workspace_size(rp, col, val, grid, (16, 16, 38))
    assert e.value.code == 3
    assert g.workspace_size(rp, col, val, grid, (16, 16, 38), factor_prec="f32") > 0
    with pytest.raises(g.Ilu0DDError) as e:
        g.workspace_size(rp, col, val, grid, (16, 16, 37), prefetch_bytes=100)
    assert e.value.code == 1


def test_context_library_builds_and_exports():
    """The measurement library beside the path (vendor global ILU0, FP64 FMA rate)."""
    import context

    context.build()
    lib = context.load()
    for name in ("ctx_vendor_ilu0_create", "ctx_vendor_ilu0_apply", "ctx_vendor_spmv", "ctx_vendor_ilu0_factors",
                 "ctx_vendor_ilu0_destroy", "ctx_fp64_fma_rate"):
        assert hasattr(lib, name), name
    assert lib.ctx_vendor_ilu0_apply(None, None, None, None) == 4



def test_trace_from_environment():
    """ILU0DD_TRACE=1 turns on the per-phase timings of the defaults (checked in
    a child process: the environment is read when the defaults are filled)."""
    code = "import paper_2508_04917_gb300 as g; print(g.default_opts().trace)"
    repo = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for value, want in (("1", "1"), ("0", "0")):
        env = dict(os.environ, ILU0DD_TRACE=value)
        out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=repo)
        assert out.returncode == 0 and out.stdout.strip() == want, out.stderr
