"""Autotuner for the subdomain box and apply block size (batching pattern).

Subdomain size trades preconditioner quality (smaller boxes drop more
couplings, Section 3.2, so BiCGSTAB needs more iterations) against parallelism
and per-block latency (larger boxes have more levels per sweep and fewer
blocks). Which side wins depends on the GPU and the system, so the tuner
measures: for each candidate (subdomain box, threads per block) it builds a
context for a representative system, runs one warm-up and one timed
BiCGSTAB solve through the library, and keeps the fastest time to solution.
"""
from __future__ import annotations

import time

from .binding import Ilu0DD, Ilu0DDError

DEFAULT_SUBS = ((8, 8, 8), (16, 8, 8), (16, 16, 8))
DEFAULT_THREADS = (0, 128)


def autotune(system, subs=DEFAULT_SUBS, threads=DEFAULT_THREADS, factor_prec="f32", **opts):
    """Return (best, trials) for a synth.System-like object (row_ptr, col, val, nx, ny, nz, b).

    best = dict(sub=..., threads_per_cta=..., seconds=..., iterations=...)."""
    import torch

    grid = (system.nx, system.ny, system.nz)
    b = torch.from_numpy(system.b).cuda()
    trials = []
    for sub in subs:
        for thr in threads:
            try:
                ctx = Ilu0DD(system.row_ptr, system.col, system.val, grid, sub, factor_prec=factor_prec,
                             threads_per_cta=thr, **opts)
            except Ilu0DDError:
                continue
            try:
                ctx.solve(b)  # warm-up: graph capture
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, info = ctx.solve(b, check=False)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                if info["status"] == 0:
                    trials.append(dict(sub=tuple(sub), threads_per_cta=ctx.query("threads"), seconds=dt,
                                       iterations=info["iterations"]))
            finally:
                ctx.close()
    if not trials:
        raise RuntimeError("no autotuning candidate solved the system")
    best = min(trials, key=lambda t: t["seconds"])
    return best, trials
