"""Autotuner for the subdomain box and apply block size (batching pattern).

Subdomain size trades preconditioner quality (smaller boxes drop more
couplings, Section 3.2, so BiCGSTAB needs more iterations) against parallelism
and per-block latency (larger boxes have more levels per sweep and fewer
blocks). Which side wins depends on the GPU and the system, so the tuner
measures time to solution through the library:

* candidates are (subdomain box, threads per block) pairs; those whose plan
  does not fit (shared memory, block size) are dropped by the library's
  host-side structural plan (``workspace_size``) before any device work;
* each remaining candidate gets a context and one warm-up solve (CUDA-graph
  capture); then ``repeats`` (5) rounds each time one solve of every
  candidate, the order rotated by one from round to round, so that drift over
  the tuning run (clocks, other work on the machine) falls on all candidates
  alike; a candidate's time is its median, with the minimum and maximum kept
  as its spread (all candidate contexts are alive at once: their device
  memory adds up);
* the choice is the first candidate (in candidate order) whose median lies
  within ``tie`` (5 %) of the fastest one, so that near-equal candidates do
  not swap places from run to run on timer noise (solves of the smallest
  systems take about a millisecond);
* a ragged batch is tuned per size class: the systems are sorted by size and
  cut into classes of equal count, and each class's subdomain box is tuned on
  its median system (``autotune_batch``); the batch's block size, one for all
  systems of a batched launch, is then tuned on the batched solve itself
  (``tune_batch_threads``).
"""
from __future__ import annotations

import time

import numpy as np

from .binding import Ilu0DD, Ilu0DDError, workspace_size

DEFAULT_SUBS = ((8, 8, 4), (8, 8, 8), (16, 8, 8), (16, 16, 8))
DEFAULT_THREADS = (0, 128, 192, 256)


def candidates(system, subs=DEFAULT_SUBS, threads=DEFAULT_THREADS, factor_prec="f32", **opts):
    """The (sub, threads_per_cta) pairs whose plan the library accepts for this
    system (host-side plan only; a box too large for shared memory or a block
    size out of range is refused there)."""
    grid = (system.nx, system.ny, system.nz)
    out = []
    for sub in subs:
        sub = tuple(min(s, g) for s, g in zip(sub, grid))
        for thr in threads:
            try:
                workspace_size(system.row_ptr, system.col, system.val, grid, sub, factor_prec=factor_prec,
                               threads_per_cta=thr, **opts)
            except Ilu0DDError:
                continue
            if (sub, thr) not in out:
                out.append((sub, thr))
    return out


def pick(trials, tie=0.05):
    """The first trial whose median is within `tie` of the fastest median."""
    fastest = min(t["seconds"] for t in trials)
    return next(t for t in trials if t["seconds"] <= (1.0 + tie) * fastest)


def autotune(system, subs=DEFAULT_SUBS, threads=DEFAULT_THREADS, factor_prec="f32", repeats=5, tie=0.05,
             **opts):
    """Return (best, trials) for a synth.System-like object (row_ptr, col, val,
    nx, ny, nz, b). Each trial: sub, threads_per_cta (as resolved by the
    library), seconds (median of `repeats` timed solves, one per round over
    all candidates), seconds_min, seconds_max, iterations. best = pick(trials,
    tie)."""
    import torch

    grid = (system.nx, system.ny, system.nz)
    b = torch.from_numpy(system.b).cuda()
    live, seen = [], set()
    try:
        for sub, thr in candidates(system, subs, threads, factor_prec, **opts):
            try:
                ctx = Ilu0DD(system.row_ptr, system.col, system.val, grid, sub, factor_prec=factor_prec,
                             threads_per_cta=thr, **opts)
            except Ilu0DDError:
                continue
            key = (sub, ctx.query("threads"))
            if key in seen:  # threads_per_cta = 0 resolved to a block size already timed
                ctx.close()
                continue
            seen.add(key)
            live.append((key, ctx))
            ctx.solve(b)  # warm-up: graph capture
        torch.cuda.synchronize()
        times = {key: [] for key, _ in live}
        infos = {}
        for rnd in range(repeats):
            k = rnd % max(1, len(live))
            for key, ctx in live[k:] + live[:k]:
                t0 = time.perf_counter()
                _, infos[key] = ctx.solve(b, check=False)
                torch.cuda.synchronize()
                times[key].append(time.perf_counter() - t0)
        trials = [dict(sub=key[0], threads_per_cta=key[1], seconds=float(np.median(times[key])),
                       seconds_min=min(times[key]), seconds_max=max(times[key]),
                       iterations=infos[key]["iterations"])
                  for key, _ in live if infos[key]["status"] == 0]
    finally:
        for _, ctx in live:
            ctx.close()
    if not trials:
        raise RuntimeError("no autotuning candidate solved the system")
    return pick(trials, tie), trials


def size_classes(systems, nclasses=3):
    """Indices of the systems sorted by size (cells) and cut into nclasses
    classes of (nearly) equal count, smallest first."""
    order = sorted(range(len(systems)), key=lambda i: systems[i].n)
    nclasses = max(1, min(nclasses, len(order)))
    return [order[len(order) * k // nclasses:len(order) * (k + 1) // nclasses] for k in range(nclasses)]


def autotune_batch(systems, nclasses=3, **kw):
    """Tune each size class of a ragged batch on its median system. Returns a
    list of dicts: members (system indices), representative (index), best,
    trials; and a per-system list of (sub, threads_per_cta)."""
    classes = []
    choice = [None] * len(systems)
    for members in size_classes(systems, nclasses):
        rep = members[len(members) // 2]
        best, trials = autotune(systems[rep], **kw)
        classes.append(dict(members=members, representative=rep, best=best, trials=trials))
        for i in members:
            s = systems[i]
            sub = tuple(min(a, g) for a, g in zip(best["sub"], (s.nx, s.ny, s.nz)))
            choice[i] = (sub, best["threads_per_cta"])
    return classes, choice


def tune_batch_threads(systems, boxes, threads=(128, 192, 256), factor_prec="f32", repeats=3, tie=0.05, **opts):
    """Block size of a batched launch (one for every system of the batch):
    for each candidate, contexts with the given per-system boxes and that
    block size, one warm-up batched solve (graph capture) and `repeats` timed
    ones. Returns (best, trials); trials hold threads, seconds (median),
    seconds_min, seconds_max."""
    import torch

    from .binding import Batch

    bs = [torch.from_numpy(s.b).cuda() for s in systems]
    trials = []
    for thr in threads:
        try:
            ctxs = [Ilu0DD(s.row_ptr, s.col, s.val, (s.nx, s.ny, s.nz), box, factor_prec=factor_prec,
                           threads_per_cta=thr, **opts) for s, box in zip(systems, boxes)]
        except Ilu0DDError:
            continue
        batch = Batch(ctxs)
        try:
            batch.solve(bs)
            torch.cuda.synchronize()
            times = []
            for _ in range(repeats):
                t0 = time.perf_counter()
                _, infos = batch.solve(bs, check=False)
                torch.cuda.synchronize()
                times.append(time.perf_counter() - t0)
            if all(i["status"] == 0 for i in infos):
                trials.append(dict(threads_per_cta=thr, seconds=float(np.median(times)), seconds_min=min(times),
                                   seconds_max=max(times)))
        finally:
            batch.close()
            for c in ctxs:
                c.close()
    if not trials:
        raise RuntimeError("no block size solved the batch")
    return pick(trials, tie), trials
