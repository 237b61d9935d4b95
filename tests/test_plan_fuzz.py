"""Host-side robustness of the structural setup (no GPU): random block
patterns, random partitions and malformed inputs go through the library's
plan (ilu0dd_plan_create_partitioned / ilu0_dd_workspace_size) and
partitioner without crashing; valid inputs give a plan, malformed ones
ILU0DD_ERR_INVALID. Seeded, a few hundred cases, seconds."""
import ctypes

import numpy as np
import pytest

import paper_2508_04917_gb300 as g
from paper_2508_04917_gb300 import binding as B


def random_pattern(rng, n, density, symmetric):
    """Sorted rows with the diagonal; off-diagonal entries drawn at random."""
    rows = [set([i]) for i in range(n)]
    m = int(density * n * n)
    for _ in range(m):
        i, j = rng.integers(0, n, 2)
        rows[i].add(int(j))
        if symmetric:
            rows[j].add(int(i))
    rp, col = [0], []
    for r in rows:
        col += sorted(r)
        rp.append(len(col))
    return np.array(rp, np.int32), np.array(col, np.int32)


def plan_rc(rp, col, labels, nparts, bs=3):
    n = len(rp) - 1
    val = np.zeros((len(col), bs, bs)) if bs == 3 else np.zeros(len(col))
    b, keep = B._bsr(rp, col, val)
    opts = B.default_opts()
    plan = ctypes.c_void_p()
    nw, ns = ctypes.c_size_t(0), ctypes.c_size_t(0)
    lab = np.ascontiguousarray(labels, np.int32)
    rc = B.load().ilu0dd_plan_create_partitioned(ctypes.byref(b), lab.ctypes.data if n else None, int(nparts),
                                                 ctypes.byref(opts), ctypes.byref(plan), ctypes.byref(nw),
                                                 ctypes.byref(ns))
    if rc == 0:
        assert nw.value > 0
        B.load().ilu0dd_plan_destroy(plan)
    del keep
    return rc


@pytest.mark.parametrize("seed", range(40))
def test_random_patterns_and_partitions_plan(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 300))
    rp, col = random_pattern(rng, n, float(rng.uniform(0.0, 0.05)), bool(seed % 2))
    # the breadth-first partition: labels in range, parts of exactly part_rows but the last
    k = int(rng.integers(1, 80))
    part, nparts = g.partition_bfs(rp, col, k)
    assert part.min() >= 0 and part.max() == nparts - 1 and nparts == (n + k - 1) // k
    counts = np.bincount(part, minlength=nparts)
    assert np.all(counts[:-1] == k) and counts[-1] == n - k * (nparts - 1)
    assert plan_rc(rp, col, part, nparts) == 0
    # arbitrary labels (parts need not be connected or balanced); empty parts too
    np_ = int(rng.integers(1, 20))
    labels = rng.integers(0, np_, n)
    assert plan_rc(rp, col, labels, np_) == 0
    assert plan_rc(rp, col, labels, np_, bs=1) == 0


@pytest.mark.parametrize("seed", range(20))
def test_malformed_inputs_are_refused(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(4, 120))
    rp, col = random_pattern(rng, n, 0.03, True)
    labels = np.zeros(n, np.int32)
    assert plan_rc(rp, col, labels, 1) == 0
    bad = col.copy()
    bad[int(rng.integers(0, len(col)))] = n + int(rng.integers(0, 5))  # column out of range
    assert plan_rc(rp, bad, labels, 1) == B.ERR_INVALID
    i = int(rng.integers(0, n))
    if rp[i + 1] - rp[i] >= 2:  # swap two entries: unsorted row
        sw = col.copy()
        sw[rp[i]], sw[rp[i] + 1] = sw[rp[i] + 1], sw[rp[i]]
        assert plan_rc(rp, sw, labels, 1) == B.ERR_INVALID
    # a duplicated column (not strictly ascending)
    q = int(rng.integers(rp[i], rp[i + 1]))
    dup_col = np.insert(col, q, col[q])
    dup_rp = rp.copy()
    dup_rp[i + 1:] += 1
    assert plan_rc(dup_rp, dup_col, labels, 1) == B.ERR_INVALID
    # labels out of range
    lab = labels.copy()
    lab[int(rng.integers(0, n))] = 3
    assert plan_rc(rp, col, lab, 1) == B.ERR_INVALID
    # the diagonal of one row removed
    j = int(np.where(col[rp[i]:rp[i + 1]] == i)[0][0]) + rp[i]
    nd_col = np.delete(col, j)
    nd_rp = rp.copy()
    nd_rp[i + 1:] -= 1
    assert plan_rc(nd_rp, nd_col, labels, 1) == B.ERR_INVALID
