"""The graph-partition path for matrices without a grid (Section 3.1's
graph-based labels; the paper uses METIS, this project breadth-first balls
grown to equal-size parts, as the paper's Section 5 balances its parts).

CPU tests: the oracle's partition pinned on graphs whose breadth-first order
is known in closed form, structural invariants on larger ones, and the
library's own implementation equal to the oracle's label by label.
"""
import numpy as np
import pytest

import oracle
import paper_2508_04917_gb300 as g
import synth


def _path(n):
    """Block pattern of a path 0 - 1 - ... - (n-1) (tridiagonal)."""
    rp, col = [0], []
    for i in range(n):
        col += [j for j in (i - 1, i, i + 1) if 0 <= j < n]
        rp.append(len(col))
    return np.array(rp, np.int32), np.array(col, np.int32)


def _union(*parts):
    """Disjoint union of patterns (block diagonal)."""
    rp, col, base = [0], [], 0
    for r, c in parts:
        for i in range(len(r) - 1):
            col += [int(x) + base for x in c[r[i]:r[i + 1]]]
            rp.append(len(col))
        base += len(r) - 1
    return np.array(rp, np.int32), np.array(col, np.int32)


def test_path_is_cut_from_its_far_end():
    """A path: the first search from vertex 0 ends at n-1; the second, from n-1,
    visits n-1, n-2, ..., 0, so vertex v is at position n-1-v."""
    n, k = 23, 5
    rp, col = _path(n)
    part, nparts = oracle.partition_bfs(rp, col, k)
    assert nparts == 5
    assert np.array_equal(part, (n - 1 - np.arange(n)) // k)


def test_disconnected_components_in_order():
    """Components are ordered by their smallest vertex, each reversed as above;
    positions run on across components."""
    a, b = _path(4), _path(6)
    rp, col = _union(a, b, _path(1))
    part, nparts = oracle.partition_bfs(rp, col, 3)
    order = [3, 2, 1, 0, 9, 8, 7, 6, 5, 4, 10]  # vertex at each position
    expect = np.empty(11, np.int32)
    for t, v in enumerate(order):
        expect[v] = t // 3
    assert nparts == 4 and np.array_equal(part, expect)


def test_grid_first_part_is_a_ball_around_the_far_corner():
    """A 2D grid (5-point pattern): from corner 0 the farthest vertex is the
    opposite corner alone, which starts the seed order; the first part is the
    first part_rows vertices of a breadth-first search from it, i.e. every
    vertex closer than the part's farthest member and nothing farther. Every
    part but the last is full."""
    nx, ny, k = 7, 5, 9
    rp, col = synth.pattern(nx, ny, 1)
    part, nparts = oracle.partition_bfs(rp, col, k)
    i, j = np.arange(nx * ny) % nx, np.arange(nx * ny) // nx
    dist = (nx - 1 - i) + (ny - 1 - j)
    first = part == 0
    dmax = dist[first].max()
    assert np.all(first[dist < dmax]) and not np.any(first[dist > dmax])
    counts = np.bincount(part, minlength=nparts)
    assert nparts == -(-nx * ny // k) and np.all(counts[:-1] == k) and counts[-1] == nx * ny - k * (nparts - 1)


def test_exhausted_ball_continues_from_next_seed():
    """Path 0..4 plus an isolated vertex 5, parts of 4: seed order 4,3,2,1,0,5;
    part 0 = {4,3,2,1}; part 1 starts at 0, whose ball ends at once, and
    continues from seed 5."""
    rp, col = _union(_path(5), _path(1))
    part, nparts = oracle.partition_bfs(rp, col, 4)
    assert nparts == 2 and np.array_equal(part, [1, 0, 0, 0, 0, 1])


def test_nonsymmetric_pattern_is_symmetrised():
    """Only A[1,0] present (no A[0,1]): the two vertices are still neighbours."""
    rp = np.array([0, 1, 3], np.int32)
    col = np.array([0, 0, 1], np.int32)
    part, nparts = oracle.partition_bfs(rp, col, 1)
    # first search from 0 ends at 1; the second visits 1, 0
    assert np.array_equal(part, [1, 0]) and nparts == 2


@pytest.mark.parametrize("grid,k", [((10, 9, 8), 64), ((16, 12, 10), 256), ((5, 5, 5), 7), ((12, 11, 10), 1000)])
def test_library_partition_equals_oracle(grid, k):
    s = synth.unstructured(*grid, 17)
    po, ko = oracle.partition_bfs(s.row_ptr, s.col, k)
    pl, kl = g.partition_bfs(s.row_ptr, s.col, k)
    assert ko == kl and np.array_equal(po, pl)
    counts = np.bincount(po, minlength=ko)
    assert np.all(counts[:-1] == k)


def test_partitioned_plan_sizes():
    """The labeled plan: workspace sizes for a valid partition; labels out of
    range and parts beyond shared memory are refused."""
    import ctypes
    from paper_2508_04917_gb300 import binding as B
    s = synth.unstructured(12, 10, 9, 3)
    part, k = g.partition_bfs(s.row_ptr, s.col, 512)
    lib = B.load()
    b, keep = B._bsr(s.row_ptr, s.col, s.val)
    opts = B.default_opts()
    plan = ctypes.c_void_p()
    nw, ns = ctypes.c_size_t(0), ctypes.c_size_t(0)
    lab = np.ascontiguousarray(part, np.int32)
    assert lib.ilu0dd_plan_create_partitioned(ctypes.byref(b), lab.ctypes.data, k, ctypes.byref(opts),
                                              ctypes.byref(plan), ctypes.byref(nw), ctypes.byref(ns)) == 0
    assert nw.value > 0 and ns.value > 0
    lib.ilu0dd_plan_destroy(plan)
    bad = lab.copy()
    bad[3] = k
    assert lib.ilu0dd_plan_create_partitioned(ctypes.byref(b), bad.ctypes.data, k, ctypes.byref(opts),
                                              ctypes.byref(plan), ctypes.byref(nw), ctypes.byref(ns)) == B.ERR_INVALID
    one = np.zeros(s.n, np.int32)  # 1,080 rows in one part: fits; 16x16x40 cells would not
    assert lib.ilu0dd_plan_create_partitioned(ctypes.byref(b), one.ctypes.data, 1, ctypes.byref(opts),
                                              ctypes.byref(plan), ctypes.byref(nw), ctypes.byref(ns)) == 0
    lib.ilu0dd_plan_destroy(plan)
    big = synth.unstructured(16, 16, 40, 3)
    bb, keep2 = B._bsr(big.row_ptr, big.col, big.val)
    z = np.zeros(big.n, np.int32)
    assert lib.ilu0dd_plan_create_partitioned(ctypes.byref(bb), z.ctypes.data, 1, ctypes.byref(opts),
                                              ctypes.byref(plan), ctypes.byref(nw), ctypes.byref(ns)) == B.ERR_SMEM
    del keep, keep2
