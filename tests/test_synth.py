"""The common input generator: determinism, an independent re-derivation of entries, shapes."""
import math

import numpy as np
import pytest

import synth

M64 = (1 << 64) - 1


def _sm64_out(z):
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def _bits(seed, stream, index):
    key = _sm64_out((seed * 0x9E3779B97F4A7C15 + stream) & M64)
    return _sm64_out((key + (index + 1) * 0x9E3779B97F4A7C15) & M64)


def _unit(seed, stream, index):
    return (_bits(seed, stream, index) >> 11) * 2.0 ** -53


def test_splitmix_reference_vector():
    """SplitMix64's output function: with the standard state increment, the first
    outputs from state 0 are the published reference values."""
    assert _sm64_out(0x9E3779B97F4A7C15) == 0xE220A8397B1DCDAF
    assert _sm64_out((2 * 0x9E3779B97F4A7C15) & M64) == 0x6E789E6AA1B965F4
    for idx in (0, 1, 12345, 2 ** 40):
        assert synth.bits(7, 3, idx) == _bits(7, 3, idx)


def test_entries_rederived():
    """Recompute some matrix entries of the laplace model from the counter generator."""
    nx, ny, nz, seed = 5, 4, 3, 9
    s = synth.system(nx, ny, nz, seed)
    g = 2 + nx * (1 + ny * 1)  # cell (2, 1, 1)
    q = [q for q in range(s.row_ptr[g], s.row_ptr[g + 1]) if s.col[q] == g][0]
    for e in range(9):
        ref = (6.5 if e % 4 == 0 else 0.0) + (-0.1 + 0.2 * _unit(seed, 1, 9 * g + e))
        assert s.val[q].reshape(-1)[e] == ref
    # +x neighbour block (direction 1)
    q = [q for q in range(s.row_ptr[g], s.row_ptr[g + 1]) if s.col[q] == g + 1][0]
    for e in range(9):
        ref = (-1.0 if e % 4 == 0 else 0.0) + (-0.1 + 0.2 * _unit(seed, 2, (6 * g + 1) * 9 + e))
        assert s.val[q].reshape(-1)[e] == ref
    for a in range(3):
        assert s.xstar[3 * g + a] == -1.0 + 2.0 * _unit(seed, 3, 3 * g + a)


def test_layered_model_structure():
    """Layered model: zero block-row sums up to the 0.01 I shift, harmonic-mean face
    weights, and kappa constant through 8-cell z-layers of a column."""
    nx, ny, nz = 4, 3, 10
    s = synth.system(nx, ny, nz, 5, model=synth.MODEL_LAYERED)
    for g in range(s.n):
        blocks = s.val[s.row_ptr[g]:s.row_ptr[g + 1]]
        assert np.abs(blocks.sum(0) - 0.01 * np.eye(3)).max() <= 1e-9 * np.abs(blocks).max()

    def kappa(i, j, k):
        idx = i + nx * (j + ny * (k // 8))
        u1, u2 = _unit(5, 4, 2 * idx), _unit(5, 4, 2 * idx + 1)
        return math.exp(2 * math.sqrt(-2 * math.log(1 - u1)) * math.cos(2 * math.pi * u2))

    g = 1 + nx * (1 + ny * 3)       # cell (1, 1, 3); +z neighbour (1, 1, 4) is in the same layer
    q = [q for q in range(s.row_ptr[g], s.row_ptr[g + 1]) if s.col[q] == g + nx * ny][0]
    ka, kb = kappa(1, 1, 3), kappa(1, 1, 4)
    assert ka == kb
    h = 2 * ka * kb / (ka + kb)
    P = np.array([-0.1 + 0.2 * _unit(5, 2, (6 * g + 5) * 9 + e) for e in range(9)]).reshape(3, 3)
    assert np.allclose(s.val[q], -h * (np.eye(3) + P), rtol=1e-12, atol=0)


@pytest.mark.parametrize("grid", [(1, 1, 1), (3, 1, 1), (4, 3, 2), (16, 16, 16)])
def test_pattern_and_counts(grid):
    s = synth.system(*grid, 1)
    assert s.nnzb == synth.nnzb(*grid) == s.n + 2 * ((grid[0] - 1) * grid[1] * grid[2]
                                                     + grid[0] * (grid[1] - 1) * grid[2]
                                                     + grid[0] * grid[1] * (grid[2] - 1))
    for i in range(s.n):
        c = s.col[s.row_ptr[i]:s.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0) and i in c
    dense_b = np.zeros(3 * s.n)
    for i in range(s.n):
        for q in range(s.row_ptr[i], s.row_ptr[i + 1]):
            dense_b[3 * i:3 * i + 3] += s.val[q] @ s.xstar[3 * s.col[q]:3 * s.col[q] + 3]
    assert np.abs(dense_b - s.b).max() <= 1e-12 * max(1.0, np.abs(s.b).max())


def test_deterministic_and_seeded():
    a = synth.system(6, 5, 4, 3)
    b = synth.system(6, 5, 4, 3)
    c = synth.system(6, 5, 4, 4)
    assert np.array_equal(a.val, b.val) and np.array_equal(a.b, b.b)
    assert not np.array_equal(a.val, c.val)


def test_ragged_sides_range():
    sides = synth.ragged_batch(64)
    flat = [v for s in sides for v in s]
    assert min(flat) >= 24 and max(flat) <= 96 and len(set(flat)) > 10
    assert sides == synth.ragged_batch(64)
