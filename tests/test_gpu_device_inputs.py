"""The boundary with a device-resident matrix: ilu0dd_bsr's arrays in device
memory (the form the boundary's setup call takes its matrix in) give the same
context as host arrays, bit for bit, on both numeric setup paths (device
factorization with scratch, host factorization) and for the graph-partition
path; mixed host/device arrays work too."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2508_04917_gb300 as g  # noqa: E402
from paper_2508_04917_gb300 import binding as B  # noqa: E402

ARRAYS = (B.X_STREAM, B.X_SELL_COL, B.X_SELL_VAL, B.X_PERM, B.X_PART_PTR, B.X_LEVEL_L, B.X_LEVEL_U, B.X_L, B.X_UT,
          B.X_INVD)


def _dev(s):
    return (torch.from_numpy(s.row_ptr).cuda(), torch.from_numpy(s.col).cuda(),
            torch.from_numpy(np.ascontiguousarray(s.val).reshape(-1)).cuda())


def _same(a, b):
    for what in ARRAYS:
        assert np.array_equal(a.export(what).view(np.uint8), b.export(what).view(np.uint8)), what


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16", "df64"])
@pytest.mark.parametrize("device_setup", [True, False])
def test_device_matrix_equals_host_matrix(prec, device_setup):
    grid, sub = (20, 18, 9), (8, 8, 4)
    s = synth.system(*grid, 7, model=synth.MODEL_LAYERED)
    h = g.Ilu0DD(s.row_ptr, s.col, s.val, grid, sub, factor_prec=prec, keep_host=1, device_setup=device_setup)
    d = g.Ilu0DD(*_dev(s), grid, sub, factor_prec=prec, keep_host=1, device_setup=device_setup)
    try:
        _same(h, d)
        b = torch.from_numpy(s.b).cuda()
        xh, ih = h.solve(b)
        xd, idd = d.solve(b)
        assert ih["iterations"] == idd["iterations"] and torch.equal(xh, xd)
    finally:
        h.close()
        d.close()


def test_device_matrix_partitioned_and_mixed():
    """Graph partition of a device-resident pattern, then contexts from device
    arrays and from a mix (host pattern, device values; device pattern, host
    values): the host-array results."""
    s = synth.unstructured(10, 10, 10, 6)
    rp, col, val = _dev(s)
    part_h, n_h = g.partition_bfs(s.row_ptr, s.col, 128)
    part_d, n_d = g.partition_bfs(rp, col, 128)
    assert n_h == n_d and np.array_equal(part_h, part_d)
    h = g.Ilu0DD(s.row_ptr, s.col, s.val, part_id=part_h, nparts=n_h, keep_host=1)
    others = [g.Ilu0DD(rp, col, val, part_id=part_h, nparts=n_h, keep_host=1),
              g.Ilu0DD(s.row_ptr, s.col, val, part_id=part_h, nparts=n_h, keep_host=1),
              g.Ilu0DD(rp, col, s.val, part_id=part_h, nparts=n_h, keep_host=1, device_setup=False)]
    try:
        for d in others:
            _same(h, d)
    finally:
        h.close()
        for d in others:
            d.close()


def test_device_arrays_must_be_tensors_of_the_right_type():
    s = synth.system(4, 4, 4, 1)
    rp, col, val = _dev(s)
    with pytest.raises(ValueError):
        g.Ilu0DD(rp.to(torch.int64), col, val, (4, 4, 4), (2, 2, 2))
    with pytest.raises(ValueError):
        g.Ilu0DD(rp, col, val.to(torch.float32), (4, 4, 4), (2, 2, 2))
