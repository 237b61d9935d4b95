"""Bounded waits of the apply: the failure path, tested without a GPU fault.

The apply's warps start a level's rows once the previous level's pieces are
complete (the level order of Section 4.4, with one shared-memory mbarrier per
piece instead of block barriers). Every wait is bounded. A piece whose
completion is never reached (the stuck piece of ilu0dd_set_wait_limits, whose
mbarrier expects one arrival too many) makes each wait on it expire:
the block stops waiting and finishes, the device error word reads 1, the
other subdomains' outputs are untouched, bicgstab_solve and the batched solve
report ILU0DD_ERR_DEVICE_WAIT, and the context stays usable: with the stuck
piece cleared the apply gives its earlier bits again.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2508_04917_gb300 as g  # noqa: E402
from paper_2508_04917_gb300 import binding as B  # noqa: E402

GRID, SUB = (16, 16, 16), (8, 8, 4)


def make(bs=3, seed=3):
    s = synth.system(*GRID, seed, bs=bs)
    return s, g.Ilu0DD(s.row_ptr, s.col, s.val, GRID, SUB)


def cu(x):
    return torch.from_numpy(np.ascontiguousarray(x, np.float64)).cuda()


@pytest.mark.parametrize("bs", [3, 1])
def test_stuck_piece_expires_and_context_recovers(bs):
    s, ctx = make(bs)
    try:
        d = oracle.decompose(s.row_ptr, s.col, s.val, GRID, SUB)
        r = np.random.default_rng(1).uniform(-1, 1, ctx.size)
        z_ref = ctx.apply(cu(r))
        assert ctx.device_error() == 0
        # piece 0 = subdomain 0's first L level: the next level waits on it
        ctx.set_wait_limits(wait_us=200, stuck_piece=0)
        z = ctx.apply(cu(r))
        torch.cuda.synchronize()
        assert ctx.device_error() == 1
        assert ctx.device_error() == 0  # read and cleared
        first = bs * int(d.part_ptr[1])
        assert torch.equal(z[first:], z_ref[first:])  # only subdomain 0's block gave up
        ctx.set_wait_limits()
        z2 = ctx.apply(cu(r))
        assert ctx.device_error() == 0 and torch.equal(z2, z_ref)
        zo = oracle.apply(d.LU, r)
        assert np.abs(z2.cpu().numpy() - zo).max() <= 1e-12 * np.abs(zo).max()
    finally:
        ctx.close()


def test_stuck_piece_fails_the_solve_then_solves():
    s, ctx = make()
    try:
        ctx.set_wait_limits(wait_us=200, stuck_piece=0)
        x, info = ctx.solve(cu(s.b), check=False)
        assert info["status"] == B.ERR_DEVICE_WAIT
        assert ctx.device_error() == 1
        ctx.set_wait_limits()
        x, info = ctx.solve(cu(s.b))
        d = oracle.decompose(s.row_ptr, s.col, s.val, GRID, SUB)
        ref = oracle.bicgstab(d.Ap, d.LU, s.b.reshape(-1, 3)[d.perm].reshape(-1))
        assert info["status"] == 0 and info["iterations"] == ref.iterations
    finally:
        ctx.close()


def test_stuck_piece_in_a_batch_fails_that_system_only():
    systems = [make(seed=k) for k in (4, 5)]
    ctxs = [c for _, c in systems]
    bvec = [cu(s.b) for s, _ in systems]
    try:
        single = ctxs[1].solve(bvec[1])
        ctxs[0].set_wait_limits(wait_us=200, stuck_piece=0)
        batch = g.Batch(ctxs, maxit=60)  # the failed system iterates on to maxit
        xs, infos = batch.solve(bvec, check=False)
        batch.close()
        assert infos[0]["status"] == B.ERR_DEVICE_WAIT
        assert infos[1]["status"] == 0 and infos[1]["iterations"] == single[1]["iterations"]
        assert torch.equal(xs[1], single[0])
        assert ctxs[0].device_error() == 1
    finally:
        for c in ctxs:
            c.close()


def test_wait_limits_reject_bad_pieces():
    _, ctx = make()
    try:
        with pytest.raises(g.Ilu0DDError):
            ctx.set_wait_limits(stuck_piece=ctx.query("pieces"))
        with pytest.raises(g.Ilu0DDError):
            ctx.set_wait_limits(stuck_piece=-2)
    finally:
        ctx.close()
