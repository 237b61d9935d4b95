"""The autotuner on the GPU: every candidate the host-side plan accepts is
timed once per round (order rotated), the choice follows the tie rule, and the
chosen configuration solves the system."""
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2508_04917_gb300 as g  # noqa: E402
from paper_2508_04917_gb300.autotune import autotune, candidates, pick  # noqa: E402


def test_autotune_times_every_candidate_and_picks_by_the_tie_rule():
    s = synth.system(24, 20, 16, 11)
    subs, threads = ((8, 8, 4), (8, 8, 8)), (128, 192)
    cands = candidates(s, subs, threads)
    best, trials = autotune(s, subs, threads, repeats=3)
    assert sorted((t["sub"], t["threads_per_cta"]) for t in trials) == sorted(cands)
    for t in trials:
        assert t["seconds_min"] <= t["seconds"] <= t["seconds_max"] and t["iterations"] > 0
    assert best == pick(trials)
    fastest = min(t["seconds"] for t in trials)
    assert best["seconds"] <= 1.05 * fastest
    ctx = g.Ilu0DD(s.row_ptr, s.col, s.val, (24, 20, 16), best["sub"], factor_prec="f32",
                   threads_per_cta=best["threads_per_cta"])
    try:
        _, info = ctx.solve(torch.from_numpy(s.b).cuda())
        assert info["status"] == 0 and info["iterations"] == best["iterations"]
    finally:
        ctx.close()

