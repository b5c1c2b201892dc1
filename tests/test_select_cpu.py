"""Host logic of the accuracy-adaptive free-space selector (no GPU): the
admissible candidates for a target precision and the choice rule."""

import pytest

import synth


@pytest.fixture(scope="module")
def sel():
    pytest.importorskip("torch")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2001_06113_gb300 import select
    return select


def test_candidates_follow_the_precision_floor(sel):
    """FP32 sums only above their floor; nu <= 4096; H grows with eps and is
    smaller for FP32 sums by log(2^29) / (2 d (1 + phimax))."""
    inst = synth.free_bump_gaussians((128,), seed=3, dt=1e-3, nsteps=30)
    loose = sel.candidates(inst, 1e-4)
    tight = sel.candidates(inst, 1e-12)
    assert {c.precision for c in loose} == {"mixed", "fp64"}
    assert {c.precision for c in tight} == {"fp64"}
    assert all(max(c.nu) <= 4096 for c in loose + tight)
    assert {c.R for c in loose} == {4, 8, 16}
    h = {c.precision: c.H for c in loose}
    assert h["fp64"] > h["mixed"] > 0
    assert max(c.H for c in tight) < h["fp64"]
    big = sel.candidates(synth.free_bump_gaussians((512,), seed=3, dt=1e-3, nsteps=30), 1e-4)
    assert {c.R for c in big} == {4, 8}                  # 16 * 512 > 4096


def test_choice_is_the_fastest_within_the_bound(sel):
    C = sel.Candidate
    cands = [C("fp64", 16, [1024], 2.0, err=1e-13, ms_per_step=3.0),
             C("fp64", 4, [256], 2.0, err=5e-6, ms_per_step=1.0),
             C("mixed", 8, [512], 1.0, err=2e-7, ms_per_step=0.5),
             C("mixed", 4, [256], 1.0, err=3e-4, ms_per_step=0.2)]
    pick = sel.choose(cands, 1e-4, safety=0.1)           # bound 1e-5: fp64 R = 4 (1.0 ms) loses to mixed R = 8
    assert (pick.precision, pick.R) == ("mixed", 8)
    pick = sel.choose(cands, 1e-5, safety=0.1)           # bound 1e-6: the mixed R = 8 candidate
    assert (pick.precision, pick.R) == ("mixed", 8)
    pick = sel.choose(cands, 1e-2, safety=0.1)           # bound 1e-3: all qualify, the fastest wins
    assert (pick.precision, pick.R) == ("mixed", 4)
    assert sel.choose(cands, 1e-13, safety=0.1) is None  # nothing within 1e-14
