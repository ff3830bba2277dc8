"""Checkpoint / resume: a search checkpointed after B1 steps and resumed for
B2 more must give exactly what one search of B1 + B2 steps gives, down to
every process's record, because every draw is keyed by (seed, process,
step)."""
import numpy as np
import pytest

from paper_2512_13365_gb300 import synth

pytestmark = pytest.mark.gpu

FIELDS = ("best_cost", "best_len", "runs", "best_hash", "traj_hash", "ops", "substeps", "best_strategy",
          "method_ops")


@pytest.fixture(scope="module")
def cse():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2512_13365_gb300 import cse as c
    return c


def _same(a, b, n_mats):
    assert a.costs == b.costs and a.lists == b.lists
    for k in range(n_mats):
        pa, pb = a.procs(k), b.procs(k)
        for f in FIELDS:
            assert np.array_equal(pa[f], pb[f]), (k, f)
    assert a.counters() == b.counters()


@pytest.mark.parametrize("gi_shared", [False, True])
def test_resume_equals_uninterrupted_step_clock(cse, gi_shared):
    s = synth.config2(n_proc=160, budget=160)
    sc = cse.Scheme(s.mats)
    whole = cse.search(sc, s.weights, s.n_proc, s.seed, 160, s.interval, s.permille, s.cap, trace=True,
                       gi_shared=gi_shared)
    first = cse.search(sc, s.weights, s.n_proc, s.seed, 96, s.interval, s.permille, s.cap, trace=True,
                       gi_shared=gi_shared)
    ck = first.checkpoint()
    first.free()
    rest = cse.resume(sc, ck, 64)
    _same(whole, rest, 3)
    # and a second hop: 96 + 32 + 32
    first = cse.search(sc, s.weights, s.n_proc, s.seed, 96, s.interval, s.permille, s.cap, trace=True,
                       gi_shared=gi_shared)
    mid = cse.resume(sc, first.checkpoint(), 32)
    last = cse.resume(sc, mid.checkpoint(), 32)
    _same(whole, last, 3)
    for r in (whole, first, mid, last, rest):
        r.free()


def test_resume_equals_uninterrupted_hbm_path(cse):
    s = synth.config4(n_proc=8, budget=48)
    sc = cse.Scheme(s.mats)
    whole = cse.search(sc, s.weights, s.n_proc, s.seed, 48, 16, s.permille, s.cap, trace=True)
    first = cse.search(sc, s.weights, s.n_proc, s.seed, 32, 16, s.permille, s.cap, trace=True)
    rest = cse.resume(sc, first.checkpoint(), 16)
    _same(whole, rest, 3)
    for r in (whole, first, rest):
        r.free()


def test_resume_equals_uninterrupted_iteration_mode(cse):
    s = synth.config2(n_proc=96, budget=12)
    sc = cse.Scheme(s.mats)
    whole = cse.search(sc, s.weights, s.n_proc, s.seed, 12, 0, s.permille, s.cap, trace=True)
    first = cse.search(sc, s.weights, s.n_proc, s.seed, 5, 0, s.permille, s.cap, trace=True)
    rest = cse.resume(sc, first.checkpoint(), 7)
    _same(whole, rest, 3)
    assert whole.iterations() == rest.iterations()
    for r in (whole, first, rest):
        r.free()


def test_checkpoint_needs_a_sharing_boundary(cse):
    s = synth.config2(n_proc=16, budget=40)   # 40 is not a multiple of the interval 32
    sc = cse.Scheme(s.mats)
    r = cse.search(sc, s.weights, s.n_proc, s.seed, 40, s.interval, s.permille, s.cap)
    with pytest.raises(cse.CseError):
        r.checkpoint()
    r.free()


def test_resume_refuses_a_scheme_with_other_entries(cse):
    """A checkpoint records a hash of the matrices it was taken on: resuming it
    on a scheme of the same shapes but other entries is refused."""
    s = synth.config2(n_proc=32, budget=32)
    sc = cse.Scheme(s.mats)
    first = cse.search(sc, s.weights, s.n_proc, s.seed, 32, s.interval, s.permille, s.cap)
    ck = first.checkpoint()
    first.free()
    other = [m.copy() for m in s.mats]
    other[1] = -other[1]  # same shapes and nonzeros, other signs
    with pytest.raises(cse.CseError) as e:
        cse.resume(cse.Scheme(other), ck, 32)
    assert e.value.code == cse.CSE_EINVAL
    cse.resume(sc, ck, 32).free()  # the scheme it was taken on still resumes


def test_resume_keeps_the_wider_kernel(cse):
    """A search run on the wider kernels (CSE_FLAG_WIDE_WORDS) resumes on the
    same kernels, whatever the resuming call asks: the checkpoint records the
    state layout."""
    s = synth.config4(n_proc=8, budget=48)
    sc = cse.Scheme(s.mats)
    whole = cse.search(sc, s.weights, s.n_proc, s.seed, 48, 16, s.permille, s.cap, trace=True)
    first = cse.search(sc, s.weights, s.n_proc, s.seed, 32, 16, s.permille, s.cap, trace=True, wide_words=True)
    rest = cse.resume(sc, first.checkpoint(), 16)
    _same(whole, rest, 3)
    for r in (whole, first, rest):
        r.free()
