"""Serving (continuous batching): requests of different shapes arrive while
others run; each result must be exactly the result of the same search run
alone, and admission must respect the device-memory budget."""
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_2512_13365_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cse():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2512_13365_gb300 import cse as c
    return c


def _requests(n, n_proc, budget):
    reqs = synth.serving_requests(n_req=n, n_proc=n_proc, budget=budget)
    out = []
    for _, s in reqs:
        s.interval, s.cap = 16, 512
        out.append(s)
    return out


def _same(cse, a, b, n_mats):
    assert a.lists == b.lists and a.costs == b.costs
    for k in range(n_mats):
        assert np.array_equal(a.procs(k), b.procs(k))


def test_served_results_equal_alone(cse):
    reqs = _requests(6, 48, 40)
    sv = cse.Server(interval=16, cap=512, trace=True)
    schemes = [cse.Scheme(s.mats) for s in reqs]
    tickets = []
    for i, (s, sc) in enumerate(zip(reqs, schemes)):
        tickets.append(sv.submit(sc, s.weights, s.n_proc, s.seed, s.budget))
        if i % 2:
            time.sleep(0.002)  # later requests join while earlier ones run
    served = [sv.wait(t, timeout_us=120_000_000) for t in tickets]
    st = sv.stats()
    assert st["completed"] == len(reqs) and st["p99_ms"] >= st["p50_ms"] > 0 and st["steps_per_s"] > 0
    assert sv.peak()[0] > 1  # requests were on the device together
    for s, sc, r in zip(reqs, schemes, served):
        alone = cse.search(sc, s.weights, s.n_proc, s.seed, s.budget, 16, s.permille, 512, trace=True)
        _same(cse, r, alone, len(s.mats))
    ref = O.search_obj(reqs[0], n_threads=8)
    assert served[0].costs == ref.cost and served[0].lists == ref.lists
    sv.free()


def test_admission_by_memory_budget(cse):
    reqs = _requests(4, 32, 48)
    # a budget smaller than any single search: requests run one at a time
    sv = cse.Server(interval=16, cap=512, hbm_budget=1)
    sv2 = cse.Server(interval=16, cap=512, max_active_processes=1)
    schemes = [cse.Scheme(s.mats) for s in reqs]
    tickets = [sv.submit(sc, s.weights, s.n_proc, s.seed, s.budget) for s, sc in zip(reqs, schemes)]
    served = [sv.wait(t) for t in tickets]
    tickets2 = [sv2.submit(sc, s.weights, s.n_proc, s.seed, s.budget) for s, sc in zip(reqs, schemes)]
    served2 = [sv2.wait(t) for t in tickets2]
    for s, sc, r, r2 in zip(reqs, schemes, served, served2):
        alone = cse.search(sc, s.weights, s.n_proc, s.seed, s.budget, 16, s.permille, 512)
        _same(cse, r, alone, len(s.mats))
        _same(cse, r2, alone, len(s.mats))
    # one search at a time, also for requests queued together while the
    # server was idle
    assert sv.peak()[0] == 1 and sv2.peak()[0] == 1
    sv.free()
    sv2.free()


def test_idle_server_admits_a_burst_within_budget(cse):
    """Requests queued together while the server is idle are admitted up to
    the budget, not all at once: a process cap of two requests' worth keeps
    at most two searches on the device."""
    reqs = _requests(6, 32, 48)
    schemes = [cse.Scheme(s.mats) for s in reqs]
    units = max(len(s.mats) * s.n_proc for s in reqs)
    sv = cse.Server(interval=16, cap=512, max_active_processes=2 * units)
    tickets = [sv.submit(sc, s.weights, s.n_proc, s.seed, s.budget) for s, sc in zip(reqs, schemes)]
    for s, sc, t in zip(reqs, schemes, tickets):
        _same(cse, sv.wait(t), cse.search(sc, s.weights, s.n_proc, s.seed, s.budget, 16, s.permille, 512),
              len(s.mats))
    peak, rounds = sv.peak()
    assert 1 <= peak <= 2 and rounds >= 6
    sv.free()


def test_wait_timeout_and_bad_requests(cse):
    s = synth.config2(n_proc=256, budget=512)
    sv = cse.Server(interval=32, cap=128)
    sc = cse.Scheme(s.mats)
    t = sv.submit(sc, s.weights, s.n_proc, s.seed, s.budget)
    with pytest.raises(cse.CseError) as ei:
        sv.wait(t, timeout_us=0)
    assert ei.value.code == cse.CSE_ETIMEOUT
    r = sv.wait(t)
    assert r.total > 0
    with pytest.raises(cse.CseError):
        sv.submit(sc, (0,) * 6, 4, 0, 10)  # all weights zero
    sv.free()


def test_allocation_failure_is_reported_and_serving_goes_on(cse):
    """A request whose device state cannot be allocated (about 750 GB: the
    (6,6,6:153) shape with 2^20 processes per matrix) fails alone with
    CSE_ENOMEM at admission; the requests around it are served as usual."""
    small = _requests(2, 32, 32)
    big = synth.config4(n_proc=1 << 20, budget=32)
    sv = cse.Server(interval=16, cap=512)
    sch = [cse.Scheme(s.mats) for s in small]
    big_sc = cse.Scheme(big.mats)
    t0 = sv.submit(sch[0], small[0].weights, small[0].n_proc, small[0].seed, small[0].budget)
    tb = sv.submit(big_sc, big.weights, big.n_proc, big.seed, big.budget)
    t1 = sv.submit(sch[1], small[1].weights, small[1].n_proc, small[1].seed, small[1].budget)
    with pytest.raises(cse.CseError) as e:
        sv.wait(tb)
    assert e.value.code == cse.CSE_ENOMEM
    for s, sc, t in zip(small, sch, (t0, t1)):
        alone = cse.search(sc, s.weights, s.n_proc, s.seed, s.budget, 16, s.permille, 512)
        _same(cse, sv.wait(t), alone, len(s.mats))
    sv.free()


def test_cancel_queued_and_running_requests(cse):
    s = synth.config2(n_proc=4096, budget=8192)       # about 0.2 s: still running when cancelled
    q = synth.config2(n_proc=64, budget=64)
    sv = cse.Server(interval=32, cap=128, max_active_processes=3 * 4096)   # the others wait in the queue
    sc, qc = cse.Scheme(s.mats), cse.Scheme(q.mats)
    t_run = sv.submit(sc, s.weights, s.n_proc, s.seed, s.budget)
    t_queued = sv.submit(qc, q.weights, q.n_proc, q.seed, q.budget)
    t_after = sv.submit(qc, q.weights, q.n_proc, q.seed + 1, q.budget)
    sv.cancel(t_queued)
    time.sleep(0.02)
    sv.cancel(t_run)
    for t in (t_queued, t_run):
        with pytest.raises(cse.CseError) as e:
            sv.wait(t)
        assert e.value.code == cse.CSE_ECANCELED
    r = sv.wait(t_after)                                 # the rest is served as usual
    alone = cse.search(qc, q.weights, q.n_proc, q.seed + 1, q.budget, 32, q.permille, 128)
    _same(cse, r, alone, 3)
    with pytest.raises(cse.CseError):
        sv.cancel(t_after)                               # already finished (and collected)
    sv.free()


def test_search_on_another_thread_beside_the_server(cse):
    """A kernel's shared-memory limit is process-wide: a small search run on
    the caller's thread while the server serves a larger shape of the same
    word width must not lower the limit under the server's launches."""
    big = synth.config2(n_proc=512, budget=256)
    big.interval, big.cap = 16, 512          # W = 1 with a large per-process slice
    small = synth.config1(n_proc=16, budget=16)  # W = 1 with a small one
    sv = cse.Server(interval=16, cap=512)
    sb, ss = cse.Scheme(big.mats), cse.Scheme(small.mats)
    t = sv.submit(sb, big.weights, big.n_proc, big.seed, big.budget)
    for _ in range(20):
        r = cse.search(ss, small.weights, small.n_proc, small.seed, small.budget, 16, small.permille, small.cap)
        r.costs
        r.free()
    served = sv.wait(t, timeout_us=300_000_000)
    alone = cse.search(sb, big.weights, big.n_proc, big.seed, big.budget, 16, big.permille, 512)
    assert served.costs == alone.costs and served.lists == alone.lists
    sv.free()
