"""Scheme-level entry points on the GPU: the Brent-equation check (Section
3.1) against the oracle, and the component-wise (hybrid) minimum over
several results (Section 5)."""
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


def test_brent_valid_schemes(cse):
    U, V, W = synth.strassen_uvw()
    assert cse.brent_check(2, 2, 2, U, V, W) == 0
    for shape in [(2, 3, 4), (3, 3, 3), (4, 1, 5), (5, 5, 5)]:
        assert cse.brent_check(*shape, *synth.standard_uvw(*shape)) == 0


def test_brent_broken_schemes_match_oracle(cse):
    U, V, W = synth.strassen_uvw()
    for l in range(7):
        U2 = U.copy()
        a = int(np.nonzero(U[l])[0][0])
        U2[l, a] = -U2[l, a]
        assert cse.brent_check(2, 2, 2, U2, V, W) == O.brent_violations(2, 2, 2, U2, V, W) > 0
    rng = np.random.default_rng(5)
    for (m, n, p, r) in [(2, 3, 2, 9), (3, 4, 5, 47), (6, 6, 6, 153)]:
        U, V, W = (rng.integers(-1, 2, (r, k)).astype(np.int8) for k in (m * n, n * p, m * p))
        assert cse.brent_check(m, n, p, U, V, W) == O.brent_violations(m, n, p, U, V, W)


def test_hybrid_takes_the_componentwise_minimum(cse):
    base = synth.config2(n_proc=96, budget=64)
    sc = cse.Scheme(base.mats)
    rs = [cse.search(sc, base.weights, base.n_proc, seed, base.budget, base.interval, base.permille, base.cap)
          for seed in range(4)]
    costs = np.array([[r.fetch(k)[1] for k in range(3)] for r in rs])
    best, total = cse.hybrid(rs)
    assert best == [int(np.argmin(costs[:, k])) for k in range(3)]
    assert total == int(costs.min(axis=0).sum()) <= int(costs.sum(axis=1).min())
    for r in rs:
        r.free()
