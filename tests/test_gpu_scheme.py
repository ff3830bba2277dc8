"""Scheme-level entry points on the GPU: the Brent-equation check (Section
3.1) against the oracle, the component-wise (hybrid) minimum over several
results (Section 5), and the device Philox4x32-10 that every draw of a
search comes from."""
import os

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


def test_device_philox_known_answers(cse):
    golden = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.txt")
    n = 0
    for ln in open(golden):
        ln = ln.split("#")[0].strip()
        if not ln:
            continue
        w = [int(x, 16) for x in ln.split()]
        seed = w[4] | w[5] << 32
        assert cse.philox(seed, np.array([w[0:4]], np.uint32)).tolist() == [w[6:10]]
        n += 1
    assert n == 3


def test_device_philox_equals_oracle(cse):
    """The device generator equals the oracle's Philox4x32-10 (pinned to the
    published known-answer vectors) on 10^6 counters: random ones under three
    keys, and the structured counters of the searches' draws (process, step,
    matrix << 24 | purpose << 20 | extra, key)."""
    rng = np.random.default_rng(11)
    total = 0
    for seed in (0, 0xFFFFFFFFFFFFFFFF, 0x243F6A8885A308D3):
        ctr = rng.integers(0, 1 << 32, size=(300000, 4), dtype=np.uint64).astype(np.uint32)
        key = [seed & 0xFFFFFFFF, seed >> 32]
        assert np.array_equal(cse.philox(seed, ctr), O.philox_n(ctr, key))
        total += ctr.shape[0]
    p, t, m, u, x = np.meshgrid(np.arange(64), np.arange(64), np.arange(3), np.arange(5), np.arange(4),
                                indexing="ij")
    ctr = np.stack([p.ravel(), t.ravel(), (m.ravel() << 24) | (u.ravel() << 20) | x.ravel(),
                    (p.ravel() * 2654435761) & 0xFFFFFFFF], axis=1).astype(np.uint32)
    assert np.array_equal(cse.philox(5, ctr), O.philox_n(ctr, [5, 0]))
    total += ctr.shape[0]
    assert total >= 10 ** 6
    assert cse.philox(0, np.zeros((0, 4), np.uint32)).shape == (0, 4)
