"""Random-flip mode (Section 3.5.3) on the device: the flip kernel's variants
equal the oracle's bit for bit (same Philox draws, same ternary flips), the
device Brent check of every variant is zero for a valid scheme and flags a
broken one, and the search of every variant equals the oracle's."""
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


@pytest.mark.parametrize("fmt", [(2, 2, 2), (2, 3, 4), (3, 3, 3), (4, 4, 4)])
def test_device_variants_equal_the_oracle(cse, fmt):
    U, V, W = synth.standard_uvw(*fmt)
    for it in (0, 3):
        fl, vU, vV, vW, bad = cse.flip_variants(*fmt, U, V, W, 12, 5, it, 20)
        assert (bad == 0).all()
        for v in range(12):
            k, oU, oV, oW = O.flip_variant(*fmt, U, V, W, 5, it, v, 20)
            assert fl[v] == k
            assert np.array_equal(vU[v], oU) and np.array_equal(vV[v], oV) and np.array_equal(vW[v], oW)
    assert fl.max() > 0


def test_strassen_variants_are_strassen(cse):
    U, V, W = synth.strassen_uvw()
    fl, vU, vV, vW, bad = cse.flip_variants(2, 2, 2, U, V, W, 8, 1, 0, 32)
    assert (fl == 0).all() and (bad == 0).all()
    assert all(np.array_equal(vU[v], U) and np.array_equal(vV[v], V) and np.array_equal(vW[v], W) for v in range(8))


def test_device_brent_check_flags_a_broken_scheme(cse):
    U, V, W = synth.standard_uvw(2, 2, 3)
    W = W.copy()
    W[0, 0] = -W[0, 0]
    fl, vU, vV, vW, bad = cse.flip_variants(2, 2, 3, U, V, W, 4, 2, 0, 8)
    want = [O.brent_violations(2, 2, 3, vU[v], vV[v], vW[v]) for v in range(4)]
    assert bad.tolist() == want and min(want) > 0


def test_flip_search_equals_the_oracle(cse):
    U, V, W = synth.standard_uvw(3, 3, 3)
    kw = dict(n_variants=4, n_proc=24, seed=3, iterations=2, budget=48, interval=16, permille=400, cap=128,
              max_flips=12)
    best = cse.flip_search(3, 3, 3, U, V, W, synth.PAPER_WEIGHTS, **kw)
    totals, lists = [], {}
    for it in range(2):
        row = []
        for v in range(4):
            _, u, vv, w = O.flip_variant(3, 3, 3, U, V, W, 3, it, v, 12)
            ref = O.search(synth.scheme_sides(u, vv, w), synth.PAPER_WEIGHTS, 24, 3 + it, 48, 16, 400, 128,
                           n_threads=8, digests=False)
            row.append(ref.total)
            lists[(it, v)] = (ref.cost, ref.lists)
        totals.append(row)
    assert best["totals"] == totals
    flat = [(t, it, v) for it, row in enumerate(totals) for v, t in enumerate(row)]
    t, it, v = min(flat)
    assert (best["total"], best["iteration"], best["variant"]) == (t, it, v)
    assert (best["costs"], best["lists"]) == lists[(it, v)]
    assert O.brent_violations(3, 3, 3, best["U"], best["V"], best["W"]) == 0
