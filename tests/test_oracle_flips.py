"""Pins of the oracle's random-flip mode (Section 3.5.3; reading R16 of the
oracle): the flip move against hand-worked flips (tests/golden/
flip_example.txt), and every generated variant against what a flip must
keep: the scheme's tensor sum_l U_l (x) V_l (x) W_l (numpy, independent of
the oracle), hence every Brent equation, ternary entries and the rank."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2512_13365_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def tensor(U, V, W):
    return np.einsum("la,lb,lc->abc", U.astype(np.int64), V.astype(np.int64), W.astype(np.int64))


def _golden():
    for ln in open(os.path.join(GOLD, "flip_example.txt")):
        f = ln.split()
        if f and not f[0].startswith("#"):
            yield f


def _rows(f, names):
    out = {}
    i = 0
    while i < len(f):
        if f[i] in names:
            out[f[i]] = [int(x) for x in f[i + 1:i + 5]]
            i += 5
        else:
            i += 1
    return out


def test_hand_worked_flips():
    U, V, W = synth.standard_uvw(2, 2, 2)
    for f in _golden():
        if f[0] == "flip":
            l, m, x, side, applied = int(f[1]), int(f[2]), int(f[3]), int(f[4]), int(f[6])
            ok, u, v, w = O.flip_apply(U, V, W, l, m, x, side)
            assert ok == bool(applied)
            want = _rows(f, ("V0", "W1", "W0", "V1"))
            got = {"U": u, "V": v, "W": w}
            for name, row in want.items():
                assert list(got[name[0]][int(name[1])]) == row, (f, name)
            changed = {(k, i) for k, a, b in (("U", u, U), ("V", v, V), ("W", w, W))
                       for i in range(a.shape[0]) if not np.array_equal(a[i], b[i])}
            assert changed == {(n[0], int(n[1])) for n in want}
            assert np.array_equal(tensor(u, v, w), tensor(U, V, W))
        elif f[0] == "twice":
            l, m, x, side = (int(t) for t in f[1:5])
            ok1, u, v, w = O.flip_apply(U, V, W, l, m, x, side)
            ok2, u2, v2, w2 = O.flip_apply(u, v, w, l, m, x, side)
            assert (ok1, ok2) == (bool(int(f[6])), bool(int(f[7])))
            assert np.array_equal(v2, v) and np.array_equal(w2, w)
        elif f[0] == "negated":
            Un, Vn = U.copy(), V.copy()
            Un[1], Vn[1] = -U[1], -V[1]
            assert np.array_equal(tensor(Un, Vn, W), tensor(U, V, W))
            ok, u, v, w = O.flip_apply(Un, Vn, W, 0, 1, 0, 0)
            assert ok
            want = _rows(f, ("V0", "W1"))
            assert list(v[0]) == want["V0"] and list(w[1]) == want["W1"]
            assert np.array_equal(tensor(u, v, w), tensor(U, V, W))


@pytest.mark.parametrize("fmt", [(2, 2, 2), (2, 3, 4), (3, 3, 3), (4, 4, 4)])
def test_variants_keep_the_scheme(fmt):
    m, n, p = fmt
    U, V, W = synth.standard_uvw(m, n, p)
    T = tensor(U, V, W)
    flips = []
    for it in range(3):
        for var in range(6):
            k, u, v, w = O.flip_variant(m, n, p, U, V, W, 11, it, var, 24)
            assert 0 <= k <= 24 and (var > 0 or k == 0)
            assert np.array_equal(tensor(u, v, w), T)
            assert O.brent_violations(m, n, p, u, v, w) == 0
            assert set(np.unique(np.concatenate([u.ravel(), v.ravel(), w.ravel()]))) <= {-1, 0, 1}
            assert all(np.any(a != 0, axis=1).all() for a in (u, v, w))   # no term vanished: rank kept
            if var == 0:
                assert np.array_equal(u, U) and np.array_equal(v, V) and np.array_equal(w, W)
            flips.append(k)
    assert max(flips) > 1


def test_variants_are_reproducible_and_differ_by_iteration():
    U, V, W = synth.standard_uvw(3, 3, 3)
    a = O.flip_variant(3, 3, 3, U, V, W, 5, 2, 3, 16)
    b = O.flip_variant(3, 3, 3, U, V, W, 5, 2, 3, 16)
    c = O.flip_variant(3, 3, 3, U, V, W, 5, 3, 3, 16)
    assert a[0] == b[0] and all(np.array_equal(x, y) for x, y in zip(a[1:], b[1:]))
    assert not all(np.array_equal(x, y) for x, y in zip(a[1:], c[1:]))


def test_strassen_has_no_flip():
    """No two terms of Strassen's scheme share a factor up to sign, so no flip
    applies and every variant is the scheme itself."""
    U, V, W = synth.strassen_uvw()
    for var in range(1, 5):
        k, u, v, w = O.flip_variant(2, 2, 2, U, V, W, 1, 0, var, 32)
        assert k == 0 and np.array_equal(u, U) and np.array_equal(v, V) and np.array_equal(w, W)
