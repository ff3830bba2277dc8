"""Pins of the CPU oracle to facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
known-answer vectors, the paper's worked example (Section 3.2.2), hand-derived
scores, closed forms of the step clock, exhaustive search on tiny inputs, and
invariants checked by independent numpy code.
"""
import itertools
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2512_13365_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _lines(name):
    with open(os.path.join(GOLD, name)) as f:
        for ln in f:
            ln = ln.strip()
            if ln and not ln.startswith("#"):
                yield ln


# ---------------------------------------------------------------- helpers
def expand(mat, entries):
    """Independent check of a substitution list: express every fresh variable
    over the original ones and rebuild each final row from them."""
    rows, nx = mat.shape
    cur = np.zeros((rows, nx + len(entries)), dtype=np.int64)
    cur[:, :nx] = mat
    defs = [np.eye(nx, dtype=np.int64)[v] for v in range(nx)]
    for t, e in enumerate(entries):
        i, j, s = O.unentry(e)
        k = nx + t
        assert i < j < k
        defs.append(defs[i] + s * defs[j])
        hit = (cur[:, i] != 0) & (cur[:, j] == s * cur[:, i])
        cur[hit, k] = cur[hit, i]
        cur[hit, i] = 0
        cur[hit, j] = 0
    D = np.stack(defs)
    return cur, cur @ D


def cost_of(cur, n_f):
    return int(n_f + sum(np.count_nonzero(r) - 1 for r in cur))


# ---------------------------------------------------------------- Philox
def test_philox_known_answers():
    n = 0
    for ln in _lines("philox4x32_10_kat.txt"):
        w = [int(x, 16) for x in ln.split()]
        assert O.philox(w[0:4], w[4:6]) == w[6:10]
        assert O.philox_n(np.array([w[0:4]] * 3, np.uint32), w[4:6]).tolist() == [w[6:10]] * 3
        n += 1
    assert n == 3


def test_philox_batch_equals_single_calls():
    rng = np.random.default_rng(7)
    ctr = rng.integers(0, 1 << 32, size=(257, 4), dtype=np.uint64).astype(np.uint32)
    key = [0x9E3779B9, 0x12345678]
    got = O.philox_n(ctr, key)
    assert got.shape == (257, 4)
    for q in (0, 1, 100, 256):
        assert got[q].tolist() == O.philox(ctr[q].tolist(), key)


# ---------------------------------------------------------------- worked example
def _example():
    mat, final, subst, pairs = [], [], [], []
    sec = None
    vals = {}
    for ln in _lines("paper_example.txt"):
        f = ln.split()
        if f[0] in ("matrix", "final"):
            sec = f[0]
            continue
        if f[0] in ("naive", "cost", "optimum"):
            vals[f[0]] = int(f[1])
            sec = None
        elif f[0] == "subst":
            subst.append(tuple(int(x) for x in f[1:]))
        elif f[0] == "pair":
            pairs.append(tuple(int(x) for x in f[1:]))
        elif sec == "matrix":
            mat.append([int(x) for x in f])
        elif sec == "final":
            final.append([int(x) for x in f])
    return np.array(mat, np.int8), np.array(final, np.int8), subst, pairs, vals


def test_paper_example_naive_and_cost():
    mat, final, subst, _, vals = _example()
    assert O.naive(mat) == vals["naive"] == 8
    out, cost = O.apply(mat, [O.entry(*s) for s in subst])
    assert cost == vals["cost"] == 6
    assert np.array_equal(out, final)


def test_paper_example_pair_counts():
    mat, _, _, pairs, _ = _example()
    got = [(O.unkey(k), c) for k, c in O.pairs(mat)]
    assert got == [((i, j, s), c) for i, j, s, c in pairs]
    # all other pairs occur exactly once
    allp = O.pairs(mat, min_c=1)
    assert sum(c for _, c in allp) == sum(3 * 2 if n == 4 else 3 for n in (4, 3, 4)) == 15
    assert all(c == 1 for k, c in allp if O.unkey(k) not in [(i, j, s) for i, j, s, _ in pairs])


def test_paper_example_optimum_and_greedy():
    mat, _, _, _, vals = _example()
    assert O.bruteforce(mat) == vals["optimum"] == 6
    # Greedy (max c, lowest canonical key) takes (x1 - x2) first, then
    # (x3 - x4) (derived by hand from the rows), and reaches 6.
    r = O.search([mat], (0, 0, 0, 0, 0, 1), 1, 0, 2, 64, 0, 16)
    assert r.cost == [6]
    assert [O.unentry(e) for e in r.lists[0]] == [(0, 1, -1), (2, 3, -1)]


# ---------------------------------------------------------------- Strassen
def test_strassen_textbook():
    U, V, W = synth.strassen_uvw()
    # Brent equations: sum_l U[l,(i,j)] V[l,(j',k)] W[l,(i',k')] = d_jj' d_ii' d_kk'
    T = np.einsum("la,lb,lc->abc", U.astype(int), V.astype(int), W.astype(int))
    ref = np.zeros((4, 4, 4), dtype=int)
    for i, j, k in itertools.product(range(2), repeat=3):
        ref[i * 2 + j, j * 2 + k, i * 2 + k] = 1
    assert np.array_equal(T, ref)
    sides = synth.scheme_sides(U, V, W)
    # Strassen's algorithm takes 18 additions (Section 2.2)
    assert sum(O.naive(m) for m in sides) == 18
    # no signed pair repeats in any side, so Algorithm 1 cannot improve it
    for m in sides:
        assert O.pairs(m) == []
        assert O.bruteforce(m) == O.naive(m)
    r = O.search(sides, synth.PAPER_WEIGHTS, 8, 3, 20, 4, 400, 32)
    assert r.total == 18 and r.length == [0, 0, 0]


# ---------------------------------------------------------------- brute force
def _py_bruteforce(mat):
    """Exhaustive search without memo, over every sequence of substitutions of
    pairs with c >= 2 (Algorithm 1), for a second route to the optimum."""
    rows, nx = mat.shape

    def rec(cur):
        nz = [np.nonzero(r)[0] for r in cur]
        cnt = {}
        for r, idx in zip(cur, nz):
            for a, b in itertools.combinations(idx, 2):
                kk = (a, b, int(r[a] * r[b]))
                cnt[kk] = cnt.get(kk, 0) + 1
        best = sum(len(x) - 1 for x in nz)
        for (a, b, s), c in cnt.items():
            if c < 2:
                continue
            nxt = np.zeros((rows, cur.shape[1] + 1), dtype=np.int64)
            nxt[:, :-1] = cur
            hit = (cur[:, a] != 0) & (cur[:, b] == s * cur[:, a])
            nxt[hit, -1] = cur[hit, a]
            nxt[hit, a] = 0
            nxt[hit, b] = 0
            best = min(best, 1 + rec(nxt))
        return best

    return rec(mat.astype(np.int64))


@pytest.mark.parametrize("seed", range(6))
def test_bruteforce_matches_plain_enumeration(seed):
    mat = synth.random_matrix(seed, 4, 5, 2, 4, n_planted=2, frac=(0.5, 0.75))
    assert O.bruteforce(mat) == _py_bruteforce(mat)


@pytest.mark.parametrize("seed", range(8))
def test_search_never_beats_optimum_and_usually_reaches_it(seed):
    mat = synth.random_matrix(100 + seed, 5, 6, 2, 4, n_planted=2, frac=(0.4, 0.8))
    opt = O.bruteforce(mat)
    r = O.search([mat], synth.PAPER_WEIGHTS, 256, seed, 64, 8, 400, 32)
    assert r.cost[0] >= opt
    assert r.cost[0] == opt  # 256 processes x 64 steps on 5 x 6 reach the optimum


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("seed", range(4))
def test_result_lists_are_valid_programs(seed):
    mats = [synth.random_matrix(200 + seed, 12, 8, 2, 5, n_planted=4),
            synth.random_matrix(300 + seed, 8, 12, 2, 5, n_planted=3)]
    r = O.search(mats, synth.PAPER_WEIGHTS, 32, seed, 96, 16, 400, 64)
    for mi, (m, lst, cost) in enumerate(zip(mats, r.lists, r.cost)):
        cur, back = expand(m, lst)
        assert np.array_equal(back, m.astype(np.int64))       # expansion reproduces E
        assert cost_of(cur, len(lst)) == cost                 # Cost = n_f + A_naive(E_final)
        # each substitution saved c - 1 >= 1: replay and count rows
        c_sum, cur2 = 0, np.zeros((m.shape[0], m.shape[1] + len(lst)), dtype=np.int64)
        cur2[:, :m.shape[1]] = m
        for t, e in enumerate(lst):
            i, j, s = O.unentry(e)
            hit = (cur2[:, i] != 0) & (cur2[:, j] == s * cur2[:, i])
            c = int(hit.sum())
            assert c >= 2
            c_sum += c - 1
            k = m.shape[1] + t
            cur2[hit, k] = cur2[hit, i]
            cur2[hit, i] = 0
            cur2[hit, j] = 0
        assert cost == O.naive(m) - c_sum
        # per-process records are valid too
        assert (r.digests[mi]["best_cost"] >= cost).all()


def test_digest_records_match_lists():
    mats = [synth.random_matrix(7, 10, 7, 2, 5, n_planted=3)]
    r = O.search(mats, synth.PAPER_WEIGHTS, 16, 5, 64, 8, 400, 48)
    d = r.digests[0]
    win = int(np.argmin(d["best_cost"]))
    assert d["best_cost"][win] == r.cost[0] and d["best_len"][win] == r.length[0]
    assert (d["substeps"] <= 64).all()


# ---------------------------------------------------------------- step clock
def test_step_clock_closed_form_greedy():
    mat, *_ = _example()
    # g only, no sharing: every run is (0,1,-), (2,3,-) and ends after its
    # second step, so B steps give ceil(B/2) runs and B substitutions.
    for B in (1, 2, 7, 10):
        r = O.search([mat], (0, 0, 0, 0, 0, 1), 1, 0, B, 1000, 0, 16)
        d = r.digests[0][0]
        assert d["runs"] == (B + 1) // 2 and d["substeps"] == B
        assert d["best_cost"] == (6 if B >= 2 else 7)


def test_sharing_replay_closed_form():
    mat, *_ = _example()
    # interval 4, permille 1000: the snapshot after step 3 is the g run
    # (L = 2, K = floor(3*2/4) = 1), so every later run replays k = 1
    # substitution and finishes in one step.  12 steps: 2 + 8 runs.
    r = O.search([mat], (0, 0, 0, 0, 0, 1), 1, 0, 12, 4, 1000, 16)
    d = r.digests[0][0]
    assert d["runs"] == 10 and d["substeps"] == 12 and r.cost == [6]
    # permille 0: no replays, 6 runs
    r0 = O.search([mat], (0, 0, 0, 0, 0, 1), 1, 0, 12, 4, 0, 16)
    assert r0.digests[0][0]["runs"] == 6


def test_share_probability():
    """A run starts from a shared prefix with probability permille / 1000
    (Section 3.5.2; the paper's 40%).  On the worked example with Greedy, a
    fresh run takes 2 steps and a shared one (k = 1) 1 step, so after the
    first run the mean run length is 2 - p: the share fraction follows from
    the run counts of 2000 processes over 200 steps."""
    mat, *_ = _example()
    for permille in (400, 40, 1000):
        r = O.search([mat], (0, 0, 0, 0, 0, 1), 2000, 0, 202, 1, permille, 16, n_threads=8)
        runs = r.digests[0]["runs"].mean()
        p_hat = 2 - 200 / (runs - 1)
        assert abs(p_hat - permille / 1000) < 0.01, (permille, p_hat)


@pytest.mark.parametrize("seed", range(3))
def test_shared_list_changes_only_when_beaten(seed):
    """The shared solution is replaced only by a strictly lower Cost
    (Section 3.5.2, reading R12): after every round whose lowest best Cost is
    unchanged the shared list is the same list, although other processes
    reach that Cost with other lists; when the Cost drops the list changes."""
    mat = synth.random_matrix(500 + seed, 16, 8, 2, 5, n_planted=4)
    w = (0, 1, 0, 1, 0, 0)    # ga and wr: many different lists of equal Cost
    cost, curve, snap = O.search_snapshots([mat], w, 256, seed, 320, 8, 400, 64, n_threads=8)
    c, h = curve[0], snap[0]
    assert c[-1] == cost[0] and all(x > 0 for x in h)
    for r in range(1, len(c)):
        if c[r] == c[r - 1]:
            assert h[r] == h[r - 1], r
        else:
            assert c[r] < c[r - 1] and h[r] != h[r - 1], r


def test_op_count_hand_derived():
    """The algorithmic op count (the roofline's numerator, counted alike by
    the oracle and the kernels) on the worked example, against the values
    derived by hand in tests/golden/ops_example.txt."""
    mat, *_ = _example()
    want = {ln.split()[0]: [int(x) for x in ln.split()[1:]] for ln in _lines("ops_example.txt")}
    g = (0, 0, 0, 0, 0, 1)
    assert O.search([mat], g, 1, 0, 1, 1000, 0, 16).digests[0][0]["ops"] == want["g_step1"][0]
    assert O.search([mat], g, 1, 0, 2, 1000, 0, 16).digests[0][0]["ops"] == want["g_step2"][0]
    # gi processes (process 0 starts with Greedy): one scoring pass, one substitution
    ops = O.search([mat], synth.GI_ONLY, 64, 0, 1, 1000, 0, 16).digests[0]["ops"][1:]
    allowed = {want["gi_select"][0] + x for x in want["gi_subst"]}
    assert set(int(x) for x in ops) <= allowed and len(set(int(x) for x in ops)) >= 2


def test_method_op_count_hand_derived():
    """The method op count (reading R15: the work the method itself must do,
    independent of the engine) on the worked example, against the values
    derived by hand in tests/golden/ops_example.txt."""
    mat, *_ = _example()
    want = {ln.split()[0]: [int(x) for x in ln.split()[1:]] for ln in _lines("ops_example.txt")}
    g = (0, 0, 0, 0, 0, 1)
    assert O.search([mat], g, 1, 0, 1, 1000, 0, 16).digests[0][0]["method_ops"] == want["m_g_step1"][0]
    assert O.search([mat], g, 1, 0, 2, 1000, 0, 16).digests[0][0]["method_ops"] == want["m_g_step2"][0]
    ops = O.search([mat], synth.GI_ONLY, 64, 0, 1, 1000, 0, 16).digests[0]["method_ops"][1:]
    allowed = {want["m_gi_select"][0] + x for x in want["m_gi_subst"]}
    assert set(int(x) for x in ops) <= allowed and len(set(int(x) for x in ops)) >= 2
    ops = O.search([mat], synth.GP_ONLY, 64, 0, 1, 1000, 0, 16).digests[0]["method_ops"][1:]
    allowed = {want["m_gp_select"][0] + x for x in want["m_gi_subst"]}
    assert set(int(x) for x in ops) <= allowed
    rows40 = np.ones((40, 2), np.int8)  # 64-bit words: ceil(40 / 64) = 1 per column
    assert O.search([rows40], g, 1, 0, 1, 1000, 0, 8).digests[0][0]["method_ops"] == want["m_g_40rows"][0]


def test_column_cap_ends_runs():
    mat = synth.random_matrix(11, 16, 6, 4, 6, n_planted=6, frac=(0.4, 0.6))
    # cap = n_x + 2: at most two substitutions per run
    r = O.search([mat], synth.PAPER_WEIGHTS, 8, 1, 40, 1000, 0, 8)
    assert max(r.length) <= 2
    assert (r.digests[0]["best_len"] <= 2).all()


def test_permille_zero_is_independent_of_interval():
    mats = [synth.random_matrix(21, 12, 8, 2, 5, n_planted=3)]
    a = O.search(mats, synth.PAPER_WEIGHTS, 16, 9, 80, 8, 0, 64)
    b = O.search(mats, synth.PAPER_WEIGHTS, 16, 9, 80, 1000, 0, 64)
    assert np.array_equal(a.digests["traj_hash"], b.digests["traj_hash"])


def test_thread_count_does_not_change_results():
    s = synth.config2(n_proc=64, budget=96)
    a = O.search_obj(s, n_threads=1)
    b = O.search_obj(s, n_threads=7)
    assert np.array_equal(a.digests, b.digests) and a.lists == b.lists


def test_subset_matches_full_run_before_first_boundary():
    s = synth.config2(n_proc=64, budget=32)
    full = O.search_obj(s)
    sub = [0, 5, 17, 63]
    part = O.search_obj(s, subset=sub)
    for mi in range(3):
        assert np.array_equal(full.digests[mi][sub], part.digests[mi][sub])


def test_first_run_of_process_zero_is_greedy():
    mat = synth.random_matrix(31, 14, 8, 2, 5, n_planted=4)
    g = O.search([mat], (0, 0, 0, 0, 0, 1), 1, 0, 6, 1000, 0, 64)
    mixed = O.search([mat], synth.GI_ONLY, 1, 0, 6, 1000, 0, 64)
    # process 0 starts with g whatever the weights
    assert g.digests[0][0]["traj_hash"] == mixed.digests[0][0]["traj_hash"]


def test_invalid_arguments_rejected():
    mat = np.array([[1, 1], [1, 0]], np.int8)
    with pytest.raises(ValueError):
        O.search([np.array([[2, 1]], np.int8)], synth.PAPER_WEIGHTS, 1, 0, 1, 1, 0, 8)
    with pytest.raises(ValueError):
        O.search([np.array([[0, 0]], np.int8)], synth.PAPER_WEIGHTS, 1, 0, 1, 1, 0, 8)
    with pytest.raises(ValueError):
        O.search([mat], (0,) * 6, 1, 0, 1, 1, 0, 8)
    with pytest.raises(ValueError):
        O.search([mat], synth.PAPER_WEIGHTS, 1, 0, 1, 1, 0, 2)  # cols >= cap


# ---------------------------------------------------------------- strategies
def test_greedy_takes_first_maximum():
    assert O.select_basic(O.G, [2, 5, 3, 5, 1 + 1], []) == 1


def test_ga_uniform_over_ties():
    counts = [3, 7, 2, 7, 7, 5, 7]
    ties = [1, 3, 4, 6]
    u = np.random.default_rng(0).integers(0, 2**32, 200000, dtype=np.uint64)
    hist = np.zeros(len(counts))
    for x in u[:40000]:
        hist[O.select_basic(O.GA, counts, [int(x)])] += 1
    assert set(np.nonzero(hist)[0]) == set(ties)
    exp = 40000 / 4
    chi2 = sum((hist[t] - exp) ** 2 / exp for t in ties)
    assert chi2 < 16.3  # 3 dof, p = 0.001
    # exact map: index (u * n_ties) >> 32 among ties in canonical order
    assert O.select_basic(O.GA, counts, [0]) == 1
    assert O.select_basic(O.GA, counts, [2**32 - 1]) == 6
    assert O.select_basic(O.GA, counts, [2**31]) == 4


def test_wr_proportional_to_profit():
    counts = [2, 5, 3, 2, 9]
    w = np.array(counts) - 1
    hist = np.zeros(len(counts))
    n = 40000
    for x in np.random.default_rng(1).integers(0, 2**32, n, dtype=np.uint64):
        hist[O.select_basic(O.WR, counts, [int(x)])] += 1
    exp = n * w / w.sum()
    chi2 = float(((hist - exp) ** 2 / exp).sum())
    assert chi2 < 18.5  # 4 dof, p = 0.001
    assert O.select_basic(O.WR, counts, [0]) == 0
    assert O.select_basic(O.WR, counts, [2**32 - 1]) == 4


def test_gr_mixes_ga_and_wr():
    counts = [2, 4, 4, 3]
    # coin below 3*2^30 -> ga on (u[1]); else wr on u[1]
    assert O.select_basic(O.GR, counts, [0, 0]) == 1
    assert O.select_basic(O.GR, counts, [3 * 2**30 - 1, 2**32 - 1]) == 2
    assert O.select_basic(O.GR, counts, [3 * 2**30, 0]) == 0
    assert O.select_basic(O.GR, counts, [2**32 - 1, 2**32 - 1]) == 3


def test_mix_step_frequencies():
    """Mixed picks gi, ga, gr, wr per step with probabilities 8:4:2:1
    (Section 3.4, reading R7): exact cut points of (u * 15) >> 32 and a
    chi-square over uniform draws."""
    want = [O.GI] * 8 + [O.GA] * 4 + [O.GR] * 2 + [O.WR]
    for r in range(15):
        first = -(-(r << 32) // 15)           # smallest u with (u * 15) >> 32 == r
        assert O.mix_strategy(first) == want[r]
        if r:
            assert O.mix_strategy(first - 1) == want[r - 1]
    assert O.mix_strategy(2**32 - 1) == O.WR
    n = 150000
    hist = {k: 0 for k in (O.GI, O.GA, O.GR, O.WR)}
    for x in np.random.default_rng(5).integers(0, 2**32, n, dtype=np.uint64):
        hist[O.mix_strategy(int(x))] += 1
    exp = {O.GI: 8 * n / 15, O.GA: 4 * n / 15, O.GR: 2 * n / 15, O.WR: n / 15}
    chi2 = sum((hist[k] - exp[k]) ** 2 / exp[k] for k in exp)
    assert chi2 < 16.3  # 3 dof, p = 0.001


def test_alpha_and_beta_reach_both_ends():
    """alpha in [0, 0.5] and beta in [0.5, 1] (Section 3.4.2) on the 2^-16 grid
    (reading R8): the lowest and highest draws reach both closed ends, and
    the values rise with the draw."""
    assert O.alpha_beta(0, 0) == (0, 32768)
    assert O.alpha_beta(2**32 - 1, 2**32 - 1) == (32768, 65536)
    u = np.sort(np.random.default_rng(3).integers(0, 2**32, 2000, dtype=np.uint64))
    ab = np.array([O.alpha_beta(int(x), int(x)) for x in u])
    assert (np.diff(ab[:, 0]) >= 0).all() and (np.diff(ab[:, 1]) >= 0).all()
    assert (ab[:, 1] - ab[:, 0] == 32768).all()


def test_best_record_changes_only_on_strict_improvement():
    """A process keeps the first run that reached its lowest Cost (reading
    R11: only a strictly lower Cost replaces the best record).  Without
    sharing, a search 10x longer whose best Cost is the same must keep the
    same best list, although many later runs tie with it."""
    mat = synth.random_matrix(77, 10, 7, 2, 5, n_planted=3)
    w = (0, 1, 0, 0, 0, 0)   # ga: uniform among the tied maxima, so tying runs differ
    short = O.search([mat], w, 32, 0, 60, 1000, 0, 64).digests[0]
    long = O.search([mat], w, 32, 0, 600, 1000, 0, 64).digests[0]
    same = short["best_cost"] == long["best_cost"]
    assert same.sum() >= 8 and (long["runs"] > short["runs"] + 5).all()
    assert (short["best_hash"][same] == long["best_hash"][same]).all()


def test_run_start_strategy_frequencies():
    """A run's strategy is drawn with probability proportional to its weight
    (Section 3.5.1; the paper's 8, 4, 2, 1, 0.1, 0, 0.01 as integers x100),
    except process 0's first run, which is Greedy.  One step per process, so
    each process's best record names its only run's strategy."""
    mat = synth.random_matrix(41, 12, 8, 2, 5, n_planted=3)
    n = 20000
    r = O.search([mat], synth.PAPER_WEIGHTS, n, 3, 1, 32, 400, 64, n_threads=8)
    bs = r.digests[0]["best_strategy"]
    assert bs[0] == O.G
    hist = np.bincount(bs[1:], minlength=O.N_STRATEGIES)
    w = np.array(synth.PAPER_WEIGHTS, float)
    assert hist[O.G] == 0                      # weight 0
    exp = (n - 1) * w / w.sum()
    live = w > 0
    chi2 = float(((hist[live] - exp[live]) ** 2 / exp[live]).sum())
    assert chi2 < 20.5  # 5 dof, p = 0.001


# ---------------------------------------------------------------- gi
def _gi_cases():
    a = b = None
    cases = []
    for ln in _lines("gi_example.txt"):
        f = ln.split()
        if f[0] == "a":
            a = int(f[1])
        elif f[0] == "b":
            b = int(f[1])
        elif f[0] == "case":
            cases.append([f[1], None, None])
        elif f[0] == "scores":
            cases[-1][1] = [int(x) for x in f[1:]]
        elif f[0] == "argmax":
            cases[-1][2] = int(f[1])
    return a, b, cases


def test_gi_hand_derived_scores():
    mat, *_ = _example()
    keys, counts = zip(*O.pairs(mat))
    a, b, cases = _gi_cases()
    m = len(keys)
    for name, scores, arg in cases:
        if name == "zeros":
            coins = np.zeros((m, m), np.uint8)
        elif name == "ones":
            coins = np.ones((m, m), np.uint8)
        else:
            coins = np.zeros((m, m), np.uint8)
            coins[2, :] = 1
        best, sc = O.gi_scores(keys, counts, a, b, coins)
        assert sc == scores, name
        assert best == arg, name


@pytest.mark.parametrize("seed", range(5))
def test_gi_with_alpha_zero_is_greedy(seed):
    mat = synth.random_matrix(400 + seed, 20, 9, 2, 5, n_planted=6)
    keys, counts = zip(*O.pairs(mat))
    m = len(keys)
    coins = np.random.default_rng(seed).integers(0, 2, (m, m)).astype(np.uint8)
    best, _ = O.gi_scores(keys, counts, 0, 50000, coins)
    assert best == O.select_basic(O.G, counts, [])


@pytest.mark.parametrize("seed", range(3))
def test_gi_score_structure(seed):
    """Disjoint candidates add alpha (c_q - 1) regardless of coins; a
    candidate sharing a variable adds alpha beta (c_q - 1) exactly when its
    coin is 1."""
    mat = synth.random_matrix(500 + seed, 18, 8, 2, 5, n_planted=5)
    keys, counts = zip(*O.pairs(mat))
    m = len(keys)
    a, b = 12345, 40000
    base = np.zeros((m, m), np.uint8)
    _, s0 = O.gi_scores(keys, counts, a, b, base)
    rng = np.random.default_rng(seed)
    for _ in range(5):
        p, q = rng.integers(0, m, 2)
        if p == q:
            continue
        flip = base.copy()
        flip[p, q] = 1
        _, s1 = O.gi_scores(keys, counts, a, b, flip)
        ip, jp, _ = O.unkey(keys[p])
        iq, jq, _ = O.unkey(keys[q])
        shares = len({ip, jp} & {iq, jq}) > 0
        delta = s1[p] - s0[p]
        assert delta == (a * b * (counts[q] - 1) if shares else 0)
        assert [x for t, x in enumerate(s1) if t != p] == [x for t, x in enumerate(s0) if t != p]
    # disjoint part: D_p = T - (c_p - 1) - sum over intersecting
    T = sum(c - 1 for c in counts)
    for p in range(m):
        ip, jp, _ = O.unkey(keys[p])
        inter = sum(counts[q] - 1 for q in range(m)
                    if q != p and ({ip, jp} & set(O.unkey(keys[q])[:2])))
        d = T - (counts[p] - 1) - inter
        assert s0[p] == ((counts[p] - 1) << 32) + a * (d << 16)


def _agree_half(a, b):
    """Two arrays of coins agree about half the time (5 sigma)."""
    a, b = np.asarray(a, float), np.asarray(b, float)
    n = a.size
    assert n > 1000
    assert abs((a == b).mean() - 0.5) < 5 * 0.5 / np.sqrt(n)


def test_gi_coins_are_fair_independent_bits():
    """Reading R9 (Section 3.4.2 fixes only that each intersecting term is
    kept with probability 1/2): exactly the intersecting pairs (q != p,
    sharing a variable) draw a coin; the coins are fair, and the coin of
    (p, q) is independent of (q, p), of another q of the same p (same Philox
    block), of the next step and of another process."""
    mat = synth.random_matrix(610, 18, 9, 2, 5, n_planted=5)
    keys, counts = zip(*O.pairs(mat))
    m = len(keys)
    var = [set(O.unkey(k)[:2]) for k in keys]
    inter = np.array([[p != q and bool(var[p] & var[q]) for q in range(m)] for p in range(m)])
    grid = {(pr, t): O.gi_philox_coins(keys, counts, 7, pr, t, 0) for pr in range(12) for t in range(12)}
    for c in grid.values():
        assert np.array_equal(c != 255, inter)
    allc = np.concatenate([c[inter] for c in grid.values()]).astype(float)
    assert abs(allc.mean() - 0.5) < 5 * 0.5 / np.sqrt(allc.size)
    pq = np.argwhere(inter)
    _agree_half(np.concatenate([c[pq[:, 0], pq[:, 1]] for c in grid.values()]),
                np.concatenate([c[pq[:, 1], pq[:, 0]] for c in grid.values()]))
    nxt = [(p, q, q2) for p in range(m) for q, q2 in zip(np.nonzero(inter[p])[0], np.nonzero(inter[p])[0][1:])]
    _agree_half(np.concatenate([[c[p, q] for p, q, _ in nxt] for c in grid.values()]),
                np.concatenate([[c[p, q2] for p, _, q2 in nxt] for c in grid.values()]))
    for dp, dt in ((0, 1), (1, 0)):
        a = np.concatenate([grid[(pr, t)][inter] for pr in range(11) for t in range(11)])
        b = np.concatenate([grid[(pr + dp, t + dt)][inter] for pr in range(11) for t in range(11)])
        _agree_half(a, b)


def test_shared_gi_coins_are_one_per_candidate():
    """Reading R9b (the shared-coin option): every p that intersects q sees
    the same coin of q, and those coins are fair across steps."""
    mat = synth.random_matrix(611, 18, 9, 2, 5, n_planted=5)
    keys, counts = zip(*O.pairs(mat))
    seen = []
    for t in range(300):
        c = O.gi_philox_coins(keys, counts, 7, 3, t, 0, shared=True)
        for q in range(len(keys)):
            col = c[:, q][c[:, q] != 255]
            if col.size:
                assert (col == col[0]).all()
                seen.append(col[0])
    seen = np.array(seen, float)
    assert abs(seen.mean() - 0.5) < 5 * 0.5 / np.sqrt(seen.size)


# ---------------------------------------------------------------- Greedy-Potential
def _gp_fixture():
    mat, gp, picks = [], [], {}
    sec = None
    for ln in _lines("gp_example.txt"):
        f = ln.split()
        if f[0] == "matrix":
            sec = "matrix"
        elif f[0] == "gp":
            gp.append(tuple(int(x) for x in f[1:]))
        elif f[0].startswith("pick_"):
            picks[f[0]] = tuple(int(x) for x in f[1:])
        elif sec == "matrix":
            mat.append([int(x) for x in f])
    return np.array(mat, np.int8), gp, picks


def _gp_pick(counts, pots, a):
    """argmax of (c - 1) 2^16 + a N, first in canonical order on ties."""
    sc = [((c - 1) << 16) + a * n for c, n in zip(counts, pots)]
    return sc.index(max(sc))


def test_gp_hand_derived_potentials():
    mat, gp, picks = _gp_fixture()
    cand = O.pairs(mat)
    assert [(*O.unkey(k), c) for k, c in cand] == [g[:4] for g in gp]
    assert O.gp_potentials(mat) == [g[4] for g in gp]
    counts = [c for _, c in cand]
    pots = [g[4] for g in gp]
    assert O.unkey(cand[_gp_pick(counts, pots, 1)][0]) == picks["pick_positive"]
    assert O.unkey(cand[_gp_pick(counts, pots, 32768)][0]) == picks["pick_positive"]
    assert O.unkey(cand[_gp_pick(counts, pots, 0)][0]) == picks["pick_zero"]
    # the oracle's own selection makes the hand-derived picks
    assert O.unkey(cand[O.gp_select(mat, 1)][0]) == picks["pick_positive"]
    assert O.unkey(cand[O.gp_select(mat, 32768)][0]) == picks["pick_positive"]
    assert O.unkey(cand[O.gp_select(mat, 0)][0]) == picks["pick_zero"]


@pytest.mark.parametrize("seed", range(6))
def test_gp_with_alpha_zero_is_greedy(seed):
    """alpha = 0 leaves only the (c - 1) term: Greedy-Potential picks what
    Greedy picks (highest c, lowest key)."""
    mat = synth.random_matrix(900 + seed, 14, 8, 2, 5, n_planted=3)
    counts = [c for _, c in O.pairs(mat)]
    assert O.gp_select(mat, 0) == O.select_basic(O.G, counts, [])


def _numpy_potential(mat, i, j, s):
    """Trial substitution and a from-scratch count of every signed pair of the
    new rows (all columns, not only the fresh one): the pairs that reach a
    count of 2 and did not have it before."""
    cur, _ = expand(mat, [O.entry(i, j, s)])

    def counts(m):
        c = {}
        for r in m:
            idx = np.nonzero(r)[0]
            for a, b in itertools.combinations(idx, 2):
                kk = (a, b, int(r[a] * r[b]))
                c[kk] = c.get(kk, 0) + 1
        return c

    before, after = counts(mat.astype(np.int64)), counts(cur)
    return sum(1 for kk, c in after.items() if c >= 2 and before.get(kk, 0) < 2)


@pytest.mark.parametrize("seed", range(4))
def test_gp_potential_counts_only_new_possibilities(seed):
    """No pair of old variables can gain occurrences, so the new possibilities
    are exactly the repeated pairs that contain the fresh variable."""
    mat = synth.random_matrix(700 + seed, 16, 8, 2, 5, n_planted=5)
    cand = O.pairs(mat)
    pots = O.gp_potentials(mat)
    assert len(pots) == len(cand) > 0
    for (k, _), n in zip(cand, pots):
        assert n == _numpy_potential(mat, *O.unkey(k))


def test_gp_search_reaches_optimum_on_the_paper_example():
    """Process 0 runs Greedy first; every other process runs Greedy-Potential
    (weights gp only), whose first pick on this matrix is x1 - x3 for any
    alpha > 0; both routes reach the exhaustive optimum 6."""
    mat, *_ = _example()
    r = O.search([mat], (0, 0, 0, 0, 0, 0, 1), 8, 3, 4, 64, 0, 16)
    assert r.cost == [6]
    assert (r.digests[0]["best_cost"] == 6).all()


@pytest.mark.parametrize("seed", range(3))
def test_gp_lists_are_valid_programs(seed):
    mats = [synth.random_matrix(900 + seed, 14, 9, 2, 5, n_planted=4)]
    r = O.search(mats, (0, 0, 0, 0, 0, 0, 1), 16, seed, 48, 8, 400, 48)
    m, lst, cost = mats[0], r.lists[0], r.cost[0]
    cur, back = expand(m, lst)
    assert np.array_equal(back, m.astype(np.int64))
    assert cost_of(cur, len(lst)) == cost
    assert cost >= O.bruteforce(m) if m.size <= 30 else cost <= O.naive(m)


# ---------------------------------------------------------------- iteration mode
def test_iteration_mode_closed_forms_on_the_example():
    """Greedy alone on the worked example: every run takes (x1 - x2), then
    (x3 - x4), and ends after 2 steps at Cost 6.  Without sharing each
    iteration costs 2 steps per process; the first iteration improves the
    total and the next `patience` do not, so the search stops after
    patience + 1 iterations.  With sharing at 100%, K = floor(3 * 2 / 4) = 1
    and every later run replays (x1 - x2) and needs a single step."""
    mat, *_ = _example()
    P, pat = 5, 4
    r = O.search_iterations([mat], (0, 0, 0, 0, 0, 1), P, 0, 100, pat, 0, 16)
    assert r.cost == [6] and r.iterations == pat + 1
    assert r.process_steps == 2 * P * (pat + 1)
    assert (r.digests[0]["runs"] == pat + 1).all() and (r.digests[0]["substeps"] == 2 * (pat + 1)).all()
    r = O.search_iterations([mat], (0, 0, 0, 0, 0, 1), P, 0, 100, pat, 1000, 16)
    assert r.iterations == pat + 1 and r.process_steps == P * (2 + pat)
    assert (r.digests[0]["substeps"] == 2 + pat).all()
    # patience 0: exactly the maximum number of iterations
    r = O.search_iterations([mat], (0, 0, 0, 0, 0, 1), P, 0, 7, 0, 0, 16)
    assert r.iterations == 7 and r.process_steps == 2 * P * 7


@pytest.mark.parametrize("seed", range(3))
def test_iteration_mode_stopping_rule(seed):
    """Stopped by patience p after I iterations: the last p iterations did not
    improve and iteration I - p did.  So a run capped at I - p iterations has
    the same costs (the lists may differ: a lower-numbered process can tie the
    best later), and one capped at I - p - 1 a strictly larger total."""
    mats = [synth.random_matrix(600 + seed, 16, 8, 2, 5, n_planted=5),
            synth.random_matrix(650 + seed, 8, 14, 2, 5, n_planted=3)]
    p = 3
    a = O.search_iterations(mats, synth.PAPER_WEIGHTS, 24, seed, 200, p, 400, 48)
    assert p < a.iterations < 200
    b = O.search_iterations(mats, synth.PAPER_WEIGHTS, 24, seed, a.iterations - p, 0, 400, 48)
    assert b.cost == a.cost
    c = O.search_iterations(mats, synth.PAPER_WEIGHTS, 24, seed, a.iterations - p - 1, 0, 400, 48)
    assert sum(c.cost) > sum(a.cost)
    for k, m in enumerate(mats):
        cur, back = expand(m, a.lists[k])
        assert np.array_equal(back, m.astype(np.int64)) and cost_of(cur, len(a.lists[k])) == a.cost[k]


# ---------------------------------------------------------------- Brent equations
@pytest.mark.parametrize("shape", [(2, 2, 2), (2, 3, 4), (3, 3, 3), (1, 5, 2)])
def test_brent_standard_algorithm_is_valid(shape):
    U, V, W = synth.standard_uvw(*shape)
    assert O.brent_violations(*shape, U, V, W) == 0


def test_brent_strassen_and_single_flips():
    """Strassen satisfies the Brent equations (Section 3.1).  Flipping one
    nonzero u_a of product l changes every sum that product l enters with
    that a, by 2 v_b w_c: exactly nnz(V[l]) * nnz(W[l]) equations break."""
    U, V, W = synth.strassen_uvw()
    assert O.brent_violations(2, 2, 2, U, V, W) == 0
    for l in range(7):
        for a in np.nonzero(U[l])[0]:
            U2 = U.copy()
            U2[l, a] = -U2[l, a]
            assert O.brent_violations(2, 2, 2, U2, V, W) == np.count_nonzero(V[l]) * np.count_nonzero(W[l])
    # a dropped product breaks the equations of its own (a, b, c) support
    assert O.brent_violations(2, 2, 2, U[1:], V[1:], W[1:]) == \
        np.count_nonzero(U[0]) * np.count_nonzero(V[0]) * np.count_nonzero(W[0])


@pytest.mark.parametrize("seed", range(3))
def test_brent_counts_match_numpy_tensor(seed):
    rng = np.random.default_rng(seed)
    m, n, p, r = 2, 3, 2, 9
    U, V, W = (rng.integers(-1, 2, (r, k)).astype(np.int8) for k in (m * n, n * p, m * p))
    T = np.einsum("la,lb,lc->abc", U.astype(int), V.astype(int), W.astype(int))
    ref = np.zeros_like(T)
    for i, j, k in itertools.product(range(m), range(n), range(p)):
        ref[i * n + j, j * p + k, i * p + k] = 1
    assert O.brent_violations(m, n, p, U, V, W) == int(np.count_nonzero(T != ref))


# ---------------------------------------------------------------- shared gi coins
def _fnv(words):
    h = 0xCBF29CE484222325
    for w in words:
        h = ((h ^ (w & 0xFFFFFFFF)) * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


def _draw4(seed, proc, t, mat, purpose, extra_hi=0, extra_lo=0):
    return O.philox([proc, t, (mat & 0xFF) << 24 | (purpose & 0xF) << 20 | (extra_hi & 0xFFFFF), extra_lo],
                    [seed & 0xFFFFFFFF, seed >> 32])


@pytest.mark.parametrize("seed", range(4))
def test_shared_coin_first_pick_from_the_stated_draws(seed):
    """Greedy-Intersections with shared coins, rebuilt from Philox (pinned by
    its known answers) and the readings: the run draw gives alpha and beta,
    each candidate q gets the coin at bit q & 31 of word (q >> 5) & 3 of the
    purpose-4 draw for block q >> 7, and the first substitution of process 1
    is the argmax of the scores with those coins (identical for every p)."""
    mat = synth.random_matrix(800 + seed, 60, 14, 3, 7, n_planted=12)   # m ~ 180: two 128-blocks
    keys, counts = zip(*O.pairs(mat))
    m = len(keys)
    run = _draw4(seed, 1, 0, 0, 0)
    a = (run[1] * 32769) >> 32
    b = 32768 + ((run[2] * 32769) >> 32)
    coins = np.array([(_draw4(seed, 1, 0, 0, 4, q >> 7)[(q >> 5) & 3] >> (q & 31)) & 1 for q in range(m)], np.uint8)
    best, _ = O.gi_scores(keys, counts, a, b, np.tile(coins, (m, 1)))
    i, j, s = O.unkey(keys[best])
    r = O.search([mat], synth.GI_ONLY, 2, seed, 1, 8, 0, 32, flags=O.GI_SHARED_COINS)
    assert r.digests[0]["best_hash"][1] == _fnv([O.entry(i, j, s)])
    assert r.digests[0]["best_len"][1] == 1


@pytest.mark.parametrize("seed", range(3))
def test_shared_coin_scores_from_per_variable_sums(seed):
    """With one coin per candidate, X_p = X_i + X_j - 2 coin_p w_p - coin_t w_t
    (t the sign twin) where X_v sums coin_q w_q over the candidates holding
    x_v; the same holds for the plain sums.  Checked against the direct
    O(m^2) scores."""
    mat = synth.random_matrix(900 + seed, 24, 10, 2, 5, n_planted=7)
    keys, counts = zip(*O.pairs(mat))
    m = len(keys)
    rng = np.random.default_rng(seed)
    coins = rng.integers(0, 2, m).astype(np.int64)
    a, b = 20000, 40000
    _, sc = O.gi_scores(keys, counts, a, b, np.tile(coins.astype(np.uint8), (m, 1)))
    w = np.array(counts, np.int64) - 1
    ij = [O.unkey(k)[:2] for k in keys]
    nv = 1 + max(max(x) for x in ij)
    G = np.zeros(nv, np.int64)
    X = np.zeros(nv, np.int64)
    for (i, j), wq, cq in zip(ij, w, coins):
        G[i] += wq
        G[j] += wq
        X[i] += cq * wq
        X[j] += cq * wq
    T = int(w.sum())
    for p, (i, j) in enumerate(ij):
        tw = [q for q in range(m) if q != p and ij[q] == (i, j)]
        wt = int(w[tw[0]]) if tw else 0
        ct = int(coins[tw[0]]) if tw else 0
        inter = G[i] + G[j] - 2 * w[p] - wt
        x = X[i] + X[j] - 2 * coins[p] * w[p] - ct * wt
        d = T - w[p] - inter
        assert sc[p] == (int(w[p]) << 32) + a * ((int(d) << 16) + b * int(x))


# ---------------------------------------------------------------- metrics
@pytest.mark.parametrize("seed", range(3))
def test_curve_and_winning_strategies(seed):
    """The best-Cost curve never rises, has one point per round and ends at
    the result; a process's best record names the strategy of its run: with
    Greedy alone every improving process names g (5), and the per-strategy
    win counts over processes add up to the processes that improved."""
    mats = [synth.random_matrix(1100 + seed, 18, 9, 2, 5, n_planted=5)]
    r = O.search(mats, synth.PAPER_WEIGHTS, 40, seed, 100, 16, 400, 48)
    c = r.curve[0]
    assert len(c) == 7 and c[-1] == r.cost[0] and all(a >= b for a, b in zip(c, c[1:]))
    d = r.digests[0]
    improved = d["best_cost"] < O.naive(mats[0])
    assert ((d["best_strategy"] >= 0) == improved).all()
    assert np.bincount(d["best_strategy"][improved], minlength=7).sum() == improved.sum()
    g = O.search(mats, (0, 0, 0, 0, 0, 1), 12, seed, 40, 16, 400, 48).digests[0]["best_strategy"]
    assert set(g.tolist()) <= {5, -1}
    it = O.search_iterations(mats, synth.PAPER_WEIGHTS, 20, seed, 30, 3, 400, 48)
    assert len(it.curve[0]) == it.iterations and it.curve[0][-1] == it.cost[0]


def test_config4_golden_is_of_the_current_inputs():
    """tests/golden/cfg4_reduced.txt (the oracle's results that the GPU parity
    test compares with) was written for the inputs synth.config4 generates
    now, and holds every process of every matrix."""
    import hashlib
    g = {}
    n_p = 0
    for ln in open(os.path.join(GOLD, "cfg4_reduced.txt")):
        f = ln.split()
        if f and f[0] in ("inputs_sha256", "params", "costs"):
            g[f[0]] = f[1:]
        n_p += bool(f) and f[0] == "p"
    n_proc, budget = int(g["params"][0]), int(g["params"][1])
    s = synth.config4(n_proc=n_proc, budget=budget)
    h = hashlib.sha256()
    for m in s.mats:
        h.update(m.tobytes())
    assert g["inputs_sha256"][0] == h.hexdigest()[:16]
    assert n_p == 3 * n_proc and len(g["costs"]) == 3
    # the results are valid programs for these inputs
    for k, ln in enumerate(l for l in open(os.path.join(GOLD, "cfg4_reduced.txt")) if l.startswith("list ")):
        lst = [int(x) for x in ln.split()[2:]]
        assert O.apply(s.mats[k], lst)[1] == int(g["costs"][k])
