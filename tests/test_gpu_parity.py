"""Parity of the CUDA search (through the C ABI) with the CPU oracle.

The method draws all its randomness from Philox keyed by (seed, process,
step), so the bar is bit-exactness: every process's trajectory hash, best
record, run count, op count and the per-matrix results must be identical.
"""
import numpy as np
import pytest

from oracle import oracle as O
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


def assert_parity(cse, s, ref=None, procs_per_cta=0, check_procs=True, gi_shared=False, **kw):
    r = cse.search_obj(s, procs_per_cta=procs_per_cta, trace=True, gi_shared=gi_shared, **kw)
    if ref is None:
        ref = O.search_obj(s, n_threads=8, flags=O.GI_SHARED_COINS if gi_shared else 0)
    assert r.costs == ref.cost
    assert r.lists == ref.lists
    if check_procs:
        for k in range(len(s.mats)):
            got, exp = r.procs(k), ref.digests[k]
            for f in FIELDS:
                bad = np.nonzero(got[f] != exp[f])[0]
                assert bad.size == 0, f"matrix {k} field {f}: {bad.size} processes differ, first {bad[:5]}"
    steps, sub, ops = r.counters()
    assert steps == len(s.mats) * s.n_proc * s.budget
    if check_procs:
        assert [r.curve(k) for k in range(len(s.mats))] == ref.curve
    assert sub == int(sum(ref.digests[k]["substeps"].sum() for k in range(len(s.mats))))
    assert ops == int(sum(ref.digests[k]["ops"].sum() for k in range(len(s.mats))))
    assert r.method_ops() == int(sum(ref.digests[k]["method_ops"].sum() for k in range(len(s.mats))))
    r.free()
    return ref


def load_cfg4_golden():
    """The oracle's results for the (6,6,6:153)-shaped workload at 512
    processes x 200 steps (tests/golden/cfg4_reduced.txt, written by
    tests/golden/make_cfg4_golden.py from the oracle alone)."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cfg4_reduced.txt")
    g = {"lists": {}, "curves": {}, "procs": {}}
    for ln in open(path):
        f = ln.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "inputs_sha256":
            g["sha"] = f[1]
        elif f[0] == "params":
            g["params"] = [int(x) for x in f[1:]]
        elif f[0] == "costs":
            g["costs"] = [int(x) for x in f[1:]]
        elif f[0] == "list":
            g["lists"][int(f[1])] = [int(x) for x in f[2:]]
        elif f[0] == "curve":
            g["curves"][int(f[1])] = [int(x) for x in f[2:]]
        elif f[0] == "p":
            vals = [int(x, 16) if name.endswith("hash") else int(x) for name, x in zip(FIELDS_CFG4, f[3:])]
            g["procs"].setdefault(int(f[1]), []).append(vals)
    return g


FIELDS_CFG4 = ("best_cost", "best_len", "runs", "best_hash", "traj_hash", "ops", "substeps", "best_strategy",
               "method_ops")


@pytest.mark.parametrize("engine", ["cta", "warp", "cta_small_lists"])
def test_config4_reduced_scale_full_parity(cse, engine):
    """The (6,6,6:153)-shaped workload at 512 processes x 200 steps, sharing
    every 32 steps (six sharing boundaries), cap 512: every process's record,
    the lists, Costs and best-Cost curves equal the oracle's.  Both large-matrix
    engines run it: one process per CTA (with its list capacity forced down to
    2048, so that processes outgrow it and finish their rounds on the warp
    engine) and one warp per process."""
    g = load_cfg4_golden()
    n_proc, budget, interval, permille, cap, seed = g["params"]
    s = synth.config4(n_proc=n_proc, budget=budget)
    assert (s.interval, s.permille, s.cap, s.seed) == (interval, permille, cap, seed)
    kw = {"warp": {}, "cta": {"cta_engine": True},
          "cta_small_lists": {"cta_engine": True, "cta_list_cap": 2048}}[engine]
    r = cse.search_obj(s, trace=True, **kw)
    assert r.costs == g["costs"]
    assert r.lists == [g["lists"][k] for k in range(3)]
    assert [r.curve(k) for k in range(3)] == [g["curves"][k] for k in range(3)]
    for k in range(3):
        got = r.procs(k)
        exp = np.array(g["procs"][k], dtype=object)
        for fi, f in enumerate(FIELDS_CFG4):
            want = np.array([int(x) for x in exp[:, fi]], dtype=got[f].dtype)
            bad = np.nonzero(got[f] != want)[0]
            assert bad.size == 0, f"{engine}: matrix {k} field {f}: {bad.size} processes differ, first {bad[:5]}"
    steps, sub, ops = r.counters()
    assert steps == 3 * n_proc * budget
    assert sub == sum(int(v[6]) for k in range(3) for v in g["procs"][k])
    assert ops == sum(int(v[5]) for k in range(3) for v in g["procs"][k])
    assert r.method_ops() == sum(int(v[8]) for k in range(3) for v in g["procs"][k])
    r.free()


def test_config1_full(cse):
    assert_parity(cse, synth.config1())


@pytest.mark.parametrize("ppc", [1, 2, 3, 4])
def test_config2_reduced_any_launch_shape(cse, ppc):
    s = synth.config2(n_proc=192, budget=160)
    assert_parity(cse, s, procs_per_cta=ppc)


@pytest.mark.parametrize("rows", [20, 33, 64, 65, 100, 130, 161, 200, 256])
def test_word_widths(cse, rows):
    # W = ceil(rows / 32) from 1 to 8; ragged process count
    mats = [synth.random_matrix(rows, rows, 10, 2, 6, n_planted=5),
            synth.random_matrix(rows + 1, 12, min(rows, 40), 2, 5, n_planted=3)]
    s = synth.Search(f"w{rows}", mats, synth.PAPER_WEIGHTS, 37, 11, 70, 16, 400, 128)
    assert_parity(cse, s)


@pytest.mark.parametrize("rows", [70, 100, 130, 161, 200])
def test_wide_words_equal_the_oracle(cse, rows):
    """CSE_FLAG_WIDE_WORDS runs matrices of 3, 5, 6 and 7 words per column
    on the 4- and 8-word kernels (zero row bits above the matrix's own): every
    result, op counts included, stays the oracle's."""
    mats = [synth.random_matrix(rows, rows, 10, 2, 6, n_planted=5),
            synth.random_matrix(rows + 1, 12, min(rows, 40), 2, 5, n_planted=3)]
    s = synth.Search(f"wide{rows}", mats, synth.PAPER_WEIGHTS, 37, 11, 70, 16, 400, 128)
    assert_parity(cse, s, wide_words=True)


@pytest.mark.parametrize("cta_engine", [False, True])
def test_wide_words_from_hbm(cse, cta_engine):
    """The (6,6,6:153) shape's 5-word matrices on the 8-word HBM-path
    kernels, alone or with the process-per-CTA engine."""
    s = synth.config4(n_proc=24, budget=48)
    s.interval = 16
    assert_parity(cse, s, wide_words=True, cta_engine=cta_engine)


@pytest.mark.parametrize("weights", [synth.GI_ONLY, (0, 1, 0, 0, 0, 0), (0, 0, 1, 0, 0, 0), (0, 0, 0, 1, 0, 0),
                                     (0, 0, 0, 0, 1, 0), (0, 0, 0, 0, 0, 1), synth.GP_ONLY, synth.PAPER_WEIGHTS,
                                     synth.PAPER_WEIGHTS_NO_GP])
def test_each_strategy(cse, weights):
    s = synth.config2(n_proc=64, budget=96)
    s.weights = weights
    assert_parity(cse, s)


@pytest.mark.parametrize("interval,permille", [(1, 400), (7, 1000), (32, 0), (1000, 400)])
def test_sharing_settings(cse, interval, permille):
    s = synth.config2(n_proc=48, budget=100)
    s.interval, s.permille = interval, permille
    assert_parity(cse, s)


@pytest.mark.parametrize("budget", [0, 1, 2, 33])
def test_small_budgets(cse, budget):
    s = synth.config2(n_proc=20, budget=budget)
    assert_parity(cse, s)


def test_column_cap_termination(cse):
    mats = [synth.random_matrix(5, 30, 9, 3, 7, n_planted=6, frac=(0.4, 0.7))]
    for cap in (10, 11, 14):
        s = synth.Search("cap", mats, synth.PAPER_WEIGHTS, 40, 3, 60, 8, 400, cap)
        ref = assert_parity(cse, s)
        assert max(ref.length) <= cap - 9


def test_no_candidates_strassen(cse):
    U, V, W = synth.strassen_uvw()
    sc = cse.Scheme.from_uvw(2, 2, 2, U, V, W)
    r = cse.search(sc, synth.PAPER_WEIGHTS, 16, 0, 40, 8, 400, 32)
    assert r.total == 18 and r.costs == [5, 5, 8] and r.lists == [[], [], []]
    assert sc.shape(2) == (4, 7)


def test_paper_example(cse):
    mat = np.array([[1, 1, -1, 1], [1, -1, 0, -1], [1, -1, -1, 1]], np.int8)
    s = synth.Search("example", [mat], (0, 0, 0, 0, 0, 1), 1, 0, 2, 64, 0, 16)
    ref = assert_parity(cse, s)
    assert ref.cost == [6]


def test_single_row_and_single_process(cse):
    mats = [np.array([[1, -1, 1, 1, -1]], np.int8), synth.random_matrix(9, 6, 5, 2, 4)]
    s = synth.Search("tiny", mats, synth.PAPER_WEIGHTS, 1, 5, 30, 4, 1000, 16)
    assert_parity(cse, s)


def test_seeds_differ(cse):
    s = synth.config2(n_proc=32, budget=64)
    a = cse.search_obj(s, trace=True)
    s.seed = 1
    b = cse.search_obj(s, trace=True)
    assert not np.array_equal(a.procs(0)["traj_hash"], b.procs(0)["traj_hash"])


def test_invalid_search_arguments(cse):
    s = synth.config1()
    sc = cse.Scheme(s.mats)
    with pytest.raises(cse.CseError):
        cse.search(sc, (0,) * 6, 4, 0, 10)                    # all weights zero
    with pytest.raises(cse.CseError):
        cse.search(sc, (0xFFFFFFFF, 0, 0, 0, 0, 0, 1), 4, 0, 10)  # weight sum above 32 bits
    with pytest.raises(cse.CseError):
        cse.search(sc, synth.GI_ONLY, 4, 0, 10, cap=7)         # cap <= cols
    with pytest.raises(cse.CseError):
        cse.search(sc, synth.GI_ONLY, 0, 0, 10)                # no processes
    with pytest.raises(cse.CseError):
        cse.search(sc, synth.GI_ONLY, 4, 0, 10, interval=32, patience=3)   # patience needs iteration mode
    with pytest.raises(cse.CseError):
        cse.search(sc, synth.GI_ONLY, 4, 0, 10, interval=0, graph=True)    # iteration mode has no graph


def test_config2_full_size(cse):
    """The benchmark workload at full size (4096 processes x 3 matrices x 1024
    steps) in the benchmark's launch configuration, against the full oracle."""
    s = synth.config2()
    assert_parity(cse, s)


def assert_valid_program(m, lst, cost):
    """lst is a program for m: its rewritten rows have the reported Cost, and
    expanding every fresh variable (numpy) reproduces m exactly."""
    out, c2 = O.apply(m, lst)
    assert c2 == cost
    nx = m.shape[1]
    defs = [np.eye(nx, dtype=np.int64)[v] for v in range(nx)]
    for e in lst:
        i, j, sg = O.unentry(e)
        assert 0 <= i < j < len(defs) and sg in (1, -1)
        defs.append(defs[i] + sg * defs[j])
    assert np.array_equal(out.astype(np.int64) @ np.stack(defs), m.astype(np.int64))


def test_results_are_valid_programs(cse):
    s = synth.config2(n_proc=256, budget=256)
    r = cse.search_obj(s)
    for k, m in enumerate(s.mats):
        lst, cost, _ = r.fetch(k)
        assert_valid_program(m, lst, cost)


@pytest.mark.parametrize("cta_engine", [False, True])
def test_large_matrices_run_from_hbm(cse, cta_engine):
    """(6,6,6:153)-shaped matrices (153 x 36 with W = 5 words per column and
    36 x 153 with 153 original columns), columns grown towards 512: their
    per-process arrays exceed a shared-memory slice, so the engine works on
    the HBM state region (and, with the CTA engine, in a CTA's shared memory
    for run starts and long lists).  Reduced process count and budget."""
    s = synth.config4(n_proc=24, budget=48)
    s.interval = 16
    assert_parity(cse, s, cta_engine=cta_engine)


@pytest.mark.parametrize("rows", [20, 64, 130, 256])
def test_greedy_potential_word_widths(cse, rows):
    # trial columns of W = 1, 2, 5 and 8 words; Greedy-Potential in every run
    mats = [synth.random_matrix(rows + 5, rows, 10, 2, 5, n_planted=6),
            synth.random_matrix(rows + 6, 14, min(rows, 40), 2, 5, n_planted=3)]
    s = synth.Search(f"gp{rows}", mats, synth.GP_ONLY, 21, 4, 40, 16, 400, 96)
    assert_parity(cse, s)


def test_greedy_potential_from_hbm(cse):
    s = synth.config4(n_proc=6, budget=12)
    s.weights, s.interval = (0, 0, 0, 0, 0, 1, 3), 8
    assert_parity(cse, s)


def test_mid_size_both_paths(cse):
    # the same search through shared memory (cap 64) and through HBM (cap 512)
    mats = [synth.random_matrix(77, 60, 14, 3, 7, n_planted=8)]
    for cap in (64, 512):
        s = synth.Search("mid", mats, synth.PAPER_WEIGHTS, 40, 2, 80, 16, 400, cap)
        assert_parity(cse, s)


def _records(cse, r, n_mats):
    return [r.procs(k) for k in range(n_mats)], r.lists, r.costs


@pytest.mark.parametrize("graph", [False, True])
def test_batch_equals_each_search_alone(cse, graph):
    """Uneven schemes (different shapes, W classes, process counts and budgets)
    in one launch sequence give exactly the results of separate searches."""
    searches = synth.config3(n_schemes=6, n_proc=40, budget=70, interval=16)
    searches[1].n_proc, searches[2].budget, searches[3].seed = 23, 33, 99
    searches.append(synth.config2(n_proc=30, budget=50))
    searches[-1].interval, searches[-1].cap = 16, 256
    batch = cse.search_batch_obj(searches, graph=graph, trace=True)
    kernels, shared = batch[0].launches()
    assert shared == len(searches) and kernels >= 1 + 5  # init + rounds x (groups + share)
    for s, rb in zip(searches, batch):
        alone = cse.search_obj(s, trace=True)
        pb, lb, cb = _records(cse, rb, len(s.mats))
        pa, la, ca = _records(cse, alone, len(s.mats))
        assert lb == la and cb == ca
        for x, y in zip(pb, pa):
            assert np.array_equal(x, y)
    # and against the oracle for two of them
    for idx in (0, len(searches) - 1):
        ref = O.search_obj(searches[idx], n_threads=8)
        assert batch[idx].costs == ref.cost and batch[idx].lists == ref.lists
        for k in range(len(searches[idx].mats)):
            got, exp = batch[idx].procs(k), ref.digests[k]
            for f in FIELDS:
                assert np.array_equal(got[f], exp[f]), f
    for r in batch:
        r.free()


@pytest.mark.parametrize("graph", [False, True])
def test_persistent_batch_equals_each_search_alone(cse, graph):
    """The whole batch as one persistent cooperative kernel (CSE_FLAG_PERSISTENT;
    in a CUDA graph or launched directly): schemes of both word widths,
    uneven process counts and budgets, exactly the results of separate
    searches, and of the oracle for two of them."""
    searches = synth.config3(n_schemes=6, n_proc=40, budget=70, interval=16)
    searches[1].n_proc, searches[2].budget, searches[3].seed = 23, 33, 99
    batch = cse.search_batch_obj(searches, graph=graph, trace=True, persistent=True)
    assert batch[0].launches()[0] == 1
    for s, rb in zip(searches, batch):
        alone = cse.search_obj(s, trace=True)
        pb, lb, cb = _records(cse, rb, len(s.mats))
        pa, la, ca = _records(cse, alone, len(s.mats))
        assert lb == la and cb == ca
        for x, y in zip(pb, pa):
            assert np.array_equal(x, y)
        assert rb.counters() == alone.counters() and rb.method_ops() == alone.method_ops()
    for idx in (0, 2):
        ref = O.search_obj(searches[idx], n_threads=8)
        assert batch[idx].costs == ref.cost and batch[idx].lists == ref.lists
    for r in batch:
        r.free()


def test_persistent_batch_barrier_time_out(cse):
    """A grid barrier that gives up (a poll limit far too small for the CTAs
    to meet) makes every CTA return; the search reports CSE_ETIMEOUT and the
    device stays usable."""
    searches = synth.config3(n_schemes=3, n_proc=512, budget=64, interval=16)
    batch = cse.search_batch_obj(searches, graph=False, persistent=True, max_spin=1)
    with pytest.raises(cse.CseError) as e:
        batch[0].costs
    assert e.value.code == cse.CSE_ETIMEOUT
    for r in batch:
        r.free()
    s = synth.config1(n_proc=16, budget=16)
    ref = O.search_obj(s)
    assert cse.search_obj(s).costs == ref.cost


def test_persistent_batch_refuses_large_matrices(cse):
    s = synth.config4(n_proc=4, budget=8)
    with pytest.raises(cse.CseError) as e:
        cse.search_batch_obj([s], persistent=True)
    assert e.value.code == cse.CSE_EINVAL


def test_graph_single_search(cse):
    s = synth.config2(n_proc=64, budget=96)
    r = cse.search(cse.Scheme(s.mats), s.weights, s.n_proc, s.seed, s.budget, s.interval, s.permille, s.cap,
                   graph=True)
    ref = O.search_obj(s, n_threads=8)
    assert r.costs == ref.cost and r.lists == ref.lists


def test_autotuner_changes_speed_not_results(cse):
    searches = synth.config3(n_schemes=4, n_proc=64, budget=64, interval=16)
    schemes = [cse.Scheme(s.mats) for s in searches]
    args = (schemes, [s.weights for s in searches], [s.n_proc for s in searches], [s.seed for s in searches],
            [s.budget for s in searches])
    before = cse.search_batch(*args, interval=16, cap=256, trace=True)
    ents = cse.autotune(*args, interval=16, cap=256, trial_steps=32)
    assert ents and all(1 <= e["procs_per_cta"] <= 4 and min(e["trial_ms"]) > 0 for e in ents)
    after = cse.search_batch(*args, interval=16, cap=256, trace=True)
    for a, b, s in zip(before, after, searches):
        assert a.lists == b.lists and a.costs == b.costs
        for k in range(len(s.mats)):
            assert np.array_equal(a.procs(k), b.procs(k))


def test_autotuner_times_the_wider_kernel(cse):
    """Classes of 3 words per column are timed on the 4-word kernel too; the
    width it keeps is reported, and searches after it still give the
    oracle's results (the width never changes them)."""
    searches = [synth.Search(f"tw{i}", [synth.random_matrix(i, 70 + i, 12, 2, 5, n_planted=3),
                                        synth.random_matrix(10 + i, 40, 20, 2, 5, n_planted=2)],
                             synth.PAPER_WEIGHTS, 48, i, 32, 16, 400, 128) for i in range(3)]
    schemes = [cse.Scheme(s.mats) for s in searches]
    args = (schemes, [s.weights for s in searches], [s.n_proc for s in searches], [s.seed for s in searches],
            [s.budget for s in searches])
    ents = cse.autotune(*args, interval=16, cap=128, trial_steps=16)
    three = [e for e in ents if e["words_per_column"] == 3]
    assert three and all(e["kernel_words"] in (3, 4) and min(e["trial_ms_wide"]) > 0 for e in three)
    assert all(e["kernel_words"] == e["words_per_column"] and max(e["trial_ms_wide"]) < 0
               for e in ents if e["words_per_column"] in (1, 2, 4, 8))
    for s, sc in zip(searches, schemes):
        assert_parity(cse, s)


def test_interval_tuner_picks_lowest_total(cse):
    searches = synth.config3(n_schemes=3, n_proc=48, budget=96, interval=16)
    schemes = [cse.Scheme(s.mats) for s in searches]
    args = (schemes, [s.weights for s in searches], [s.n_proc for s in searches], [s.seed for s in searches],
            [s.budget for s in searches])
    best, total = cse.tune_interval(*args, candidates=(8, 16, 48), cap=256, trial_steps=96)
    totals = {}
    for iv in (8, 16, 48):
        rs = cse.search_batch(*args, interval=iv, cap=256)
        totals[iv] = sum(r.total for r in rs)
    assert total == totals[best] == min(totals.values())
    assert best == [8, 16, 48][[totals[8], totals[16], totals[48]].index(min(totals.values()))]


def test_large_search_full_process_count_sampled(cse):
    """(6,6,6:153)-shaped search at its full 65536 processes per matrix, up to
    the first sharing boundary (32 steps): no snapshot exists yet, so every
    process is independent and the oracle can replay a sample of them exactly."""
    s = synth.config4(budget=32)
    r = cse.search_obj(s, trace=True)
    sample = [0, 1, 777, 4095, 31337, 65535]
    ref = O.search_obj(s, n_threads=8, subset=sample)
    for k in range(3):
        got, exp = r.procs(k)[sample], ref.digests[k][sample]
        for f in FIELDS:
            assert np.array_equal(got[f], exp[f]), (k, f)
    # the published result is the best over all processes: never worse than the sample
    assert all(c <= int(ref.digests[k][sample]["best_cost"].min()) for k, c in enumerate(r.costs))
    r.free()


def test_config4_full_size_properties(cse):
    """The (6,6,6:153)-shaped search at full size: 65536 processes x 3
    matrices x 2000 steps, in the launch configuration the benchmark uses.
    Its processes interact at every sharing boundary, so no sample of them
    can be replayed past the first one; this checks what holds at any size.
    Each result is a valid program whose Cost is recomputed from its rows and
    is below A_naive; the best-Cost curve never rises and ends at the result;
    the result is the lowest per-process record; every process ran every
    step, and the substitution count is the sum of the processes' counts."""
    s = synth.config4()
    r = cse.search_obj(s)
    steps, sub, _ = r.counters()
    assert steps == len(s.mats) * s.n_proc * s.budget
    n_sub = 0
    for k, m in enumerate(s.mats):
        lst, cost, _ = r.fetch(k)
        assert_valid_program(m, lst, cost)
        assert cost < O.apply(m, [])[1]
        curve = r.curve(k)
        assert len(curve) == -(-s.budget // s.interval)
        assert all(a >= b for a, b in zip(curve, curve[1:])) and curve[-1] == cost
        p = r.procs(k)
        assert int(p["best_cost"].min()) == cost
        assert (p["best_len"] <= s.cap - m.shape[1]).all() and (p["runs"] >= 1).all()
        assert (p["substeps"] <= s.budget).all()
        n_sub += int(p["substeps"].sum())
    assert sub == n_sub
    r.free()


def test_config4_full_process_count_any_launch_shape(cse):
    """65536 processes per matrix of the (6,6,6:153) shape over 8 sharing
    rounds: one process per CTA and the default four give identical
    processes, lists and curves (launch parameters never change results)."""
    s = synth.config4(budget=256)
    a = cse.search_obj(s, procs_per_cta=1, trace=True)
    b = cse.search_obj(s, trace=True)
    assert a.costs == b.costs and a.lists == b.lists
    for k in range(len(s.mats)):
        pa, pb = a.procs(k), b.procs(k)
        for f in FIELDS:
            assert np.array_equal(pa[f], pb[f]), (k, f)
        assert a.curve(k) == b.curve(k)
    assert a.counters() == b.counters()
    a.free()
    b.free()


def test_trace_flag_only_changes_the_trajectory_record(cse):
    s = synth.config2(n_proc=64, budget=80)
    plain = cse.search_obj(s)
    traced = cse.search_obj(s, trace=True)
    assert plain.lists == traced.lists and plain.costs == traced.costs
    for k in range(3):
        a, b = plain.procs(k), traced.procs(k)
        assert (a["traj_hash"] == 0xCBF29CE484222325).all()
        for f in ("best_cost", "best_len", "runs", "best_hash", "ops", "substeps", "method_ops"):
            assert np.array_equal(a[f], b[f])


# ---------------------------------------------------------------- iteration mode
def assert_parity_iterations(cse, s, patience, ref=None, r=None, gi_shared=False):
    """Iteration mode (share_interval = 0): s.budget is the maximum number of
    iterations."""
    if r is None:
        r = cse.search_obj(s, patience=patience, trace=True, gi_shared=gi_shared)
    if ref is None:
        ref = O.search_iterations(s.mats, s.weights, s.n_proc, s.seed, s.budget, patience, s.permille, s.cap,
                                  n_threads=8, flags=O.GI_SHARED_COINS if gi_shared else 0)
    assert r.costs == ref.cost
    assert r.lists == ref.lists
    for k in range(len(s.mats)):
        got, exp = r.procs(k), ref.digests[k]
        for f in FIELDS:
            bad = np.nonzero(got[f] != exp[f])[0]
            assert bad.size == 0, f"matrix {k} field {f}: {bad.size} processes differ, first {bad[:5]}"
    steps, sub, ops = r.counters()
    assert steps == ref.process_steps
    assert sub == int(sum(ref.digests[k]["substeps"].sum() for k in range(len(s.mats))))
    assert ops == int(sum(ref.digests[k]["ops"].sum() for k in range(len(s.mats))))
    it, conv, total = r.iterations()
    assert it == ref.iterations and total == sum(ref.cost)
    assert [r.curve(k) for k in range(len(s.mats))] == ref.curve
    assert conv == (ref.iterations < s.budget)
    r.free()
    return ref


def test_iteration_mode_paper_example(cse):
    mat = np.array([[1, 1, -1, 1], [1, -1, 0, -1], [1, -1, -1, 1]], np.int8)
    for permille in (0, 1000):
        s = synth.Search("example", [mat], (0, 0, 0, 0, 0, 1), 5, 0, 100, 0, permille, 16)
        ref = assert_parity_iterations(cse, s, 4)
        assert ref.iterations == 5 and ref.cost == [6]


@pytest.mark.parametrize("patience,max_it", [(4, 60), (0, 9), (10, 200)])
def test_iteration_mode_config2_reduced(cse, patience, max_it):
    s = synth.config2(n_proc=128, budget=max_it)
    s.interval = 0
    assert_parity_iterations(cse, s, patience)


@pytest.mark.parametrize("rows", [20, 100, 256])
def test_iteration_mode_word_widths(cse, rows):
    mats = [synth.random_matrix(rows + 11, rows, 10, 2, 5, n_planted=6),
            synth.random_matrix(rows + 12, 12, min(rows, 40), 2, 5, n_planted=3)]
    s = synth.Search(f"it{rows}", mats, synth.PAPER_WEIGHTS, 33, 8, 30, 0, 400, 96)
    assert_parity_iterations(cse, s, 3)


def test_iteration_mode_from_hbm(cse):
    s = synth.config4(n_proc=4, budget=2)
    s.interval = 0
    assert_parity_iterations(cse, s, 0)


def test_iteration_mode_batch_equals_alone(cse):
    ss = [synth.config2(n_proc=64, budget=40), synth.config1(n_proc=40, budget=40)]
    for k, s in enumerate(ss):
        s.interval, s.seed, s.cap = 0, 3 + k, 128
    scs = [cse.Scheme(s.mats) for s in ss]
    rs = cse.search_batch(scs, [s.weights for s in ss], [s.n_proc for s in ss], [s.seed for s in ss],
                          [s.budget for s in ss], interval=0, permille=400, cap=128, graph=False, trace=True,
                          patience=5)
    for s, r in zip(ss, rs):
        assert_parity_iterations(cse, s, 5, r=r)


# ---------------------------------------------------------------- shared gi coins
@pytest.mark.parametrize("weights", [synth.GI_ONLY, synth.PAPER_WEIGHTS, (0, 0, 0, 0, 1, 0)])
def test_shared_coins_config2_reduced(cse, weights):
    s = synth.config2(n_proc=160, budget=120)
    s.weights = weights
    assert_parity(cse, s, gi_shared=True)


@pytest.mark.parametrize("rows", [20, 64, 130, 256])
def test_shared_coins_word_widths(cse, rows):
    # m up to several hundred candidates: several 128-candidate coin blocks
    mats = [synth.random_matrix(rows + 21, rows, 12, 3, 7, n_planted=10),
            synth.random_matrix(rows + 22, 16, min(rows, 48), 3, 7, n_planted=5)]
    s = synth.Search(f"gs{rows}", mats, synth.GI_ONLY, 29, 6, 48, 16, 400, 128)
    assert_parity(cse, s, gi_shared=True)


def test_shared_coins_from_hbm(cse):
    s = synth.config4(n_proc=16, budget=24)
    s.interval = 8
    assert_parity(cse, s, gi_shared=True)


def test_shared_coins_iteration_mode(cse):
    s = synth.config2(n_proc=96, budget=40)
    s.interval = 0
    assert_parity_iterations(cse, s, 4, gi_shared=True)


def test_shared_coins_change_results(cse):
    s = synth.config2(n_proc=64, budget=64)
    s.weights = synth.GI_ONLY
    a = cse.search_obj(s, trace=True)
    b = cse.search_obj(s, trace=True, gi_shared=True)
    assert not np.array_equal(a.procs(0)["traj_hash"], b.procs(0)["traj_hash"])


# ---------------------------------------------------------------- limits
def test_largest_process_count_sampled(cse):
    """2^20 processes per matrix (the largest the ABI accepts) on the
    (3,3,3:23) shape, 16 steps (before the first sharing boundary), sampled
    processes replayed by the oracle."""
    s = synth.config2(n_proc=1 << 20, budget=16)
    r = cse.search_obj(s, trace=True)
    sample = [0, 1, 2, 65535, 524287, 999999, (1 << 20) - 1]
    ref = O.search_obj(s, n_threads=8, subset=sample)
    for k in range(3):
        got, exp = r.procs(k)[sample], ref.digests[k][sample]
        for f in FIELDS:
            assert np.array_equal(got[f], exp[f]), (k, f)
    steps, _, _ = r.counters()
    assert steps == 3 * (1 << 20) * 16
    r.free()


def _dense(seed, rows, cols):
    rng = np.random.default_rng(seed)
    mat = (rng.integers(0, 2, (rows, cols)) * rng.choice([-1, 1], (rows, cols))).astype(np.int8)
    mat[:, 0] = 1  # no empty row
    return mat


def test_longest_candidate_lists(cse):
    """Dense 256-row matrices repeat nearly every signed pair.  With 200
    columns that is 39800 initial candidates, more than the 32767 a list
    holds: loading refuses the matrix.  With 181 columns it is 32580: the
    matrix loads, but its first substitution grows the list to 32937 (the
    oracle's count), so the search stops with the overflow status instead of
    continuing on a clipped list."""
    with pytest.raises(cse.CseError, match="initial repeated pairs") as e:
        cse.Scheme([_dense(9, 256, 200)])
    assert e.value.code == cse.CSE_EINVAL
    mat = _dense(9, 256, 181)
    assert len(O.pairs(mat)) == 32580
    s = synth.Search("dense-181", [mat], (0, 0, 0, 0, 0, 1), 1, 1, 3, 2, 400, 512)
    ref = O.search_obj(s)
    assert len(O.pairs(O.apply(mat, ref.lists[0][:1])[0])) > 32767
    r = cse.search_obj(s)   # enqueued; the status is read with the result
    with pytest.raises(cse.CseError, match="candidate list overflow") as e:
        r.fetch(0)
    assert e.value.code == cse.CSE_ESTATE
    r.free()


def test_largest_shapes(cse):
    """Sixteen matrices (the most a scheme may hold), among them 256 rows
    (8 words per column) and 511 columns with the 512-column cap, plus
    single-row and single-column-pair matrices; sparse rows keep the oracle
    fast."""
    mats = [synth.random_matrix(3000, 256, 24, 2, 3, n_planted=6),
            synth.random_matrix(3001, 12, 511, 2, 3, n_planted=4),
            synth.random_matrix(3002, 1, 6, 2, 6),
            np.array([[1, 1], [1, 1], [-1, -1]], np.int8)]
    mats += [synth.random_matrix(3003 + k, 8 + 3 * k, 6 + k, 2, 4, n_planted=2) for k in range(12)]
    s = synth.Search("limits", mats, synth.PAPER_WEIGHTS, 9, 4, 24, 8, 400, 512)
    ref = assert_parity(cse, s)
    assert len(ref.cost) == 16
    # the 511-column matrix has room for one substitution only
    assert ref.length[1] <= 1
