"""ctypes binding of the C oracle (cse_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it to check and time the CUDA library.  The
library itself never imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cse_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

G, GI, GA, GR, WR, MIX, GP = 5, 0, 1, 2, 3, 4, 6
N_STRATEGIES = 7
GI_SHARED_COINS = 1  # search flag: one Greedy-Intersections coin per candidate per step


class Digest(ctypes.Structure):
    _fields_ = [("best_cost", ctypes.c_int64), ("best_len", ctypes.c_int32), ("runs", ctypes.c_int32),
                ("best_hash", ctypes.c_uint64), ("traj_hash", ctypes.c_uint64), ("ops", ctypes.c_int64),
                ("substeps", ctypes.c_int64), ("best_strategy", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("method_ops", ctypes.c_int64)]


DIGEST_DTYPE = np.dtype([("best_cost", "<i8"), ("best_len", "<i4"), ("runs", "<i4"),
                         ("best_hash", "<u8"), ("traj_hash", "<u8"), ("ops", "<i8"),
                         ("substeps", "<i8"), ("best_strategy", "<i4"), ("pad", "<i4"),
                         ("method_ops", "<i8")])
CURVE_POINTS = 4096  # rounds recorded in the best-Cost curve
assert DIGEST_DTYPE.itemsize == ctypes.sizeof(Digest)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build (plain -O2, no SIMD flags)."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lpthread"])
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        # ORACLE_LIB: a separately compiled copy of this oracle (the pin
        # tests load deliberately broken copies through it, to show that the
        # pins catch each planted mistake)
        L = ctypes.CDLL(os.environ.get("ORACLE_LIB") or build())
        i8p = ctypes.POINTER(ctypes.c_int8)
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        L.oracle_philox.argtypes = [u32p, u32p, u32p]
        L.oracle_philox.restype = None
        L.oracle_philox_n.argtypes = [u32p, u32p, ctypes.c_int64, u32p]
        L.oracle_philox_n.restype = None
        L.oracle_mix_strategy.argtypes = [ctypes.c_uint32]
        L.oracle_mix_strategy.restype = ctypes.c_int32
        L.oracle_gi_philox_coins.argtypes = [u32p, i32p, ctypes.c_int32, ctypes.c_uint64, ctypes.c_int32,
                                             ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.POINTER(ctypes.c_uint8)]
        L.oracle_gi_philox_coins.restype = ctypes.c_int32
        L.oracle_gp_select.argtypes = [i8p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
        L.oracle_gp_select.restype = ctypes.c_int32
        L.oracle_alpha.argtypes = [ctypes.c_uint32]
        L.oracle_alpha.restype = ctypes.c_int32
        L.oracle_beta.argtypes = [ctypes.c_uint32]
        L.oracle_beta.restype = ctypes.c_int32
        L.oracle_naive.argtypes = [i8p, ctypes.c_int32, ctypes.c_int32]
        L.oracle_naive.restype = ctypes.c_int64
        L.oracle_pairs.argtypes = [i8p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, u32p, i32p, ctypes.c_int32]
        L.oracle_pairs.restype = ctypes.c_int32
        L.oracle_apply.argtypes = [i8p, ctypes.c_int32, ctypes.c_int32, i32p, ctypes.c_int32, i8p]
        L.oracle_apply.restype = ctypes.c_int64
        L.oracle_select_basic.argtypes = [ctypes.c_int32, i32p, ctypes.c_int32, u32p]
        L.oracle_select_basic.restype = ctypes.c_int32
        L.oracle_gi_scores_coins.argtypes = [u32p, i32p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint32,
                                             ctypes.POINTER(ctypes.c_uint8), i64p]
        L.oracle_gi_scores_coins.restype = ctypes.c_int32
        L.oracle_gp_potentials.argtypes = [i8p, ctypes.c_int32, ctypes.c_int32, i32p, ctypes.c_int32]
        L.oracle_gp_potentials.restype = ctypes.c_int32
        L.oracle_brent_violations.argtypes = [ctypes.c_int32] * 4 + [i8p, i8p, i8p]
        L.oracle_brent_violations.restype = ctypes.c_int64
        L.oracle_flip_apply.argtypes = [ctypes.c_int32] * 4 + [i8p, i8p, i8p] + [ctypes.c_int32] * 4
        L.oracle_flip_apply.restype = ctypes.c_int32
        L.oracle_flip_variant.argtypes = [ctypes.c_int32] * 4 + [i8p, i8p, i8p, ctypes.c_uint64] + \
            [ctypes.c_int32] * 3 + [i8p, i8p, i8p]
        L.oracle_flip_variant.restype = ctypes.c_int32
        L.oracle_bruteforce.argtypes = [i8p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
        L.oracle_bruteforce.restype = ctypes.c_int64
        L.oracle_search.argtypes = [ctypes.c_int32, ctypes.POINTER(i8p), i32p, i32p, u32p, ctypes.c_int32,
                                    ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_int32, ctypes.c_int32, i32p, ctypes.c_int32, i64p, i32p, i32p,
                                    ctypes.POINTER(Digest)]
        L.oracle_search.restype = ctypes.c_int
        L.oracle_search_iterations.argtypes = [ctypes.c_int32, ctypes.POINTER(i8p), i32p, i32p, u32p, ctypes.c_int32,
                                               ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                               ctypes.c_int32, ctypes.c_uint32, ctypes.c_int32, i64p, i32p, i32p,
                                               ctypes.POINTER(Digest), i64p, i32p, ctypes.c_int32]
        L.oracle_search_flags.argtypes = [ctypes.c_int32, ctypes.POINTER(i8p), i32p, i32p, u32p, ctypes.c_int32,
                                          ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_uint32, ctypes.c_int32, i32p, ctypes.c_int32,
                                          i64p, i32p, i32p, ctypes.POINTER(Digest), i32p, ctypes.c_int32]
        L.oracle_search_flags.restype = ctypes.c_int
        L.oracle_search_snapshots.argtypes = [ctypes.c_int32, ctypes.POINTER(i8p), i32p, i32p, u32p, ctypes.c_int32,
                                              ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_int32, ctypes.c_int32, i64p, i32p,
                                              ctypes.POINTER(ctypes.c_uint64), ctypes.c_int32]
        L.oracle_search_snapshots.restype = ctypes.c_int
        L.oracle_search_iterations.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def philox(ctr: Sequence[int], key: Sequence[int]) -> List[int]:
    c = np.array(ctr, dtype=np.uint32)
    k = np.array(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32), _p(o, ctypes.c_uint32))
    return [int(x) for x in o]


def philox_n(ctr: np.ndarray, key: Sequence[int]) -> np.ndarray:
    """Philox4x32-10 of every row of ctr (n x 4 uint32) under one key."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.array(key, dtype=np.uint32)
    o = np.zeros_like(c)
    lib().oracle_philox_n(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32), c.shape[0], _p(o, ctypes.c_uint32))
    return o


def naive(mat: np.ndarray) -> int:
    m = np.ascontiguousarray(mat, dtype=np.int8)
    return int(lib().oracle_naive(_p(m, ctypes.c_int8), m.shape[0], m.shape[1]))


def key(i: int, j: int, s: int) -> int:
    """Canonical key of pair (x_i + s x_j), i < j (0-based)."""
    return (((j << 10) | i) << 1) | (1 if s < 0 else 0)


def unkey(k: int):
    return (k >> 1) & 0x3FF, (k >> 11) & 0x3FF, -1 if k & 1 else 1


def entry(i: int, j: int, s: int) -> int:
    return i | (j << 10) | ((1 if s < 0 else 0) << 20)


def unentry(e: int):
    return e & 0x3FF, (e >> 10) & 0x3FF, -1 if (e >> 20) & 1 else 1


def pairs(mat: np.ndarray, min_c: int = 2):
    """Canonical pairs with count >= min_c, in canonical order: list of (key, c)."""
    m = np.ascontiguousarray(mat, dtype=np.int8)
    cap = m.shape[0] * m.shape[1] * m.shape[1] + 1
    keys = np.zeros(cap, dtype=np.uint32)
    cnt = np.zeros(cap, dtype=np.int32)
    n = lib().oracle_pairs(_p(m, ctypes.c_int8), m.shape[0], m.shape[1], min_c, _p(keys, ctypes.c_uint32),
                           _p(cnt, ctypes.c_int32), cap)
    return [(int(keys[t]), int(cnt[t])) for t in range(n)]


def apply(mat: np.ndarray, entries: Sequence[int]):
    """Apply a substitution list; returns (final matrix, Cost) (Cost -1 if invalid)."""
    m = np.ascontiguousarray(mat, dtype=np.int8)
    lst = np.ascontiguousarray(np.array(list(entries), dtype=np.int32))
    out = np.zeros((m.shape[0], m.shape[1] + len(lst)), dtype=np.int8)
    c = lib().oracle_apply(_p(m, ctypes.c_int8), m.shape[0], m.shape[1], _p(lst, ctypes.c_int32), len(lst),
                           _p(out, ctypes.c_int8))
    return out, int(c)


def select_basic(kind: int, counts: Sequence[int], u: Sequence[int]) -> int:
    c = np.ascontiguousarray(np.array(counts, dtype=np.int32))
    uu = np.zeros(2, dtype=np.uint32)
    uu[:len(u)] = u
    return int(lib().oracle_select_basic(kind, _p(c, ctypes.c_int32), len(c), _p(uu, ctypes.c_uint32)))


def mix_strategy(u: int) -> int:
    """The strategy (GI, GA, GR or WR) a Mixed step runs for its draw u."""
    return int(lib().oracle_mix_strategy(u))


def alpha_beta(u_alpha: int, u_beta: int):
    """A run's (a, b): alpha and beta in units of 2^-16 from its two draws."""
    return int(lib().oracle_alpha(u_alpha)), int(lib().oracle_beta(u_beta))


def gi_philox_coins(keys: Sequence[int], counts: Sequence[int], seed: int, proc: int, t: int, mat: int,
                    shared: bool = False) -> np.ndarray:
    """The m x m Greedy-Intersections coins a process draws at step t
    (255 where none is drawn)."""
    k = np.ascontiguousarray(np.array(keys, dtype=np.uint32))
    c = np.ascontiguousarray(np.array(counts, dtype=np.int32))
    m = len(k)
    out = np.zeros((m, m), dtype=np.uint8)
    lib().oracle_gi_philox_coins(_p(k, ctypes.c_uint32), _p(c, ctypes.c_int32), m, seed, proc, t, mat,
                                 1 if shared else 0, _p(out, ctypes.c_uint8))
    return out


def gi_scores(keys: Sequence[int], counts: Sequence[int], a: int, b: int, coins: np.ndarray):
    k = np.ascontiguousarray(np.array(keys, dtype=np.uint32))
    c = np.ascontiguousarray(np.array(counts, dtype=np.int32))
    m = len(k)
    cb = np.ascontiguousarray(np.asarray(coins, dtype=np.uint8).reshape(m, m))
    sc = np.zeros(m, dtype=np.int64)
    best = lib().oracle_gi_scores_coins(_p(k, ctypes.c_uint32), _p(c, ctypes.c_int32), m, a, b,
                                        _p(cb, ctypes.c_uint8), _p(sc, ctypes.c_int64))
    return int(best), [int(x) for x in sc]


def gp_select(mat: np.ndarray, a: int) -> int:
    """Index (canonical order) of the candidate Greedy-Potential picks for
    alpha = a / 2^16; -1 if no pair repeats."""
    m = np.ascontiguousarray(mat, dtype=np.int8)
    return int(lib().oracle_gp_select(_p(m, ctypes.c_int8), m.shape[0], m.shape[1], a))


def gp_potentials(mat: np.ndarray) -> List[int]:
    """Greedy-Potential potential of every candidate (c >= 2) in canonical order."""
    m = np.ascontiguousarray(mat, dtype=np.int8)
    cap = m.shape[0] * m.shape[1] * m.shape[1] + 1
    pot = np.zeros(cap, dtype=np.int32)
    n = lib().oracle_gp_potentials(_p(m, ctypes.c_int8), m.shape[0], m.shape[1], _p(pot, ctypes.c_int32), cap)
    return [int(x) for x in pot[:n]]


def brent_violations(m: int, n: int, p: int, U: np.ndarray, V: np.ndarray, W: np.ndarray) -> int:
    """Number of violated Brent equations of the scheme (m,n,p:r)."""
    U, V, W = (np.ascontiguousarray(x, dtype=np.int8) for x in (U, V, W))
    r = U.shape[0]
    assert U.shape == (r, m * n) and V.shape == (r, n * p) and W.shape == (r, m * p)
    return int(lib().oracle_brent_violations(m, n, p, r, _p(U, ctypes.c_int8), _p(V, ctypes.c_int8),
                                             _p(W, ctypes.c_int8)))


def flip_apply(U, V, W, l: int, m: int, x: int, side: int):
    """One flip (R16) on copies of U, V, W; returns (applied, U, V, W)."""
    U, V, W = (np.array(a, dtype=np.int8, order="C") for a in (U, V, W))
    r = U.shape[0]
    ok = lib().oracle_flip_apply(r, U.shape[1], V.shape[1], W.shape[1], _p(U, ctypes.c_int8), _p(V, ctypes.c_int8),
                                 _p(W, ctypes.c_int8), l, m, x, side)
    return bool(ok), U, V, W


def flip_variant(m: int, n: int, p: int, U, V, W, seed: int, iteration: int, variant: int, max_flips: int):
    """Variant `variant` of flip iteration `iteration` (R16): (flips, U, V, W)."""
    U, V, W = (np.ascontiguousarray(a, dtype=np.int8) for a in (U, V, W))
    r = U.shape[0]
    oU, oV, oW = np.zeros_like(U), np.zeros_like(V), np.zeros_like(W)
    k = lib().oracle_flip_variant(m, n, p, r, _p(U, ctypes.c_int8), _p(V, ctypes.c_int8), _p(W, ctypes.c_int8), seed,
                                  iteration, variant, max_flips, _p(oU, ctypes.c_int8), _p(oV, ctypes.c_int8),
                                  _p(oW, ctypes.c_int8))
    return int(k), oU, oV, oW


def bruteforce(mat: np.ndarray, cap: Optional[int] = None) -> int:
    m = np.ascontiguousarray(mat, dtype=np.int8)
    if cap is None:
        cap = m.shape[1] + 64
    return int(lib().oracle_bruteforce(_p(m, ctypes.c_int8), m.shape[0], m.shape[1], cap))


class SearchResult:
    def __init__(self, cost, length, lists, digests):
        self.cost = cost            # per matrix best Cost
        self.length = length        # per matrix best list length
        self.lists = lists          # per matrix list of packed entries
        self.digests = digests      # (n_mats, n_proc) structured array or None

    @property
    def total(self) -> int:
        return int(sum(self.cost))


def search(mats: Sequence[np.ndarray], weights, n_proc: int, seed: int, budget: int, interval: int,
           permille: int, cap: int, n_threads: int = 1, subset: Optional[Sequence[int]] = None,
           digests: bool = True, flags: int = 0) -> SearchResult:
    ms = [np.ascontiguousarray(m, dtype=np.int8) for m in mats]
    n = len(ms)
    ptrs = (ctypes.POINTER(ctypes.c_int8) * n)(*[_p(m, ctypes.c_int8) for m in ms])
    rows = np.array([m.shape[0] for m in ms], dtype=np.int32)
    cols = np.array([m.shape[1] for m in ms], dtype=np.int32)
    w = np.zeros(N_STRATEGIES, dtype=np.uint32)   # gi, ga, gr, wr, mix, g, gp; missing trailing weights are 0
    if len(weights) > N_STRATEGIES:
        raise ValueError("at most 7 strategy weights")
    w[:len(weights)] = list(weights)
    cost = np.zeros(n, dtype=np.int64)
    length = np.zeros(n, dtype=np.int32)
    lists = np.zeros((n, cap), dtype=np.int32)
    dig = np.zeros((n, n_proc), dtype=DIGEST_DTYPE) if digests else None
    curve = np.full((n, CURVE_POINTS), -1, dtype=np.int32)
    sub = None if subset is None else np.ascontiguousarray(np.array(subset, dtype=np.int32))
    rc = lib().oracle_search_flags(n, ptrs, _p(rows, ctypes.c_int32), _p(cols, ctypes.c_int32),
                             _p(w, ctypes.c_uint32), n_proc, seed, budget, interval, permille, cap, flags, n_threads,
                             None if sub is None else _p(sub, ctypes.c_int32), 0 if sub is None else len(sub),
                             _p(cost, ctypes.c_int64), _p(length, ctypes.c_int32), _p(lists, ctypes.c_int32),
                             None if dig is None else dig.ctypes.data_as(ctypes.POINTER(Digest)),
                             _p(curve, ctypes.c_int32), CURVE_POINTS)
    if rc != 0:
        raise ValueError(f"oracle_search rejected its arguments (rc={rc})")
    r = SearchResult([int(x) for x in cost], [int(x) for x in length],
                     [[int(e) for e in lists[k, :length[k]]] for k in range(n)], dig)
    rounds = min(CURVE_POINTS, (budget + interval - 1) // interval)
    r.curve = [[int(v) for v in curve[k, :rounds]] for k in range(n)]
    return r


def search_snapshots(mats: Sequence[np.ndarray], weights, n_proc: int, seed: int, budget: int, interval: int,
                     permille: int, cap: int, n_threads: int = 1):
    """Step-clock search: (costs, best-Cost curve, hash of the shared list in
    force after each round; 0 while none), per matrix."""
    ms = [np.ascontiguousarray(m, dtype=np.int8) for m in mats]
    n = len(ms)
    ptrs = (ctypes.POINTER(ctypes.c_int8) * n)(*[_p(m, ctypes.c_int8) for m in ms])
    rows = np.array([m.shape[0] for m in ms], dtype=np.int32)
    cols = np.array([m.shape[1] for m in ms], dtype=np.int32)
    w = np.zeros(N_STRATEGIES, dtype=np.uint32)
    w[:len(weights)] = list(weights)
    cost = np.zeros(n, dtype=np.int64)
    curve = np.full((n, CURVE_POINTS), -1, dtype=np.int32)
    snap = np.zeros((n, CURVE_POINTS), dtype=np.uint64)
    rc = lib().oracle_search_snapshots(n, ptrs, _p(rows, ctypes.c_int32), _p(cols, ctypes.c_int32),
                                       _p(w, ctypes.c_uint32), n_proc, seed, budget, interval, permille, cap,
                                       n_threads, _p(cost, ctypes.c_int64), _p(curve, ctypes.c_int32),
                                       _p(snap, ctypes.c_uint64), CURVE_POINTS)
    if rc != 0:
        raise ValueError(f"oracle_search_snapshots rejected its arguments (rc={rc})")
    rounds = min(CURVE_POINTS, (budget + interval - 1) // interval)
    return [int(x) for x in cost], curve[:, :rounds].tolist(), snap[:, :rounds]


def search_iterations(mats: Sequence[np.ndarray], weights, n_proc: int, seed: int, max_iterations: int,
                      patience: int, permille: int, cap: int, n_threads: int = 1,
                      digests: bool = True, flags: int = 0) -> SearchResult:
    """Iteration mode (the paper's schedule): one whole run per process per
    iteration, sharing between iterations, stop on patience.  The result's
    `iterations` and `process_steps` say how long it ran."""
    ms = [np.ascontiguousarray(m, dtype=np.int8) for m in mats]
    n = len(ms)
    ptrs = (ctypes.POINTER(ctypes.c_int8) * n)(*[_p(m, ctypes.c_int8) for m in ms])
    rows = np.array([m.shape[0] for m in ms], dtype=np.int32)
    cols = np.array([m.shape[1] for m in ms], dtype=np.int32)
    w = np.zeros(N_STRATEGIES, dtype=np.uint32)
    w[:len(weights)] = list(weights)
    cost = np.zeros(n, dtype=np.int64)
    length = np.zeros(n, dtype=np.int32)
    lists = np.zeros((n, cap), dtype=np.int32)
    dig = np.zeros((n, n_proc), dtype=DIGEST_DTYPE) if digests else None
    stats = np.zeros(2, dtype=np.int64)
    curve = np.full((n, CURVE_POINTS), -1, dtype=np.int32)
    rc = lib().oracle_search_iterations(n, ptrs, _p(rows, ctypes.c_int32), _p(cols, ctypes.c_int32),
                                        _p(w, ctypes.c_uint32), n_proc, seed, max_iterations, patience, permille,
                                        cap, flags, n_threads, _p(cost, ctypes.c_int64), _p(length, ctypes.c_int32),
                                        _p(lists, ctypes.c_int32),
                                        None if dig is None else dig.ctypes.data_as(ctypes.POINTER(Digest)),
                                        _p(stats, ctypes.c_int64), _p(curve, ctypes.c_int32), CURVE_POINTS)
    if rc != 0:
        raise ValueError(f"oracle_search_iterations rejected its arguments (rc={rc})")
    r = SearchResult([int(x) for x in cost], [int(x) for x in length],
                     [[int(e) for e in lists[k, :length[k]]] for k in range(n)], dig)
    r.iterations, r.process_steps = int(stats[0]), int(stats[1])
    r.curve = [[int(v) for v in curve[k, :min(CURVE_POINTS, r.iterations)]] for k in range(n)]
    return r


def search_obj(s, **kw) -> SearchResult:
    """Run the oracle on a synth.Search description."""
    return search(s.mats, s.weights, s.n_proc, s.seed, s.budget, s.interval, s.permille, s.cap, **kw)
