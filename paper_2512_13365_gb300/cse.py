"""Python binding of the GB300 CSE library (include/cse.h).

Argument marshalling only: every step of the search runs in the library's
CUDA kernels.  There is no CPU fallback: if the compiled library is missing
the import of the binding fails loudly with the build command to run.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("CSE_GB300_LIB") or os.path.join(_HERE, "_build", "libcse_gb300.so")

CSE_OK, CSE_EINVAL, CSE_ENOMEM, CSE_ECUDA, CSE_ETIMEOUT, CSE_EBUSY, CSE_ESTATE, CSE_ECANCELED = range(8)


class CseError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"cse error {code}: {msg}")
        self.code = code


class Mix(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in ("w_gi", "w_ga", "w_gr", "w_wr", "w_mix", "w_g", "w_gp")]


class Opts(ctypes.Structure):
    _fields_ = [("share_interval", ctypes.c_uint32), ("share_permille", ctypes.c_uint32),
                ("col_cap", ctypes.c_uint32), ("patience_rounds", ctypes.c_uint32),
                ("max_spin", ctypes.c_uint64), ("procs_per_cta", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("cta_list_cap", ctypes.c_uint32), ("cta_min_list", ctypes.c_uint32)]


class ProcRecord(ctypes.Structure):
    _fields_ = [("best_cost", ctypes.c_int64), ("best_len", ctypes.c_int32), ("runs", ctypes.c_int32),
                ("best_hash", ctypes.c_uint64), ("traj_hash", ctypes.c_uint64), ("ops", ctypes.c_int64),
                ("substeps", ctypes.c_int64), ("best_strategy", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("method_ops", ctypes.c_int64)]


class TuneEntry(ctypes.Structure):
    _fields_ = [("words_per_column", ctypes.c_int32), ("hbm_path", ctypes.c_int32),
                ("candidate_bound", ctypes.c_int32), ("procs_per_cta", ctypes.c_int32),
                ("trial_ms", ctypes.c_float * 4), ("kernel_words", ctypes.c_int32),
                ("trial_ms_wide", ctypes.c_float * 4)]


PROC_DTYPE = np.dtype([("best_cost", "<i8"), ("best_len", "<i4"), ("runs", "<i4"), ("best_hash", "<u8"),
                       ("traj_hash", "<u8"), ("ops", "<i8"), ("substeps", "<i8"), ("best_strategy", "<i4"),
                       ("pad", "<i4"), ("method_ops", "<i8")])
STRATEGIES = ("gi", "ga", "gr", "wr", "mix", "g", "gp")  # best_strategy indices
assert PROC_DTYPE.itemsize == ctypes.sizeof(ProcRecord)

_lib = None

# every symbol include/cse.h declares
EXPORTS = ["cse_opts_default", "cse_scheme_load", "cse_scheme_load_uvw", "cse_scheme_shape", "cse_search",
           "cse_search_batch", "cse_autotune", "cse_tune_interval", "cse_result_fetch", "cse_result_procs", "cse_result_counters", "cse_result_method_ops", "cse_result_engine_rounds", "cse_result_timing",
           "cse_result_iterations", "cse_result_curve", "cse_result_hybrid", "cse_brent_check", "cse_philox", "cse_checkpoint_size",
           "cse_checkpoint_save", "cse_search_resume", "cse_result_launches",
           "cse_result_free", "cse_scheme_free", "cse_last_error",
           "cse_server_create", "cse_server_submit", "cse_server_cancel", "cse_server_wait", "cse_server_stats",
           "cse_server_peak",
           "cse_server_free",
           "cse_search_static", "cse_int_peak", "cse_search_shard", "cse_shard_round", "cse_shard_best_list",
           "cse_shard_share", "cse_flip_variants"]

FLAG_GRAPH = 1
FLAG_TRACE = 2
FLAG_GI_SHARED_COINS = 4
FLAG_WARP_ENGINE = 8
FLAG_PERSISTENT = 16
FLAG_WIDE_WORDS = 32
FLAG_CTA_ENGINE = 64


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library {LIB_PATH} is not built: run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    pi32, pi64 = ctypes.POINTER(i32), ctypes.POINTER(i64)
    L.cse_last_error.restype = ctypes.c_char_p
    L.cse_opts_default.argtypes = [ctypes.POINTER(Opts)]
    L.cse_opts_default.restype = None
    L.cse_scheme_load.argtypes = [ctypes.POINTER(ctypes.POINTER(ctypes.c_int8)), pi32, pi32, i32,
                                  ctypes.POINTER(vp)]
    L.cse_scheme_load_uvw.argtypes = [i32, i32, i32, i32, vp, vp, vp, ctypes.POINTER(vp)]
    L.cse_scheme_shape.argtypes = [vp, i32, pi32, pi32]
    L.cse_search.argtypes = [vp, ctypes.POINTER(Mix), i32, u64, i64, ctypes.POINTER(Opts), vp,
                             ctypes.POINTER(vp)]
    L.cse_search_batch.argtypes = [i32, ctypes.POINTER(vp), ctypes.POINTER(Mix), pi32, ctypes.POINTER(u64), pi64,
                                   ctypes.POINTER(Opts), vp, ctypes.POINTER(vp)]
    L.cse_result_launches.argtypes = [vp, pi32, pi32]
    L.cse_result_iterations.argtypes = [vp, pi32, pi32, pi64]
    L.cse_result_curve.argtypes = [vp, i32, pi32, i32, pi32]
    L.cse_result_hybrid.argtypes = [ctypes.POINTER(vp), i32, pi32, pi64]
    L.cse_brent_check.argtypes = [i32, i32, i32, i32, vp, vp, vp, pi64]
    L.cse_philox.argtypes = [ctypes.c_uint64, vp, i64, vp]
    L.cse_checkpoint_size.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    L.cse_checkpoint_save.argtypes = [vp, vp, ctypes.c_size_t]
    L.cse_search_resume.argtypes = [vp, vp, ctypes.c_size_t, i64, ctypes.POINTER(Opts), vp, ctypes.POINTER(vp)]
    batch_args = [i32, ctypes.POINTER(vp), ctypes.POINTER(Mix), pi32, ctypes.POINTER(u64), pi64, ctypes.POINTER(Opts)]
    L.cse_autotune.argtypes = batch_args + [i32, vp, ctypes.POINTER(TuneEntry), i32, pi32]
    L.cse_tune_interval.argtypes = batch_args + [ctypes.POINTER(ctypes.c_uint32), i32, i32, vp,
                                                 ctypes.POINTER(ctypes.c_uint32), pi64]
    L.cse_result_fetch.argtypes = [vp, i32, pi32, i32, pi32, pi64, pi64]
    L.cse_result_procs.argtypes = [vp, i32, ctypes.POINTER(ProcRecord)]
    L.cse_result_counters.argtypes = [vp, pi64, pi64, pi64]
    L.cse_result_method_ops.argtypes = [vp, pi64]
    L.cse_result_engine_rounds.argtypes = [vp, pi64, pi64]
    L.cse_result_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), pi32]
    L.cse_result_free.argtypes = [vp]
    L.cse_result_free.restype = None
    L.cse_scheme_free.argtypes = [vp]
    L.cse_scheme_free.restype = None
    L.cse_server_create.argtypes = [ctypes.POINTER(Opts), ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(vp)]
    L.cse_server_submit.argtypes = [vp, vp, ctypes.POINTER(Mix), i32, u64, i64, ctypes.POINTER(ctypes.c_uint64)]
    L.cse_server_wait.argtypes = [vp, ctypes.c_uint64, i64, ctypes.POINTER(vp)]
    L.cse_server_cancel.argtypes = [vp, ctypes.c_uint64]
    L.cse_server_peak.argtypes = [vp, pi32, pi32]
    L.cse_server_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double), pi32]
    L.cse_search_static.argtypes = [vp, ctypes.POINTER(Mix), i32, u64, i64, ctypes.POINTER(Opts), vp, vp, vp]
    L.cse_int_peak.argtypes = [i32, i64, vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double)]
    L.cse_search_shard.argtypes = [vp, ctypes.POINTER(Mix), i32, i32, i32, u64, i64, ctypes.POINTER(Opts), vp,
                                   ctypes.POINTER(vp)]
    L.cse_shard_round.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64), pi32]
    L.cse_shard_best_list.argtypes = [vp, i32, ctypes.c_uint64, pi32, pi32]
    L.cse_shard_share.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64), pi32, pi32]
    L.cse_flip_variants.argtypes = [i32, i32, i32, i32, vp, vp, vp, i32, u64, i32, i32, vp, vp, vp, pi32, pi64]
    L.cse_server_free.argtypes = [vp]
    L.cse_server_free.restype = None
    for n in EXPORTS:
        if n not in ("cse_opts_default", "cse_result_free", "cse_scheme_free", "cse_last_error", "cse_server_free"):
            getattr(L, n).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc: int):
    if rc != CSE_OK:
        raise CseError(rc, lib().cse_last_error().decode())


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


class Scheme:
    """Expression sets loaded on the device (cse_scheme_load)."""

    def __init__(self, mats: Sequence[np.ndarray]):
        self.mats = [np.ascontiguousarray(m, dtype=np.int8) for m in mats]
        n = len(self.mats)
        ptrs = (ctypes.POINTER(ctypes.c_int8) * n)(*[m.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))
                                                       for m in self.mats])
        rows = (ctypes.c_int32 * n)(*[m.shape[0] for m in self.mats])
        cols = (ctypes.c_int32 * n)(*[m.shape[1] for m in self.mats])
        h = ctypes.c_void_p()
        _check(lib().cse_scheme_load(ptrs, rows, cols, n, ctypes.byref(h)))
        self.handle = h

    @classmethod
    def from_uvw(cls, m: int, n: int, p: int, U: np.ndarray, V: np.ndarray, W: np.ndarray) -> "Scheme":
        self = cls.__new__(cls)
        U, V, W = (np.ascontiguousarray(x, dtype=np.int8) for x in (U, V, W))
        r = U.shape[0]
        h = ctypes.c_void_p()
        _check(lib().cse_scheme_load_uvw(m, n, p, r, U.ctypes.data, V.ctypes.data, W.ctypes.data,
                                         ctypes.byref(h)))
        self.handle = h
        self.mats = [U, V, np.ascontiguousarray(W.T)]
        return self

    def shape(self, k: int) -> Tuple[int, int]:
        r, c = ctypes.c_int32(), ctypes.c_int32()
        _check(lib().cse_scheme_shape(self.handle, k, ctypes.byref(r), ctypes.byref(c)))
        return r.value, c.value

    def free(self):
        if getattr(self, "handle", None):
            lib().cse_scheme_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Result:
    """A running or finished search (cse_result)."""

    def __init__(self, handle, n_mats: int, n_proc: int, cap: int):
        self.handle = handle
        self.n_mats, self.n_proc, self.cap = n_mats, n_proc, cap

    def fetch(self, mat: int) -> Tuple[List[int], int, int]:
        """(best substitution list of matrix mat, its Cost, total over matrices)."""
        buf = (ctypes.c_int32 * self.cap)()
        n, add, tot = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().cse_result_fetch(self.handle, mat, buf, self.cap, ctypes.byref(n), ctypes.byref(add),
                                      ctypes.byref(tot)))
        return [int(buf[x]) for x in range(n.value)], int(add.value), int(tot.value)

    @property
    def costs(self) -> List[int]:
        return [self.fetch(k)[1] for k in range(self.n_mats)]

    @property
    def lists(self) -> List[List[int]]:
        return [self.fetch(k)[0] for k in range(self.n_mats)]

    @property
    def total(self) -> int:
        return self.fetch(0)[2]

    def procs(self, mat: int) -> np.ndarray:
        out = np.zeros(self.n_proc, dtype=PROC_DTYPE)
        _check(lib().cse_result_procs(self.handle, mat, out.ctypes.data_as(ctypes.POINTER(ProcRecord))))
        return out

    def counters(self) -> Tuple[int, int, int]:
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().cse_result_counters(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def method_ops(self) -> int:
        """cse_result_method_ops: the method's own op count of the search."""
        a = ctypes.c_int64()
        _check(lib().cse_result_method_ops(self.handle, ctypes.byref(a)))
        return a.value

    def engine_rounds(self) -> Tuple[int, int]:
        """cse_result_engine_rounds: large-matrix process-rounds on the
        process-per-CTA engine and on the HBM warp engine."""
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().cse_result_engine_rounds(self.handle, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def timing(self) -> Tuple[float, float, int]:
        a, b, n = ctypes.c_float(), ctypes.c_float(), ctypes.c_int32()
        _check(lib().cse_result_timing(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(n)))
        return a.value, b.value, n.value

    def iterations(self) -> Tuple[int, bool, int]:
        """Iteration mode: (iterations run, stopped by the patience rule, final best total)."""
        it, cv, tot = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        _check(lib().cse_result_iterations(self.handle, ctypes.byref(it), ctypes.byref(cv), ctypes.byref(tot)))
        return it.value, bool(cv.value), tot.value

    def curve(self, mat: int) -> List[int]:
        """cse_result_curve: the lowest best Cost after each round."""
        n = ctypes.c_int32()
        _check(lib().cse_result_curve(self.handle, mat, None, 0, ctypes.byref(n)))
        buf = (ctypes.c_int32 * max(1, n.value))()
        _check(lib().cse_result_curve(self.handle, mat, buf, n.value, ctypes.byref(n)))
        return list(buf[:n.value])

    def checkpoint(self) -> bytes:
        """cse_checkpoint_save: the finished search's checkpoint as bytes."""
        n = ctypes.c_size_t()
        _check(lib().cse_checkpoint_size(self.handle, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _check(lib().cse_checkpoint_save(self.handle, buf, n.value))
        return buf.raw

    def launches(self) -> Tuple[int, int]:
        """(kernel launches of the launch sequence, searches that shared it)."""
        k, n = ctypes.c_int32(), ctypes.c_int32()
        _check(lib().cse_result_launches(self.handle, ctypes.byref(k), ctypes.byref(n)))
        return k.value, n.value

    def free(self):
        if getattr(self, "handle", None):
            lib().cse_result_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def hybrid(results: Sequence["Result"]) -> Tuple[List[int], int]:
    """cse_result_hybrid: per matrix, the index of the result with the lowest
    Cost (first on ties), and the total of those Costs."""
    n = len(results)
    hs = (ctypes.c_void_p * n)(*[r.handle.value for r in results])
    nm = results[0].n_mats
    best = (ctypes.c_int32 * nm)()
    tot = ctypes.c_int64()
    _check(lib().cse_result_hybrid(hs, n, best, ctypes.byref(tot)))
    return list(best), tot.value


def brent_check(m: int, n: int, p: int, U: np.ndarray, V: np.ndarray, W: np.ndarray) -> int:
    """cse_brent_check: the number of violated Brent equations (0 = valid scheme)."""
    U, V, W = (np.ascontiguousarray(x, dtype=np.int8) for x in (U, V, W))
    r = U.shape[0]
    if U.shape != (r, m * n) or V.shape != (r, n * p) or W.shape != (r, m * p):
        raise ValueError("U, V, W must be r x mn, r x np, r x mp")
    out = ctypes.c_int64()
    _check(lib().cse_brent_check(m, n, p, r, U.ctypes.data, V.ctypes.data, W.ctypes.data, ctypes.byref(out)))
    return out.value


def philox(seed: int, counters: np.ndarray) -> np.ndarray:
    """cse_philox: Philox4x32-10 of every row of counters (n x 4 uint32) under
    the key (seed & 0xFFFFFFFF, seed >> 32), computed on the device."""
    c = np.ascontiguousarray(counters, dtype=np.uint32).reshape(-1, 4)
    out = np.zeros_like(c)
    _check(lib().cse_philox(seed, c.ctypes.data, c.shape[0], out.ctypes.data))
    return out


INT_PEAK_KINDS = ("lop3+iadd3", "and+popc+iadd", "imad", "imad.hi", "lop3", "iadd3")


def int_peak(kind: int, iters: int = 100000, stream=None) -> dict:
    """cse_int_peak: measured lane-ops per SM clock (and per second) of one
    integer instruction mix (INT_PEAK_KINDS[kind])."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().cse_int_peak(kind, iters, _stream_ptr(stream), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return {"kind": INT_PEAK_KINDS[kind], "ops_per_clk_per_sm": a.value, "lane_ops_per_s": b.value,
            "seconds": c.value}


def make_mix(weights) -> Mix:
    w = list(weights) + [0] * (7 - len(weights))
    return Mix(*[int(x) for x in w])


def make_opts(interval: int = 32, permille: int = 400, cap: int = 128, procs_per_cta: int = 0,
              graph: bool = False, trace: bool = False, patience: int = 0, gi_shared: bool = False,
              warp_engine: bool = False, cta_list_cap: int = 0, cta_min_list: int = 0, persistent: bool = False,
              max_spin: int = 0, wide_words: bool = False, cta_engine: bool = False) -> Opts:
    """interval 0 selects iteration mode (budget = maximum iterations, stop
    after `patience` iterations without improvement).  warp_engine,
    cta_engine, cta_list_cap and cta_min_list choose how large matrices are
    launched; never results."""
    o = Opts()
    lib().cse_opts_default(ctypes.byref(o))
    o.share_interval, o.share_permille, o.col_cap, o.procs_per_cta = interval, permille, cap, procs_per_cta
    o.patience_rounds = patience
    o.flags = ((FLAG_GRAPH if graph else 0) | (FLAG_TRACE if trace else 0) |
               (FLAG_GI_SHARED_COINS if gi_shared else 0) | (FLAG_WARP_ENGINE if warp_engine else 0) |
               (FLAG_PERSISTENT if persistent else 0) | (FLAG_WIDE_WORDS if wide_words else 0) |
               (FLAG_CTA_ENGINE if cta_engine else 0))
    o.max_spin = max_spin
    o.cta_list_cap = cta_list_cap
    o.cta_min_list = cta_min_list
    return o


@dataclasses.dataclass
class Options:
    """The fields of cse_opts (include/cse.h) as a Python record; the flags
    are spelled out.  to_struct() gives the C struct, from_struct() reads
    one back."""
    share_interval: int = 32
    share_permille: int = 400
    col_cap: int = 128
    patience_rounds: int = 0
    procs_per_cta: int = 0
    graph: bool = False
    trace: bool = False
    gi_shared: bool = False

    def to_struct(self) -> Opts:
        return make_opts(self.share_interval, self.share_permille, self.col_cap, self.procs_per_cta, self.graph,
                         self.trace, self.patience_rounds, self.gi_shared)

    @classmethod
    def from_struct(cls, o: Opts) -> "Options":
        return cls(o.share_interval, o.share_permille, o.col_cap, o.patience_rounds, o.procs_per_cta,
                   bool(o.flags & FLAG_GRAPH), bool(o.flags & FLAG_TRACE), bool(o.flags & FLAG_GI_SHARED_COINS))

    @classmethod
    def library_default(cls) -> "Options":
        o = Opts()
        lib().cse_opts_default(ctypes.byref(o))
        return cls.from_struct(o)


def search(scheme: Scheme, weights, n_proc: int, seed: int, budget: int, interval: int = 32,
           permille: int = 400, cap: int = 128, stream=None, procs_per_cta: int = 0, graph: bool = False,
           trace: bool = False, patience: int = 0, gi_shared: bool = False, warp_engine: bool = False,
           cta_list_cap: int = 0, cta_min_list: int = 0, wide_words: bool = False,
           cta_engine: bool = False) -> Result:
    """cse_search: enqueue the search and return its Result handle."""
    mix = make_mix(weights)
    opts = make_opts(interval, permille, cap, procs_per_cta, graph, trace, patience, gi_shared, warp_engine,
                     cta_list_cap, cta_min_list, wide_words=wide_words, cta_engine=cta_engine)
    h = ctypes.c_void_p()
    _check(lib().cse_search(scheme.handle, ctypes.byref(mix), n_proc, seed, budget, ctypes.byref(opts),
                            _stream_ptr(stream), ctypes.byref(h)))
    return Result(h, len(scheme.mats), n_proc, cap)


def resume(scheme: Scheme, checkpoint: bytes, more_steps: int, stream=None, procs_per_cta: int = 0,
           warp_engine: bool = False, cta_min_list: int = 0, cta_engine: bool = False) -> Result:
    """cse_search_resume: continue a checkpointed search for more_steps steps
    (the launch options may differ from the original search's)."""
    import struct
    cap, = struct.unpack_from("<I", checkpoint, 20)       # header fields (cse_api.cu): col_cap ...
    n_proc, = struct.unpack_from("<i", checkpoint, 36)    # ... and the process count
    opts = make_opts(procs_per_cta=procs_per_cta, warp_engine=warp_engine, cta_min_list=cta_min_list,
                     cta_engine=cta_engine)
    buf = ctypes.create_string_buffer(checkpoint, len(checkpoint))
    h = ctypes.c_void_p()
    _check(lib().cse_search_resume(scheme.handle, buf, len(checkpoint), more_steps, ctypes.byref(opts),
                                   _stream_ptr(stream), ctypes.byref(h)))
    r = Result(h, len(scheme.mats), n_proc, cap)
    r._scheme = scheme
    return r


def search_obj(s, scheme: Optional[Scheme] = None, **kw) -> Result:
    """Run a synth.Search description on the device."""
    sc = scheme if scheme is not None else Scheme(s.mats)
    r = search(sc, s.weights, s.n_proc, s.seed, s.budget, s.interval, s.permille, s.cap, **kw)
    r._scheme = sc  # keep the device inputs alive while the search runs
    return r


def search_batch(schemes: Sequence[Scheme], weights: Sequence, n_procs: Sequence[int], seeds: Sequence[int],
                 budgets: Sequence[int], interval: int = 32, permille: int = 400, cap: int = 128, stream=None,
                 procs_per_cta: int = 0, graph: bool = True, trace: bool = False,
                 patience: int = 0, gi_shared: bool = False, persistent: bool = False,
                 max_spin: int = 0, wide_words: bool = False) -> List[Result]:
    """cse_search_batch: independent searches in one launch sequence (with
    persistent, one cooperative kernel over every round)."""
    n = len(schemes)
    hs = (ctypes.c_void_p * n)(*[s.handle for s in schemes])
    mixes = (Mix * n)(*[make_mix(w) for w in weights])
    np_ = (ctypes.c_int32 * n)(*n_procs)
    sd = (ctypes.c_uint64 * n)(*seeds)
    bd = (ctypes.c_int64 * n)(*budgets)
    opts = make_opts(interval, permille, cap, procs_per_cta, graph, trace, patience, gi_shared,
                     persistent=persistent, max_spin=max_spin, wide_words=wide_words)
    outs = (ctypes.c_void_p * n)()
    _check(lib().cse_search_batch(n, hs, mixes, np_, sd, bd, ctypes.byref(opts), _stream_ptr(stream), outs))
    res = []
    for i in range(n):
        r = Result(ctypes.c_void_p(outs[i]), len(schemes[i].mats), n_procs[i], cap)
        r._scheme = schemes[i]
        res.append(r)
    return res


def search_batch_obj(searches, **kw) -> List[Result]:
    """Run several synth.Search descriptions (same interval, permille and cap) as one batch."""
    s0 = searches[0]
    assert all((s.interval, s.permille, s.cap) == (s0.interval, s0.permille, s0.cap) for s in searches)
    schemes = [Scheme(s.mats) for s in searches]
    return search_batch(schemes, [s.weights for s in searches], [s.n_proc for s in searches],
                        [s.seed for s in searches], [s.budget for s in searches], s0.interval, s0.permille,
                        s0.cap, **kw)


def _batch_args(schemes, weights, n_procs, seeds, budgets, interval, permille, cap, procs_per_cta=0, graph=False):
    n = len(schemes)
    return (n, (ctypes.c_void_p * n)(*[s.handle for s in schemes]), (Mix * n)(*[make_mix(w) for w in weights]),
            (ctypes.c_int32 * n)(*n_procs), (ctypes.c_uint64 * n)(*seeds), (ctypes.c_int64 * n)(*budgets),
            ctypes.byref(make_opts(interval, permille, cap, procs_per_cta, graph)))


def autotune(schemes, weights, n_procs, seeds, budgets, interval=32, permille=400, cap=128, trial_steps=64,
             stream=None) -> List[dict]:
    """cse_autotune: time 1..4 processes per CTA per matrix class (and the
    next power-of-two words per column); cache the fastest."""
    args = _batch_args(schemes, weights, n_procs, seeds, budgets, interval, permille, cap)
    ent = (TuneEntry * 64)()
    ne = ctypes.c_int32()
    _check(lib().cse_autotune(*args, trial_steps, _stream_ptr(stream), ent, 64, ctypes.byref(ne)))
    return [{"words_per_column": e.words_per_column, "hbm_path": e.hbm_path, "candidate_bound": e.candidate_bound,
             "procs_per_cta": e.procs_per_cta, "trial_ms": list(e.trial_ms), "kernel_words": e.kernel_words,
             "trial_ms_wide": list(e.trial_ms_wide)} for e in ent[:ne.value]]


def tune_interval(schemes, weights, n_procs, seeds, budgets, candidates=(16, 32, 64), permille=400, cap=128,
                  trial_steps=128, stream=None) -> Tuple[int, int]:
    """cse_tune_interval: the candidate interval with the lowest total additions after a trial."""
    args = _batch_args(schemes, weights, n_procs, seeds, budgets, candidates[0], permille, cap)
    c = (ctypes.c_uint32 * len(candidates))(*candidates)
    best, tot = ctypes.c_uint32(), ctypes.c_int64()
    _check(lib().cse_tune_interval(*args, c, len(candidates), trial_steps, _stream_ptr(stream), ctypes.byref(best),
                                   ctypes.byref(tot)))
    return best.value, tot.value


def flip_variants(m: int, n: int, p: int, U: np.ndarray, V: np.ndarray, W: np.ndarray, n_variants: int, seed: int,
                  iteration: int, max_flips: int = 16):
    """cse_flip_variants: (flips per variant, U, V, W stacked by variant,
    violated Brent equations per variant), all generated and checked on the
    device (Section 3.5.3)."""
    U, V, W = (np.ascontiguousarray(x, dtype=np.int8) for x in (U, V, W))
    r = U.shape[0]
    if U.shape != (r, m * n) or V.shape != (r, n * p) or W.shape != (r, m * p):
        raise ValueError("U, V, W must be r x mn, r x np, r x mp")
    oU = np.zeros((n_variants, r, m * n), np.int8)
    oV = np.zeros((n_variants, r, n * p), np.int8)
    oW = np.zeros((n_variants, r, m * p), np.int8)
    fl = np.zeros(n_variants, np.int32)
    bad = np.zeros(n_variants, np.int64)
    _check(lib().cse_flip_variants(m, n, p, r, U.ctypes.data, V.ctypes.data, W.ctypes.data, n_variants, seed,
                                   iteration, max_flips, oU.ctypes.data, oV.ctypes.data, oW.ctypes.data,
                                   fl.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   bad.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return fl, oU, oV, oW, bad


def flip_search(m: int, n: int, p: int, U: np.ndarray, V: np.ndarray, W: np.ndarray, weights, n_variants: int = 32,
                n_proc: int = 1024, seed: int = 0, iterations: int = 4, budget: int = 256, interval: int = 32,
                permille: int = 400, cap: int = 256, max_flips: int = 16, stream=None) -> dict:
    """The random-flip mode (Section 3.5.3): every iteration regenerates
    n_variants variants of the scheme (variant 0 the scheme itself), checks
    them on the device, and searches all of them side by side (one search of
    n_proc processes per variant, in one batch, seed + iteration); the best
    total over every variant and iteration is kept.  Returns the best
    (iteration, variant, total, costs, lists, U, V, W) and every total."""
    best, totals = None, []
    for it in range(iterations):
        fl, vU, vV, vW, bad = flip_variants(m, n, p, U, V, W, n_variants, seed, it, max_flips)
        if bad.any():
            raise CseError(CSE_ESTATE, f"flip variants broke a Brent equation: {bad.tolist()}")
        schemes = [Scheme.from_uvw(m, n, p, vU[v], vV[v], vW[v]) for v in range(n_variants)]
        rs = search_batch(schemes, [weights] * n_variants, [n_proc] * n_variants, [seed + it] * n_variants,
                          [budget] * n_variants, interval, permille, cap, stream=stream, graph=True)
        row = []
        for v, r in enumerate(rs):
            tot = r.total
            row.append(tot)
            if best is None or tot < best["total"]:
                best = {"iteration": it, "variant": v, "flips": int(fl[v]), "total": tot, "costs": r.costs,
                        "lists": r.lists, "U": vU[v].copy(), "V": vV[v].copy(), "W": vW[v].copy()}
            r.free()
        for sc in schemes:
            sc.free()
        totals.append(row)
    best["totals"] = totals
    return best


def shard_range(n_proc: int, rank: int, world: int) -> Tuple[int, int]:
    """(first process, count) of rank's shard of n_proc processes."""
    b, e = rank * n_proc // world, (rank + 1) * n_proc // world
    return b, e - b


def exchange_boundary(keys: Sequence[int], best_list, cap: int, group=None, device="cpu"):
    """The sharing-boundary exchange of a search split across ranks
    (torch.distributed): the minimum over the ranks of each matrix's round
    key (best Cost << 32 | global process), and the winner's best list, sent
    by the rank that owns it.  best_list(k, key) returns this rank's list for
    a key it owns, or None.  Two collectives per round: an allreduce-min of
    the keys and an allreduce-sum of one row of (length, list) per matrix,
    filled only by the owner.  Returns (keys, lists, lens) as numpy arrays."""
    import torch
    import torch.distributed as dist
    n = len(keys)
    k = torch.tensor([int(x) if int(x) < (1 << 63) else (1 << 63) - 1 for x in keys], dtype=torch.int64,
                     device=device)
    dist.all_reduce(k, op=dist.ReduceOp.MIN, group=group)
    gk = [int(x) for x in k.cpu().tolist()]
    rows = torch.zeros((n, cap + 1), dtype=torch.int64, device=device)
    for m in range(n):
        got = best_list(m, gk[m])
        if got is not None:
            rows[m, 0] = len(got)
            if got:
                rows[m, 1:1 + len(got)] = torch.tensor(got, dtype=torch.int64)
    dist.all_reduce(rows, op=dist.ReduceOp.SUM, group=group)
    rows = rows.cpu().numpy()
    lens = rows[:, 0].astype(np.int32)
    lists = np.ascontiguousarray(rows[:, 1:].astype(np.int32))
    gk = [x if x < (1 << 63) - 1 else (1 << 64) - 1 for x in gk]  # no report: the all-ones key
    return np.array(gk, dtype=np.uint64), lists, lens


class Shard(Result):
    """One rank's shard of a search split across ranks (cse_search_shard)."""

    def __init__(self, scheme: Scheme, weights, n_proc: int, rank: int, world: int, seed: int, budget: int,
                 interval: int = 32, permille: int = 400, cap: int = 128, stream=None, trace: bool = False,
                 procs_per_cta: int = 0):
        self.begin, count = shard_range(n_proc, rank, world)
        h = ctypes.c_void_p()
        opts = make_opts(interval, permille, cap, procs_per_cta, trace=trace)
        _check(lib().cse_search_shard(scheme.handle, ctypes.byref(make_mix(weights)), n_proc, self.begin, count,
                                      seed, budget, ctypes.byref(opts), _stream_ptr(stream), ctypes.byref(h)))
        super().__init__(h, len(scheme.mats), count, cap)
        self._scheme = scheme

    def round(self):
        """(this shard's round keys, rounds left including this one)."""
        keys = (ctypes.c_uint64 * self.n_mats)()
        left = ctypes.c_int32()
        _check(lib().cse_shard_round(self.handle, keys, ctypes.byref(left)))
        return [int(x) for x in keys], left.value

    def best_list(self, mat: int, key: int):
        """The best list of the process named by key, or None if another shard holds it."""
        proc = key & 0xFFFFFFFF
        if not (self.begin <= proc < self.begin + self.n_proc):
            return None
        buf = (ctypes.c_int32 * self.cap)()
        n = ctypes.c_int32()
        _check(lib().cse_shard_best_list(self.handle, mat, key, buf, ctypes.byref(n)))
        return [int(buf[x]) for x in range(n.value)]

    def share(self, keys, lists=None, lens=None):
        k = (ctypes.c_uint64 * self.n_mats)(*[int(x) for x in keys])
        lp = None if lists is None else np.ascontiguousarray(lists, dtype=np.int32)
        ln = None if lens is None else np.ascontiguousarray(lens, dtype=np.int32)
        _check(lib().cse_shard_share(self.handle, k,
                                     None if lp is None else lp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                     None if ln is None else ln.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))

    def run(self, group=None, device="cpu") -> "Shard":
        """Every round of the search, with the boundary exchange over the
        process group (torch.distributed) after each."""
        while True:
            keys, left = self.round()
            if left == 0:
                return self
            gk, lists, lens = exchange_boundary(keys, self.best_list, self.cap, group, device)
            self.share(gk, lists, lens)


class Server:
    """Continuous-batching server (cse_server_*)."""

    def __init__(self, interval: int = 32, permille: int = 400, cap: int = 128, hbm_budget: int = 0,
                 max_active_processes: int = 0, procs_per_cta: int = 0, trace: bool = False,
                 gi_shared: bool = False):
        h = ctypes.c_void_p()
        opts = make_opts(interval, permille, cap, procs_per_cta, trace=trace, gi_shared=gi_shared)
        _check(lib().cse_server_create(ctypes.byref(opts),
                                       hbm_budget,
                                       max_active_processes, ctypes.byref(h)))
        self.handle = h
        self.cap = cap
        self._keep = {}

    def submit(self, scheme: Scheme, weights, n_proc: int, seed: int, budget: int) -> int:
        t = ctypes.c_uint64()
        _check(lib().cse_server_submit(self.handle, scheme.handle, ctypes.byref(make_mix(weights)), n_proc, seed,
                                       budget, ctypes.byref(t)))
        self._keep[t.value] = (scheme, n_proc)
        return t.value

    def cancel(self, ticket: int) -> None:
        """cse_server_cancel: wait() on the ticket then raises CSE_ECANCELED."""
        _check(lib().cse_server_cancel(self.handle, ticket))

    def wait(self, ticket: int, timeout_us: int = -1) -> Result:
        h = ctypes.c_void_p()
        rc = lib().cse_server_wait(self.handle, ticket, timeout_us, ctypes.byref(h))
        if rc != CSE_OK:
            if rc != CSE_ETIMEOUT:  # the ticket is consumed: release its inputs
                self._keep.pop(ticket, None)
            _check(rc)
        scheme, n_proc = self._keep.pop(ticket)
        r = Result(h, len(scheme.mats), n_proc, self.cap)
        r._scheme = scheme
        return r

    def stats(self):
        a, b, c, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
        _check(lib().cse_server_stats(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(n)))
        return {"p50_ms": a.value, "p99_ms": b.value, "steps_per_s": c.value, "completed": n.value}

    def peak(self):
        """cse_server_peak: (most searches active in one round, rounds run)."""
        a, b = ctypes.c_int32(), ctypes.c_int32()
        _check(lib().cse_server_peak(self.handle, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def free(self):
        if getattr(self, "handle", None):
            lib().cse_server_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
