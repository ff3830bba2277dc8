"""cse_search_static, the entry point for callers that may not allocate device
memory while they run a search (their device memory belongs to another
framework's pool, or an allocation could stall a latency-critical loop).
It must give exactly what cse_search gives, call after call, although every
call reuses the same static scratch array.

This file is collected last so that, if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2512_13365_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2512_13365_gb300 import cse
    return cse, torch


def _static(cse, torch, scheme, s):
    """One cse_search_static call through the C ABI; returns per matrix
    (best list, Cost) read from the caller-owned device buffers."""
    n = len(s.mats)
    lists = torch.full((n, s.cap), -1, dtype=torch.int32, device="cuda")
    meta = torch.full((n, 2), -1, dtype=torch.int32, device="cuda")
    rc = cse.lib().cse_search_static(scheme.handle, ctypes.byref(cse.make_mix(s.weights)), s.n_proc, s.seed,
                                     s.budget, ctypes.byref(cse.make_opts(s.interval, s.permille, s.cap)), None,
                                     ctypes.c_void_p(lists.data_ptr()), ctypes.c_void_p(meta.data_ptr()))
    assert rc == cse.CSE_OK, cse.lib().cse_last_error()
    lists, meta = lists.cpu().numpy(), meta.cpu().numpy()
    return [(list(lists[k, :meta[k, 1]]), int(meta[k, 0])) for k in range(n)]


def _reference(cse, scheme, s):
    r = cse.search(scheme, s.weights, s.n_proc, s.seed, s.budget, s.interval, s.permille, s.cap)
    out = [(r.fetch(k)[0], r.fetch(k)[1]) for k in range(len(s.mats))]
    r.free()
    return out


def test_static_scratch_matches_cse_search_on_consecutive_calls(env):
    cse, torch = env
    a = synth.config2(n_proc=256, budget=96)
    b = synth.config2(n_proc=200, budget=70)
    b.seed = 7
    sa, sb = cse.Scheme(a.mats), cse.Scheme(b.mats)
    ra, rb = _reference(cse, sa, a), _reference(cse, sb, b)
    assert _static(cse, torch, sa, a) == ra   # first call (sets up the scratch address)
    assert _static(cse, torch, sb, b) == rb   # second call: a different search on stale scratch
    assert _static(cse, torch, sa, a) == ra   # and back


def test_static_scratch_large_matrices(env):
    cse, torch = env
    s = synth.config4(n_proc=8, budget=40)
    s.interval = 16
    sc = cse.Scheme(s.mats)
    ref = _reference(cse, sc, s)
    assert _static(cse, torch, sc, s) == ref
    assert _static(cse, torch, sc, s) == ref


def test_static_scratch_refuses_searches_that_do_not_fit(env):
    cse, torch = env
    s = synth.config2(n_proc=65536, budget=10)
    sc = cse.Scheme(s.mats)
    lists = torch.zeros((3, s.cap), dtype=torch.int32, device="cuda")
    meta = torch.zeros((3, 2), dtype=torch.int32, device="cuda")
    rc = cse.lib().cse_search_static(sc.handle, ctypes.byref(cse.make_mix(s.weights)), s.n_proc, s.seed,
                                     s.budget, ctypes.byref(cse.make_opts(s.interval, s.permille, s.cap)), None,
                                     ctypes.c_void_p(lists.data_ptr()), ctypes.c_void_p(meta.data_ptr()))
    assert rc == cse.CSE_ENOMEM
    assert b"static scratch holds" in cse.lib().cse_last_error()


def test_static_scratch_refuses_the_graph_flag(env):
    """The no-allocation entry point runs its own launch sequence and takes no
    CSE_FLAG_GRAPH: the flag is refused instead of being ignored."""
    cse, torch = env
    s = synth.config1(n_proc=8, budget=8)
    sc = cse.Scheme(s.mats)
    lists = torch.zeros((2, s.cap), dtype=torch.int32, device="cuda")
    meta = torch.zeros((2, 2), dtype=torch.int32, device="cuda")
    rc = cse.lib().cse_search_static(sc.handle, ctypes.byref(cse.make_mix(s.weights)), s.n_proc, s.seed,
                                     s.budget, ctypes.byref(cse.make_opts(s.interval, s.permille, s.cap, graph=True)),
                                     None, ctypes.c_void_p(lists.data_ptr()), ctypes.c_void_p(meta.data_ptr()))
    assert rc == cse.CSE_EINVAL
    assert b"CSE_FLAG_GRAPH" in cse.lib().cse_last_error()
