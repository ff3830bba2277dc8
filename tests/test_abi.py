"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function include/cse.h declares, and rejects invalid arguments before
touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2512_13365_gb300 import build as B
from paper_2512_13365_gb300 import cse

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return cse.lib()


def declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(cse_\w+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(L):
    names = declared()
    assert len(names) >= 12
    for n in sorted(names):
        assert hasattr(L, n), n
    assert names == set(cse.EXPORTS)


def _load(mats):
    n = len(mats)
    mats = [np.ascontiguousarray(m, dtype=np.int8) for m in mats]
    ptrs = (ctypes.POINTER(ctypes.c_int8) * n)(*[m.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)) for m in mats])
    rows = (ctypes.c_int32 * n)(*[m.shape[0] for m in mats])
    cols = (ctypes.c_int32 * n)(*[m.shape[1] for m in mats])
    h = ctypes.c_void_p()
    rc = cse.lib().cse_scheme_load(ptrs, rows, cols, n, ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("bad", [
    [np.array([[2, 1]])],                      # not ternary
    [np.array([[1, 1], [0, 0]])],              # zero row
    [np.zeros((257, 3), np.int8) + 1],         # too many rows
    [np.ones((2, 512), np.int8)],              # too many columns
])
def test_scheme_load_rejects_invalid(L, bad):
    rc, h = _load(bad)
    assert rc == cse.CSE_EINVAL and not h.value
    assert L.cse_last_error()


def test_search_rejects_invalid_arguments_without_device(L):
    # argument checks come before any CUDA call; a NULL scheme is rejected
    mix = cse.make_mix((1, 0, 0, 0, 0, 0))
    opts = cse.make_opts()
    h = ctypes.c_void_p()
    assert L.cse_search(None, ctypes.byref(mix), 4, 0, 10, ctypes.byref(opts), None, ctypes.byref(h)) == \
        cse.CSE_EINVAL
    assert L.cse_result_fetch(None, 0, None, 0, None, None, None) == cse.CSE_EINVAL


def test_opts_default(L):
    o = cse.Opts()
    L.cse_opts_default(ctypes.byref(o))
    assert (o.share_interval, o.share_permille, o.col_cap, o.flags) == (32, 400, 128, 0)


@pytest.mark.parametrize("interval,patience,graph,msg", [
    (32, 3, False, b"patience_rounds applies to iteration mode"),
    (0, 10, True, b"cannot be captured in a graph"),
])
def test_iteration_mode_option_checks_without_device(L, interval, patience, graph, msg):
    dummy = ctypes.c_void_p(1)   # never dereferenced: the options are checked first
    schemes = (ctypes.c_void_p * 1)(dummy)
    mixes = (cse.Mix * 1)(cse.make_mix((1, 0, 0, 0, 0, 0)))
    n_proc = (ctypes.c_int32 * 1)(4)
    seeds = (ctypes.c_uint64 * 1)(0)
    budgets = (ctypes.c_int64 * 1)(10)
    opts = cse.make_opts(interval=interval, graph=graph, patience=patience)
    outs = (ctypes.c_void_p * 1)()
    rc = L.cse_search_batch(1, schemes, mixes, n_proc, seeds, budgets, ctypes.byref(opts), None, outs)
    assert rc == cse.CSE_EINVAL and msg in L.cse_last_error()


def test_server_rejects_iteration_mode_without_device(L):
    opts = cse.make_opts(interval=0, patience=10)
    h = ctypes.c_void_p()
    assert L.cse_server_create(ctypes.byref(opts), 0, 0, ctypes.byref(h)) == cse.CSE_EINVAL
    assert b"share_interval >= 1" in L.cse_last_error()


def test_brent_and_hybrid_argument_checks_without_device(L):
    out = ctypes.c_int64()
    a = np.ones(4, np.int8)
    assert L.cse_brent_check(0, 2, 2, 1, a.ctypes.data, a.ctypes.data, a.ctypes.data, ctypes.byref(out)) == \
        cse.CSE_EINVAL
    assert L.cse_brent_check(2, 2, 2, 1, None, a.ctypes.data, a.ctypes.data, ctypes.byref(out)) == cse.CSE_EINVAL
    assert L.cse_brent_check(100, 100, 2, 1, a.ctypes.data, a.ctypes.data, a.ctypes.data, ctypes.byref(out)) == \
        cse.CSE_EINVAL
    best = (ctypes.c_int32 * 3)()
    assert L.cse_result_hybrid(None, 2, best, None) == cse.CSE_EINVAL


def test_philox_argument_checks_without_device(L):
    c = np.zeros(8, np.uint32)
    assert L.cse_philox(0, c.ctypes.data, -1, c.ctypes.data) == cse.CSE_EINVAL
    assert L.cse_philox(0, c.ctypes.data, (1 << 24) + 1, c.ctypes.data) == cse.CSE_EINVAL
    assert L.cse_philox(0, None, 2, c.ctypes.data) == cse.CSE_EINVAL
    assert L.cse_philox(0, c.ctypes.data, 2, None) == cse.CSE_EINVAL
    assert b"NULL" in L.cse_last_error()
    # n = 0 touches neither array nor the device
    assert L.cse_philox(0, None, 0, None) == cse.CSE_OK


def test_resume_rejects_foreign_data_without_device(L):
    bogus = ctypes.create_string_buffer(b"\0" * 4096, 4096)
    h = ctypes.c_void_p()
    dummy = ctypes.c_void_p(1)   # never dereferenced: the header is checked first
    assert L.cse_search_resume(dummy, bogus, 4096, 10, None, None, ctypes.byref(h)) == cse.CSE_EINVAL
    assert b"not a checkpoint" in L.cse_last_error()
    assert L.cse_search_resume(dummy, bogus, 8, 10, None, None, ctypes.byref(h)) == cse.CSE_EINVAL


def test_binding_fails_loudly_without_the_library(tmp_path):
    """No CPU fallback: with the compiled library absent, the binding raises
    instead of computing anything."""
    import subprocess
    import sys
    code = ("from paper_2512_13365_gb300 import cse\n"
            "try:\n    cse.lib()\nexcept ImportError as e:\n    print('refused:', e)\n")
    env = dict(os.environ, CSE_GB300_LIB=str(tmp_path / "absent.so"))
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=120)
    assert out.returncode == 0 and "refused:" in out.stdout and "is not built" in out.stdout


def test_device_calls_report_no_device(L):
    """On a machine without a GPU the calls that need one return CSE_ECUDA:
    there is no host path that would compute a result."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    m = np.array([[1, 1, 0], [1, 1, 1], [0, 1, 1]], np.int8)
    ptrs = (ctypes.POINTER(ctypes.c_int8) * 1)(m.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)))
    rows = (ctypes.c_int32 * 1)(3)
    cols = (ctypes.c_int32 * 1)(3)
    h = ctypes.c_void_p()
    assert L.cse_scheme_load(ptrs, rows, cols, 1, ctypes.byref(h)) == cse.CSE_ECUDA
    assert not h.value
    c = np.zeros(4, np.uint32)
    assert L.cse_philox(0, c.ctypes.data, 1, c.ctypes.data) == cse.CSE_ECUDA


def test_options_record_mirrors_cse_opts(L):
    """cse.Options has the library's defaults and round-trips through the C
    struct, flags included."""
    assert cse.Options.library_default() == cse.Options()
    o = cse.Options(share_interval=0, share_permille=1000, col_cap=512, patience_rounds=10, procs_per_cta=3,
                    graph=False, trace=True, gi_shared=True)
    st = o.to_struct()
    assert st.flags == cse.FLAG_TRACE | cse.FLAG_GI_SHARED_COINS and st.max_spin == 0
    assert cse.Options.from_struct(st) == o
