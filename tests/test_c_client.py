"""The C ABI used from plain C: tests/c_client.c is compiled with gcc against
include/cse.h and linked to the library; on the CPU it runs the argument
checks (and sees the no-device status), on the GPU it runs a search whose
result equals the Python binding's and the oracle's."""
import os
import struct
import subprocess

import numpy as np
import pytest

from paper_2512_13365_gb300 import build as B
from paper_2512_13365_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    lib = B.build()
    exe = str(tmp_path_factory.mktemp("c_client") / "c_client")
    subprocess.check_call(["gcc", "-std=c11", "-O1", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "c_client.c"), "-o", exe, lib,
                           "-Wl,-rpath," + os.path.dirname(lib)])
    return exe


def test_c_client_argument_checks(client):
    import torch
    out = subprocess.run([client, "checks"], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and "checks ok" in out.stdout, out.stdout
    if not torch.cuda.is_available():
        assert "device 3" in out.stdout   # CSE_ECUDA: no host path computes anything


def test_binding_structs_match_the_header(client):
    """The ctypes records of the binding have the sizes and field offsets
    that a C compiler gives the header's structs."""
    import ctypes
    from paper_2512_13365_gb300 import cse
    out = subprocess.run([client, "sizes"], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stdout
    c = {ln.split()[0]: (int(ln.split()[1]), int(ln.split()[2])) for ln in out.stdout.splitlines()}
    py = {"cse_strategy_mix": (cse.Mix, "w_gp"), "cse_opts": (cse.Opts, "cta_min_list"),
          "cse_tune_entry": (cse.TuneEntry, "trial_ms_wide"), "cse_proc_record": (cse.ProcRecord, "method_ops")}
    assert set(c) == set(py)
    for name, (cls, last) in py.items():
        assert (ctypes.sizeof(cls), getattr(cls, last).offset) == c[name], name


def _write(path, s):
    with open(path, "wb") as f:
        w = list(s.weights) + [0] * (7 - len(s.weights))
        f.write(struct.pack("<15i", len(s.mats), s.n_proc, s.seed & 0xFFFFFFFF, s.seed >> 32, s.budget,
                            s.interval, s.permille, s.cap, *w))
        for m in s.mats:
            f.write(struct.pack("<2i", *m.shape))
            f.write(np.ascontiguousarray(m, dtype=np.int8).tobytes())


@pytest.mark.gpu
def test_c_client_search_equals_binding_and_oracle(client, tmp_path):
    from oracle import oracle as O
    from paper_2512_13365_gb300 import cse
    s = synth.config2(n_proc=256, budget=96)
    path = str(tmp_path / "search.bin")
    _write(path, s)
    out = subprocess.run([client, "search", path], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout
    lines = out.stdout.splitlines()
    total = int(lines[0].split()[1])
    costs, lists = [], []
    for ln in lines[1:]:
        f = ln.split()
        costs.append(int(f[3]))
        lists.append([int(x) for x in f[5:]])
    r = cse.search_obj(s)
    assert costs == r.costs and lists == r.lists and total == sum(r.costs)
    ref = O.search_obj(s, n_threads=8)
    assert costs == ref.cost and lists == ref.lists
