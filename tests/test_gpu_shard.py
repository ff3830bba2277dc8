"""One search split across ranks: two gloo ranks on one GPU each run a shard
(half the processes) and exchange the round minima and winner lists at every
sharing boundary on the host.  The union must be the unsharded search, bit
for bit: the result, the best-Cost curve, and every process's record.  The
ranks' kernels never wait on each other; only the host exchange does."""
import os
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2512_13365_gb300 import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _shard_rank(rank, world, port, which, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_2512_13365_gb300 import cse, synth as sy
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s = _workload(sy, which)
    sc = cse.Scheme(s.mats)
    sh = cse.Shard(sc, s.weights, s.n_proc, rank, world, s.seed, s.budget, s.interval, s.permille, s.cap,
                   trace=True).run()
    out = {"costs": sh.costs, "lists": sh.lists, "curves": [sh.curve(k) for k in range(len(s.mats))],
           "procs": [sh.procs(k).tobytes() for k in range(len(s.mats))], "counters": sh.counters(),
           "mops": sh.method_ops()}
    sh.free()
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, out))


def _workload(sy, which):
    if which == "small":
        return sy.config2(n_proc=201, budget=160)
    s = sy.config4(n_proc=13, budget=64)
    s.interval = 16
    return s


@pytest.mark.parametrize("which", ["small", "large"])
def test_two_shards_equal_the_whole_search(which):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2512_13365_gb300 import cse
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29800 + os.getpid() % 90 + (0 if which == "small" else 7)
    ps = [ctx.Process(target=_shard_rank, args=(r, 2, port, which, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = dict(q.get(timeout=600) for _ in ps)
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    s = _workload(synth, which)
    whole = cse.search_obj(s, trace=True)
    for rank in (0, 1):
        assert got[rank]["costs"] == whole.costs and got[rank]["lists"] == whole.lists
        assert got[rank]["curves"] == [whole.curve(k) for k in range(len(s.mats))]
    for k in range(len(s.mats)):
        parts = [np.frombuffer(got[r]["procs"][k], dtype=cse.PROC_DTYPE) for r in (0, 1)]
        assert np.array_equal(np.concatenate(parts), whole.procs(k))
    steps, sub, ops = whole.counters()
    assert sum(got[r]["counters"][1] for r in (0, 1)) == sub
    assert sum(got[r]["counters"][2] for r in (0, 1)) == ops
    assert sum(got[r]["mops"] for r in (0, 1)) == whole.method_ops()
    whole.free()
