"""The sharing-boundary exchange of a search split across ranks, on the CPU:
two gloo ranks, each holding its shard's round keys and best lists, must
agree on the minimum key of every matrix (lowest Cost, then lowest global
process) and receive the winner's list from the rank that owns it."""
import os
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# rank r owns the global processes [10 r, 10 r + 10)
KEYS = {0: [(50 << 32) | 3, (40 << 32) | 7, (30 << 32) | 9],
        1: [(45 << 32) | 12, (41 << 32) | 15, (30 << 32) | 11]}
LISTS = {3: [1, 2, 3], 7: [4, 5], 9: [6], 12: [7, 8, 9, 10], 15: [11], 11: [12, 13]}


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2512_13365_gb300 import cse
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b, n = cse.shard_range(20, rank, world)

    def best_list(k, key):
        p = key & 0xFFFFFFFF
        return LISTS[p] if b <= p < b + n else None

    gk, lists, lens = cse.exchange_boundary(KEYS[rank], best_list, cap=8)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, [int(x) for x in gk], lists.tolist(), lens.tolist()))


def test_boundary_exchange_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29900 + os.getpid() % 90
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    want_keys = [(45 << 32) | 12, (40 << 32) | 7, (30 << 32) | 9]   # ties on Cost go to the lower process
    for rank, keys, lists, lens in got:
        assert keys == want_keys
        assert lens == [4, 2, 1]
        assert [row[:n] for row, n in zip(lists, lens)] == [[7, 8, 9, 10], [4, 5], [6]]
        assert all(x == 0 for row, n in zip(lists, lens) for x in row[n:])


def test_shard_ranges_cover_the_processes():
    sys.path.insert(0, ROOT)
    from paper_2512_13365_gb300 import cse
    for n, world in ((7, 2), (4096, 3), (65536, 8), (5, 5)):
        got = [cse.shard_range(n, r, world) for r in range(world)]
        assert got[0][0] == 0 and all(c >= 1 for _, c in got)
        assert all(got[r][0] + got[r][1] == got[r + 1][0] for r in range(world - 1))
        assert got[-1][0] + got[-1][1] == n
