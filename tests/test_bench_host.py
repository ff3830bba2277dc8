"""Host-side parts of bench.py that need no GPU: the multi-rank aggregation
(world size 2 over gloo on the CPU, as the benchmark does over NCCL with one
rank per GPU) and the CPU reference arm."""
import json
import os
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, bench.whole_job_rate(1000, world, ms)))


def test_max_over_ranks_and_weak_scaling_rate_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the slowest rank's time; the job rate counts both ranks' work
    assert [g[1] for g in got] == [15.0, 15.0]
    assert got[0][2] == pytest.approx(2 * 1000 / 0.015)


def test_single_process_aggregation_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, "cpu") == 3.5
    assert bench.whole_job_rate(100, 1, 2.0) == pytest.approx(50000.0)


def test_reference_arm_prints_one_line_on_cpu():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--cpu-budget", "2"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0


def test_clock_record_keeps_timed_region_samples(tmp_path):
    """The clock record keeps the nvidia-smi samples time-stamped inside the
    timed region (widened by one 100 ms period), with their throttle reasons."""
    import datetime
    import time
    sys.path.insert(0, ROOT)
    import bench

    class Proc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    now = time.time()
    path = tmp_path / "clocks.csv"
    with open(path, "w") as f:
        for k in range(8):
            ts = datetime.datetime.fromtimestamp(now + 0.1 * k).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
            cap = "Active" if k == 7 else "Not Active"
            f.write(f"0, {1500 + 50 * k}, 2070, 500.0, 0x0, Not Active, Not Active, Not Active, {cap}, {ts}\n")
    c = bench.Clocks.__new__(bench.Clocks)
    c.path, c.p, c.t0, c.t1 = str(path), Proc(), None, None
    c.f = open(os.devnull, "w")
    whole = c.stop()
    assert whole["samples"] == 8 and whole["reasons"] == ["sw_power_cap"] and whole["scope"] == "whole run"
    c.f = open(os.devnull, "w")
    c.window(now + 0.25, now + 0.45)
    got = c.stop()
    assert got["samples"] == 4 and got["sm_mhz"] == 1675.0 and got["reasons"] == []
    assert got["scope"] == "timed region" and got["sm_max_mhz"] == 2070.0


def test_measured_traffic_only_for_the_captured_workload(tmp_path):
    """The DRAM traffic of an ncu capture is reported only on the line of the
    workload it was taken on, for the current kernel source, scaled from the
    captured launch to the bench's process count."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2512_13365_gb300 import synth
    s4 = synth.config4(n_proc=4096, budget=64)
    rec = [{"kernel_source_sha256_prefix": bench.kernel_source_sha(), "workload_name": s4.name,
            "n_processes": 4096, "share_interval": 32, "dram_bytes_per_launch": 1000}]
    path = tmp_path / "traffic.json"
    path.write_text(json.dumps(rec))
    assert bench.measured_traffic(s4, str(path)) == 1000
    s4.n_proc = 65536
    assert bench.measured_traffic(s4, str(path)) == 16000
    assert bench.measured_traffic(synth.config2(), str(path)) is None
    rec[0]["kernel_source_sha256_prefix"] = "0" * 16
    path.write_text(json.dumps(rec))
    assert bench.measured_traffic(s4, str(path)) is None


def test_reference_arm_under_torchrun_prints_once():
    """Launched as the multi-GPU benchmark is (torchrun, two ranks on
    127.0.0.1), the reference arm runs on rank 0 alone, prints one line, and
    the other rank exits 0 without work."""
    port = 29700 + os.getpid() % 200
    out = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                          "--master-addr", "127.0.0.1", "--master-port", str(port),
                          os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
                          "--warmup", "0", "--cpu-budget", "2"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
