"""Benchmark: CSE process-steps/s of the GB300 library on the largest
single-GPU workload, a synthetic (6,6,6:153)-shaped scheme (E_U, E_V 153 x 36,
E_W 36 x 153, variables grown to 512; 65536 processes per matrix, mixed
strategies, sharing every 32 steps, 2000 steps).  `--workload cfg2` runs the
(3,3,3:23)-shaped scheme (4096 processes, 1024 steps) instead.

One benchmark step = one complete search (cse_search) over that workload.
`value` is timed on the device with CUDA events, inputs resident in HBM;
`e2e` times the public C-ABI sequence a user runs (load from host buffers,
search, fetch results to the host).  The roofline's numerator is the
method's own op count (cse_result_method_ops) and its peak the integer-pipe
rate measured by cse_int_peak on this GPU at the clock sampled during the
timed region.  `--impl reference` times the CPU oracle on a bounded sample of
the same workload.
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CSE process-steps/s & best additions @ fixed budget vs oracle; p50/p99 latency"
UNIT = "process-steps/s"
SM_COUNT_NOMINAL = 152
LANES_PER_SM = 128  # 4 schedulers x 32 lanes: one warp instruction per scheduler per clock (derived, not measured)
# bounded oracle samples (processes per matrix, steps) of each workload: about
# 10-30 s of host work for the CPU baseline, a few seconds per reference step
CPU_SAMPLE = {"cfg4": (48, 64), "cfg2": (4096, 1024), "cfg1": (64, 200)}
REF_SAMPLE = {"cfg4": (32, 16), "cfg2": (4096, 128), "cfg1": (64, 200)}


def measured_int_peak(stream, iters: int = 100000):
    """cse_int_peak on this GPU: lane-ops per SM clock of the integer mixes
    (LOP3 + IADD3, AND + POPC + IADD, IMAD, IMAD.HI, LOP3 alone, IADD3 alone)."""
    from paper_2512_13365_gb300 import cse
    out = {}
    for kind in range(6):
        cse.int_peak(kind, 1000, stream)  # warm-up
        r = cse.int_peak(kind, iters, stream)
        out[r["kind"]] = round(r["ops_per_clk_per_sm"], 2)
    return out


def roofline(ops_per_launch, avg_launch_ms, eng_ops_per_launch, peak_clk, sms, clk, traffic, kernel):
    """Roofline of the round kernels against the measured integer peak: the
    best plain-integer rate cse_int_peak measured (LOP3 / IADD3 lane-ops per
    SM clock) x SMs x the median SM clock sampled in the timed region (the
    maximum clock if no sample)."""
    mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0
    per_clk = max(peak_clk[k] for k in ("lop3+iadd3", "lop3", "iadd3"))
    peak = per_clk * sms * mhz * 1e6 / 1e12
    achieved = ops_per_launch / (avg_launch_ms / 1000.0) / 1e12
    eng = eng_ops_per_launch / (avg_launch_ms / 1000.0) / 1e12
    derived = sms * LANES_PER_SM * mhz * 1e6 / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
            "frac_s8d": achieved / peak,
            "numerator": "method ops (cse_result_method_ops): 6 per 64-bit word + nnz of the rewritten rows per "
                         "rewrite, m per selection, 2 per Greedy-Intersections intersect term",
            "peak_source": f"measured by cse_int_peak: {per_clk:.1f} integer (LOP3/IADD3) lane-ops per SM clock, the "
                           f"best of its plain-integer mixes, x {sms} SMs x {mhz:.0f} MHz (median SM clock of the "
                           f"timed region)",
            "measured_ops_per_clk_per_sm": peak_clk,
            "engine_weighted": {"achieved": eng, "frac": eng / peak,
                                "definition": "cse_result_counters alg_ops (10W per rewrite, 5W per changed "
                                              "pair count, 3 per gi term + 8 + 40 per Philox block)"},
            "derived_peak_note": f"{sms} SMs x {LANES_PER_SM} lanes x {mhz:.0f} MHz = {derived:.2f} T (not used)",
            "traffic": traffic,
            "traffic_unit": "bytes per launch (dram read + write; ncu capture of this kernel source, scaled by "
                            "processes when taken on a smaller launch)",
            "kernel": kernel, "alg_ops_per_launch": ops_per_launch, "avg_launch_ms": avg_launch_ms}


def workload(name: str, procs: int = 0):
    from paper_2512_13365_gb300 import synth
    if name == "cfg1":
        s = synth.config1()
    elif name == "cfg2":
        s = synth.config2()
    elif name == "cfg4":
        s = synth.config4()
    else:
        raise SystemExit(f"unknown workload {name}")
    if procs:
        s.n_proc = procs
    return s


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, out_path: str, index: int):
        self.path = out_path
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,timestamp")
        self.t0 = self.t1 = None
        try:
            self.f = open(out_path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None
            return
        # nvidia-smi takes a moment to start: wait (at most 3 s) for its first
        # sample so that the timed region is covered from its start
        deadline = time.time() + 3.0
        while time.time() < deadline and self.p.poll() is None:
            if os.path.getsize(out_path) > 0:
                break
            time.sleep(0.02)

    def window(self, t0: float, t1: float):
        """The timed region in host wall-clock seconds (time.time())."""
        self.t0, self.t1 = t0, t1

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.close()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for ln in open(self.path):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                mhz, mx = float(f[1]), float(f[2])
            except ValueError:
                continue
            ts = None
            if len(f) >= 10:
                try:
                    ts = datetime.datetime.strptime(f[9], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                except ValueError:
                    ts = None
            rows.append((ts, mhz, mx, [n for n, v in zip(names, f[5:9]) if v.lower().startswith("active")]))
        scope = "whole run"
        if self.t0 is not None:
            # samples inside the timed region, widened by one sampling period
            inside = [r for r in rows if r[0] is not None and self.t0 - 0.1 <= r[0] <= self.t1 + 0.1]
            if inside:
                rows, scope = inside, "timed region"
        sm = [r[1] for r in rows]
        reasons = sorted({n for r in rows for n in r[3]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(r[2] for r in rows) if rows else None,
                "reasons": reasons, "samples": len(sm), "scope": scope}


def max_over_ranks(x: float, device) -> float:
    """The largest value of x over all ranks (the slowest rank's time); x on
    a single process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, max_ms: float) -> float:
    """Weak scaling: every rank runs its own search of the same size, so the
    job processes world * units in the slowest rank's time."""
    return units_per_rank * world / (max_ms / 1000.0)


def kernel_source_sha() -> str:
    """sha256 prefix of the round kernels' sources (the engines and their units)."""
    import hashlib
    h = hashlib.sha256()
    for f in ("cse_engine.cuh", "cse_kernels.cu", "cse_cta.cuh", "cse_kernels_cta.cu", "cse_internal.h"):
        with open(os.path.join(ROOT, "paper_2512_13365_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(s, path=None):
    """DRAM bytes per launch of the round kernels from the ncu capture of the
    current kernel source on this workload (search s), scaled to s's process
    count when the capture was taken on a smaller launch (each process reads
    and writes its own state, so the traffic grows with the processes); else
    None."""
    try:
        rec = json.load(open(path or os.path.join(ROOT, "profiles", "round_kernel_traffic.json")))
        sha = kernel_source_sha()
    except (OSError, ValueError):
        return None
    recs = rec if isinstance(rec, list) else [rec]
    for r in recs:
        if (r.get("kernel_source_sha256_prefix") == sha and r.get("workload_name") == s.name and
                r.get("share_interval") == s.interval):
            # the state each launch reads and writes grows with the process count
            return int(r["dram_bytes_per_launch"] * s.n_proc / r["n_processes"])
    return None


def flush_l2(buf):
    buf.zero_()


def run_ours(args):
    import torch
    from paper_2512_13365_gb300 import cse

    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    s = workload(args.workload, args.procs)
    if args.budget:
        s.budget = args.budget
    s.seed = s.seed + rank  # weak scaling: each rank searches its own seed, no data-path collective
    stream = torch.cuda.Stream(device=dev)
    scheme = cse.Scheme(s.mats)
    l2 = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def one():
        return cse.search(scheme, s.weights, s.n_proc, s.seed, s.budget, s.interval, s.permille, s.cap,
                          stream=stream, procs_per_cta=args.ppc, gi_shared=args.gi_shared,
                          warp_engine=args.warp_engine, cta_min_list=args.cta_min_list,
                          cta_engine=args.cta_engine)

    for _ in range(args.warmup):
        r = one()
        r.fetch(0)
        r.free()
    peak_clk = measured_int_peak(stream)
    clocks = Clocks(os.path.join(args.out, f"clocks_rank{rank}.csv"), local)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    evs = []
    results = []
    t_wall = time.perf_counter()
    tw0 = time.time()
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush_l2(l2)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = one()
        b.record(stream)
        evs.append((a, b))
        results.append(r)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - t_wall
    clocks.window(tw0, time.time())
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    round_ms, n_rounds, ops_total, mops_total = [], 0, 0, 0
    for r in results:
        rm, tm, nr = r.timing()
        round_ms.append(rm)
        n_rounds = nr
        steps, sub, ops = r.counters()
        ops_total = ops
        mops_total = r.method_ops()
    kernels_per_search = results[-1].launches()[0]
    total = results[-1].total
    costs = results[-1].costs
    # the best-additions curve (sum over matrices, one point per round) and
    # which strategies produced the processes' best records
    curves = [results[-1].curve(k) for k in range(len(s.mats))]
    curve = [sum(c[i] for c in curves) for i in range(min(len(c) for c in curves))]
    wins = [0] * len(cse.STRATEGIES)
    for k in range(len(s.mats)):
        bs = results[-1].procs(k)["best_strategy"]
        for v in bs[bs >= 0]:
            wins[int(v)] += 1
    for r in results:
        r.free()
    ms = max_over_ranks(statistics.mean(step_ms), dev)
    psteps = s.process_steps()
    value = whole_job_rate(psteps, world, ms)

    # end to end through the public API: host buffers in, results to the host
    e2e_ms = []
    h2d = sum(m.nbytes for m in s.mats)
    d2h = 0
    # the inputs sit in pinned host memory, as a serving host would keep them
    pinned = [torch.from_numpy(m).pin_memory().numpy() for m in s.mats]
    n_e2e = 1 if statistics.mean(step_ms) > 5000 else max(1, min(args.steps, 3))
    for it in range(0 if args.no_e2e else n_e2e):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sc = cse.Scheme(pinned)
        r = cse.search(sc, s.weights, s.n_proc, s.seed, s.budget, s.interval, s.permille, s.cap, stream=stream,
                       procs_per_cta=args.ppc, gi_shared=args.gi_shared, warp_engine=args.warp_engine,
                       cta_min_list=args.cta_min_list, cta_engine=args.cta_engine)
        lists = [r.fetch(k) for k in range(len(s.mats))]
        e2e_ms.append((time.perf_counter() - t0) * 1000.0)
        d2h = sum(4 * len(l) + 16 for l, _, _ in lists)
        r.free()
        sc.free()
    e2e_value = None
    if e2e_ms:
        e2e_value = whole_job_rate(psteps, world, max_over_ranks(statistics.mean(e2e_ms), dev))

    # roofline of the dominant kernel (the round kernels)
    props = torch.cuda.get_device_properties(dev)
    avg_round_ms = statistics.mean(round_ms) / n_rounds

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": s.name + (" (shared gi coins)" if args.gi_shared else ""),
                   "matrices": [list(m.shape) for m in s.mats], "n_processes": s.n_proc,
                   "step_budget": s.budget, "share_interval": s.interval, "share_permille": s.permille,
                   "col_cap": s.cap, "strategy_weights_gi_ga_gr_wr_mix_g_gp": list(s.weights),
                   "process_steps_per_step": psteps,
                   "l2": "flushed (256 MB write) between timed steps; the per-process state is larger than L2"
                         if s.n_proc * len(s.mats) > 100000 else "flushed (256 MB write) between timed steps",
                   "parallelism": f"{world} independent searches (one per GPU)"},
        "best_additions": total, "best_additions_per_matrix": costs,
        "best_additions_per_round": curve,
        "best_records_by_strategy": dict(zip(cse.STRATEGIES, wins)),
        "wall_s": wall,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": statistics.mean(e2e_ms) if e2e_ms else None, "inputs": "pinned host memory"},
        "roofline": roofline(mops_total / n_rounds, avg_round_ms, ops_total / n_rounds, peak_clk,
                             props.multi_processor_count, clk, None if args.gi_shared else measured_traffic(s),
                             "round_kernel (all matrix classes of a round; one launch per class)"),
        "clocks": clk,
        "gpu_launches": kernels_per_search * args.steps,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(s, args.workload, args.cpu_budget, args.gi_shared)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


def cpu_baseline(s, wl, budget=0, gi_shared=False):
    """The oracle, as it stands, on a bounded sample of the same workload
    (about 10-30 s on the host cores): the first processes and steps of the
    search, on every host core; process-steps/s of that sample."""
    from oracle import oracle as O
    import copy
    cores = len(os.sched_getaffinity(0))
    procs, steps = CPU_SAMPLE.get(wl, (s.n_proc, s.budget))
    smp = copy.copy(s)
    smp.n_proc = min(procs, s.n_proc)
    smp.budget = budget or min(steps, s.budget)
    t0 = time.perf_counter()
    ref = O.search_obj(smp, n_threads=cores, digests=False, flags=O.GI_SHARED_COINS if gi_shared else 0)
    dt = time.perf_counter() - t0
    out = {"value": smp.process_steps() / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{s.name}: first {smp.n_proc} of {s.n_proc} processes x {len(s.mats)} matrices, first "
                     f"{smp.budget} of {s.budget} steps ({smp.process_steps()} process-steps, {dt:.1f} s)"}
    if smp.budget == s.budget and smp.n_proc == s.n_proc:
        out["best_additions"] = ref.total  # the same search on the CPU: equal to the GPU's by parity
    elif smp.n_proc < s.n_proc:
        out["note"] = ("the sample covers the earliest steps, where the candidate lists are longest; the rate is "
                       "not extrapolated to the whole search")
    # the same oracle on one thread, on a shorter sample (about 4 s)
    one = copy.copy(smp)
    one.n_proc = min(smp.n_proc, 8 if wl == "cfg4" else smp.n_proc)
    one.budget = min(smp.budget, 16 if wl == "cfg4" else 32)
    t0 = time.perf_counter()
    O.search_obj(one, n_threads=1, digests=False, flags=O.GI_SHARED_COINS if gi_shared else 0)
    dt1 = time.perf_counter() - t0
    out["single_thread"] = {"value": one.process_steps() / dt1, "unit": UNIT, "cores": 1,
                            "sample": f"first {one.budget} steps ({one.process_steps()} process-steps, {dt1:.1f} s)"}
    return out


def run_batched(args):
    """32 schemes of uneven shapes (config 3) in one CUDA-graph launch
    sequence, against one launch sequence per scheme on the same GPU."""
    import torch
    from paper_2512_13365_gb300 import cse, synth
    dev = torch.device("cuda", 0)
    searches = synth.config3()
    if args.budget:
        for s in searches:
            s.budget = args.budget
    cap = searches[0].cap
    schemes = [cse.Scheme(s.mats) for s in searches]
    ba = (schemes, [s.weights for s in searches], [s.n_proc for s in searches], [s.seed for s in searches],
          [s.budget for s in searches])
    stream = torch.cuda.Stream(device=dev)
    t0 = time.perf_counter()
    tuned = cse.autotune(*ba, interval=32, cap=cap, trial_steps=64, stream=stream)
    interval, _ = cse.tune_interval(*ba, candidates=(16, 32, 64), cap=cap, trial_steps=128, stream=stream)
    tune_s = time.perf_counter() - t0
    psteps = sum(s.process_steps() for s in searches)
    l2 = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def batched():
        rs = cse.search_batch(*ba, interval=interval, cap=cap, stream=stream, graph=True)
        return rs

    def persistent():
        return cse.search_batch(*ba, interval=interval, cap=cap, stream=stream, graph=True, persistent=True)

    def per_scheme():
        return [cse.search(sc, s.weights, s.n_proc, s.seed, s.budget, interval, s.permille, cap, stream=stream)
                for sc, s in zip(schemes, searches)]

    out = {}
    for name, fn in (("batched", batched), ("persistent", persistent), ("per_scheme", per_scheme)):
        for _ in range(args.warmup):
            for r in fn():
                r.free()
        ms = []
        totals = None
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush_l2(l2)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            rs = fn()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
            totals = [r.total for r in rs]
            kernels = rs[0].launches()[0] if name != "per_scheme" else sum(r.launches()[0] for r in rs)
            if name == "batched":
                round_ms, _, n_rounds = rs[0].timing()
                ops_total = sum(r.counters()[2] for r in rs)
                mops_total = sum(r.method_ops() for r in rs)
            for r in rs:
                r.free()
        out[name] = {"ms": statistics.mean(ms), "value": psteps / (statistics.mean(ms) / 1000.0),
                     "best_additions_total": sum(totals), "kernel_launches": kernels}
    assert out["batched"]["best_additions_total"] == out["per_scheme"]["best_additions_total"]
    assert out["persistent"]["best_additions_total"] == out["per_scheme"]["best_additions_total"]

    # best additions at a fixed wall-clock budget: the per-scheme launches get
    # the step budget B; the batched graph gets as many steps (a multiple of
    # the sharing interval) as fit in the same device time
    B = searches[0].budget
    wall = out["per_scheme"]["ms"]
    B2 = max(B, int(B * wall / out["batched"]["ms"]) // interval * interval)
    fixed = None
    while B2 >= B:
        ba2 = ba[:4] + ([B2] * len(searches),)
        with torch.cuda.stream(stream):
            flush_l2(l2)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rs = cse.search_batch(*ba2, interval=interval, cap=cap, stream=stream, graph=True)
        b.record(stream)
        torch.cuda.synchronize()
        t2 = a.elapsed_time(b)
        tot2 = sum(r.total for r in rs)
        for r in rs:
            r.free()
        if t2 <= wall or B2 == B:
            fixed = {"device_ms_budget": wall,
                     "one_launch_sequence_per_scheme": {"step_budget": B,
                                                        "best_additions_total": out["per_scheme"]["best_additions_total"]},
                     "batched_graph": {"step_budget": B2, "ms": t2, "best_additions_total": tot2}}
            break
        B2 -= interval
    props = torch.cuda.get_device_properties(dev)
    peak_clk = measured_int_peak(stream)
    # the oracle on the same batch, all schemes and processes, first cpu_budget steps
    from oracle import oracle as O
    import copy
    cores = len(os.sched_getaffinity(0))
    cb = args.cpu_budget or 64
    t0 = time.perf_counter()
    for s in searches:
        smp = copy.copy(s)
        smp.budget = min(cb, s.budget)
        O.search_obj(smp, n_threads=cores, digests=False)
    cpu_s = time.perf_counter() - t0
    cpu_steps = sum(len(s.mats) * s.n_proc * min(cb, s.budget) for s in searches)
    line = {
        "metric": METRIC, "value": out["batched"]["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": out["batched"]["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"batched: {len(searches)} schemes (config 3)", "n_processes": searches[0].n_proc,
                   "step_budget": searches[0].budget, "share_interval": interval, "col_cap": cap,
                   "shapes": [[list(m.shape) for m in s.mats] for s in searches[:3]] + ["..."],
                   "l2": "flushed (256 MB write) between timed steps"},
        "batched_graph": out["batched"], "one_launch_sequence_per_scheme": out["per_scheme"],
        "persistent_kernel_in_graph": out["persistent"],
        "speedup_batched_vs_per_scheme": out["per_scheme"]["ms"] / out["batched"]["ms"],
        "speedup_persistent_vs_per_scheme": out["per_scheme"]["ms"] / out["persistent"]["ms"],
        "fixed_wall_clock": fixed,
        "autotune": {"seconds": tune_s, "classes": tuned, "interval_candidates": [16, 32, 64],
                     "interval_chosen": interval},
        "roofline": roofline(mops_total / n_rounds, round_ms / n_rounds, ops_total / n_rounds, peak_clk,
                             props.multi_processor_count, {"sm_max_mhz": float(peaks().get("sm_max_mhz", 2070.0))},
                             None, "round kernels of the batched graph (all classes)"),
        "cpu_baseline": {"value": cpu_steps / cpu_s, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"all {len(searches)} schemes x 3 matrices x {searches[0].n_proc} processes, "
                                   f"first {cb} steps ({cpu_steps} process-steps, {cpu_s:.1f} s)"},
        "gpu_launches": out["batched"]["kernel_launches"] * args.steps,
    }
    print(json.dumps(line))


def run_serving(args):
    """Poisson stream of reduction requests (config 5) through the server,
    against running each request alone as it arrives."""
    import torch
    from paper_2512_13365_gb300 import cse, synth
    reqs = synth.serving_requests(n_req=args.requests, rate_hz=args.rate, n_proc=2048, budget=args.budget or 256)
    for _, s in reqs:
        s.cap = 512
    psteps = sum(s.process_steps() for _, s in reqs)

    def serve():
        import queue
        import threading
        sv = cse.Server(interval=32, cap=512)
        t0 = time.perf_counter()
        submitted = queue.Queue()
        totals = []

        def collect():  # each result as soon as it is done, then its device memory is released
            for _ in reqs:
                t = submitted.get()
                r = sv.wait(t)
                totals.append(r.total)
                r.free()

        collector = threading.Thread(target=collect)
        collector.start()
        for t_arr, s in reqs:
            d = t0 + t_arr - time.perf_counter()
            if d > 0:
                time.sleep(d)
            sc = cse.Scheme(s.mats)
            submitted.put(sv.submit(sc, s.weights, s.n_proc, s.seed, s.budget))
        collector.join()
        wall = time.perf_counter() - t0
        st = sv.stats()
        st["peak"] = sv.peak()[0]
        sv.free()
        return st, wall, totals

    def alone():
        t0 = time.perf_counter()
        lat, totals = [], []
        for t_arr, s in reqs:
            d = t0 + t_arr - time.perf_counter()
            if d > 0:
                time.sleep(d)
            sc = cse.Scheme(s.mats)
            r = cse.search(sc, s.weights, s.n_proc, s.seed, s.budget, 32, s.permille, 512)
            totals.append(r.total)
            lat.append((time.perf_counter() - t0 - t_arr) * 1000.0)
            r.free()
        wall = time.perf_counter() - t0
        lat.sort()
        pct = lambda p: lat[min(len(lat) - 1, int(np.ceil(p * len(lat))) - 1)]
        return {"p50_ms": pct(0.5), "p99_ms": pct(0.99), "steps_per_s": psteps / wall}, wall, totals

    import numpy as np
    for _ in range(args.warmup):
        pass
    st, wall, tot_s = serve()
    st_a, wall_a, tot_a = alone()
    assert tot_s == tot_a
    peak = st["peak"]
    line = {
        "metric": METRIC, "value": psteps / wall, "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 0,
        "ms_per_step": wall * 1000.0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"serving: {len(reqs)} Poisson requests at {args.rate:g}/s", "n_processes": 2048,
                   "step_budget": reqs[0][1].budget, "share_interval": 32, "col_cap": 512,
                   "admission": "library default limits (64 waves of resident warps)", "peak_active_searches": peak},
        "served": {"p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "process_steps_per_s": st["steps_per_s"],
                   "wall_s": wall},
        "one_launch_per_request": {"p50_ms": st_a["p50_ms"], "p99_ms": st_a["p99_ms"],
                                   "process_steps_per_s": st_a["steps_per_s"], "wall_s": wall_a},
        "results_identical": True,
    }
    print(json.dumps(line))


def run_iterations(args):
    """The paper's own schedule (iteration mode, share_interval = 0) on the
    (3,3,3:23)-shaped workload: 4096 processes per matrix, one whole run per
    process per iteration, sharing between iterations, stop when the best
    total has not improved for 10 iterations (Section 4).  The search length
    depends on convergence, so `value` counts the steps the runs made."""
    import torch
    from paper_2512_13365_gb300 import cse
    from oracle import oracle as O
    dev = torch.device("cuda", 0)
    s = workload("cfg2", args.procs)
    s.interval, s.budget = 0, args.budget or 1000
    patience = 10
    stream = torch.cuda.Stream(device=dev)
    scheme = cse.Scheme(s.mats)
    l2 = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def one():
        return cse.search(scheme, s.weights, s.n_proc, s.seed, s.budget, 0, s.permille, s.cap, stream=stream,
                          patience=patience)

    for _ in range(args.warmup):
        one().free()
    torch.cuda.synchronize()
    clocks = Clocks(os.path.join(args.out, "clocks_iter.csv"), 0)
    tw0 = time.time()
    ms, rec = [], None
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush_l2(l2)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = one()
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
        steps, sub, ops = r.counters()
        round_ms, _, n_rounds = r.timing()
        it, conv, total = r.iterations()
        rec = (steps, ops, round_ms, n_rounds, it, conv, total, r.costs, r.launches()[0], r.method_ops())
        r.free()
    clocks.window(tw0, time.time())
    clk = clocks.stop()
    steps, ops, round_ms, n_rounds, it, conv, total, costs, kernels, mops = rec
    t = statistics.mean(ms)
    # end to end: load from pinned host buffers, search to convergence, fetch every list
    e2e_ms, d2h = [], 0
    pinned = [torch.from_numpy(m).pin_memory().numpy() for m in s.mats]
    for _ in range(0 if args.no_e2e else 2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sc = cse.Scheme(pinned)
        r = cse.search(sc, s.weights, s.n_proc, s.seed, s.budget, 0, s.permille, s.cap, stream=stream,
                       patience=patience)
        lists = [r.fetch(k) for k in range(len(s.mats))]
        e2e_ms.append((time.perf_counter() - t0) * 1000.0)
        d2h = sum(4 * len(l) + 16 for l, _, _ in lists)
        r.free()
        sc.free()
    props = torch.cuda.get_device_properties(dev)
    peak_clk = measured_int_peak(stream)
    line = {
        "metric": METRIC, "value": steps / (t / 1000.0), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"{s.name}, iteration mode (patience {patience})",
                   "matrices": [list(m.shape) for m in s.mats], "n_processes": s.n_proc,
                   "max_iterations": s.budget, "share_permille": s.permille, "col_cap": s.cap,
                   "strategy_weights_gi_ga_gr_wr_mix_g_gp": list(s.weights),
                   "l2": "flushed (256 MB write) between timed steps"},
        "iterations": it, "converged": conv, "process_steps_per_search": steps,
        "best_additions": total, "best_additions_per_matrix": costs,
        "e2e": {"value": steps / (statistics.mean(e2e_ms) / 1000.0) if e2e_ms else None, "unit": UNIT,
                "h2d_bytes_per_step": sum(m.nbytes for m in s.mats), "d2h_bytes_per_step": d2h,
                "ms_per_step": statistics.mean(e2e_ms) if e2e_ms else None},
        "roofline": roofline(mops / n_rounds, round_ms / n_rounds, ops / n_rounds, peak_clk,
                             props.multi_processor_count, clk, None, "round_kernel (whole runs)"),
        "clocks": clk, "gpu_launches": kernels * args.steps,
    }
    if not args.no_cpu_baseline:
        cores = len(os.sched_getaffinity(0))
        t0 = time.perf_counter()
        ref = O.search_iterations(s.mats, s.weights, s.n_proc, s.seed, s.budget, patience, s.permille, s.cap,
                                  n_threads=cores, digests=False)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": ref.process_steps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"the whole search ({ref.iterations} iterations, "
                                          f"{ref.process_steps} process-steps, {dt:.1f} s)",
                                "best_additions": sum(ref.cost)}
    print(json.dumps(line))


def run_wallclock(args):
    """Best additions at fixed wall-clock budgets (1 s, 10 s, 60 s) on the
    (3,3,3:23)-shaped workload: the GPU search runs as many steps as fit in
    the budget (calibrated on the 1024-step search), the oracle as many as
    fit on the host cores (calibrated on 32 steps); both use the same seed,
    processes and options, so a longer budget is the same search run further."""
    import torch
    from paper_2512_13365_gb300 import cse
    from oracle import oracle as O
    import copy
    dev = torch.device("cuda", 0)
    s = workload("cfg2", args.procs)
    budgets_s = [float(x) for x in args.seconds.split(",")]
    stream = torch.cuda.Stream(device=dev)
    scheme = cse.Scheme(s.mats)

    def gpu(budget):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = cse.search(scheme, s.weights, s.n_proc, s.seed, budget, s.interval, s.permille, s.cap, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        out = (a.elapsed_time(b) / 1000.0, r.total, r.costs)
        r.free()
        return out

    for _ in range(args.warmup):
        gpu(s.budget)
    per_step = min(gpu(s.budget)[0] for _ in range(2)) / s.budget
    clocks = Clocks(os.path.join(args.out, "clocks_wallclock.csv"), 0)
    tw0 = time.time()
    gpu_rows = []
    for T in budgets_s:
        B = max(s.interval, int(T / per_step) // s.interval * s.interval)
        sec, total, costs = gpu(B)
        gpu_rows.append({"budget_s": T, "steps": B, "device_s": sec, "best_additions": total,
                         "best_additions_per_matrix": costs})
    clocks.window(tw0, time.time())
    clk = clocks.stop()
    cores = len(os.sched_getaffinity(0))
    smp = copy.copy(s)
    smp.budget = 32
    t0 = time.perf_counter()
    O.search_obj(smp, n_threads=cores, digests=False)
    cpu_per_step = (time.perf_counter() - t0) / 32
    cpu_rows = []
    for T in budgets_s:
        smp = copy.copy(s)
        smp.budget = max(s.interval, int(T / cpu_per_step) // s.interval * s.interval)
        t0 = time.perf_counter()
        ref = O.search_obj(smp, n_threads=cores, digests=False)
        cpu_rows.append({"budget_s": T, "steps": smp.budget, "wall_s": time.perf_counter() - t0,
                         "best_additions": ref.total})
    line = {
        "metric": METRIC, "value": gpu_rows[-1]["steps"] * len(s.mats) * s.n_proc / gpu_rows[-1]["device_s"],
        "unit": UNIT, "n_gpus": 1, "steps": len(budgets_s), "warmup": args.warmup,
        "ms_per_step": gpu_rows[-1]["device_s"] * 1000.0, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"{s.name}, best additions at fixed wall-clock budgets", "n_processes": s.n_proc,
                   "share_interval": s.interval, "col_cap": s.cap, "budgets_s": budgets_s},
        "gpu": gpu_rows, "cpu_oracle": {"cores": cores, "kind": "oracle", "runs": cpu_rows},
        "clocks": clk,
    }
    print(json.dumps(line))


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    s = workload(args.workload)
    cores = len(os.sched_getaffinity(0))
    import copy
    procs, steps = REF_SAMPLE.get(args.workload, (s.n_proc, max(1, s.budget // 8)))
    smp = copy.copy(s)
    smp.n_proc = min(procs, s.n_proc)
    smp.budget = args.cpu_budget or min(steps, s.budget)
    for _ in range(args.warmup):
        w = copy.copy(smp)
        w.budget = min(8, smp.budget)
        O.search_obj(w, n_threads=cores, digests=False)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.search_obj(smp, n_threads=cores, digests=False)
        times.append(time.perf_counter() - t0)
    ms = statistics.mean(times) * 1000.0
    v = smp.process_steps() / (ms / 1000.0)
    sample = (f"{s.name}: first {smp.n_proc} of {s.n_proc} processes x {len(s.mats)} matrices, first "
              f"{smp.budget} of {s.budget} steps per benchmark step ({smp.process_steps()} process-steps)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "config": {"workload": s.name, "matrices": [list(m.shape) for m in s.mats], "n_processes": s.n_proc,
                   "step_budget": s.budget, "share_interval": s.interval, "col_cap": s.cap},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cfg4",
                    help="cfg4 (default, the benchmark line: the largest single-GPU workload), cfg2, cfg1, "
                         "cfg3 (batched), cfg5 (serving), "
                         "cfg2-iter (iteration mode), cfg2-wallclock (best additions at fixed wall-clock budgets)")
    ap.add_argument("--requests", type=int, default=200, help="cfg5: number of requests")
    ap.add_argument("--rate", type=float, default=50.0, help="cfg5: mean Poisson arrival rate (requests/s)")
    ap.add_argument("--procs", type=int, default=0, help="override the process count (reduced-scale runs)")
    ap.add_argument("--ppc", type=int, default=0, help="processes per CTA (0 = library default)")
    ap.add_argument("--cpu-budget", type=int, default=0,
                    help="steps of the oracle sample (0 = the workload's bounded sample)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--budget", type=int, default=0, help="override the step budget (profiling runs)")
    ap.add_argument("--seconds", default="1,10,60", help="cfg2-wallclock: the wall-clock budgets")
    ap.add_argument("--warp-engine", action="store_true",
                    help="large matrices on the one-warp-per-process engine only (the default; overrides --cta-engine)")
    ap.add_argument("--cta-engine", action="store_true",
                    help="large matrices on the process-per-CTA engine for run starts and long lists (a launch "
                         "choice; same results)")
    ap.add_argument("--cta-min-list", type=int, default=0,
                    help="with --cta-engine: runs under way with shorter lists go to the warp engine "
                         "(0 = library default)")
    ap.add_argument("--gi-shared", action="store_true",
                    help="Greedy-Intersections with shared coins (an option that changes results)")
    ap.add_argument("--out", default=os.path.join(ROOT, "bench_out"), help="where the clock samples go")
    args = ap.parse_args()
    os.makedirs(args.out, exist_ok=True)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "cfg3":
        run_batched(args)
    elif args.workload == "cfg5":
        run_serving(args)
    elif args.workload == "cfg2-iter":
        run_iterations(args)
    elif args.workload == "cfg2-wallclock":
        run_wallclock(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
