"""Writes tests/golden/cfg4_reduced.txt: the oracle's results for the
(6,6,6:153)-shaped workload at reduced scale (512 processes per matrix, 200
steps, sharing every 32 steps, column cap 512: six sharing boundaries).

Every value in that file comes from oracle/ (the CPU oracle) on inputs from
paper_2512_13365_gb300/synth.py; nothing comes from the CUDA library.  The
GPU parity test compares the library's search with it process by process.

    python tests/golden/make_cfg4_golden.py [n_threads]
"""
import hashlib
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2512_13365_gb300 import synth  # noqa: E402

N_PROC, BUDGET = 512, 200
FIELDS = ("best_cost", "best_len", "runs", "best_hash", "traj_hash", "ops", "substeps", "best_strategy",
          "method_ops")
OUT = os.path.join(HERE, "cfg4_reduced.txt")


def inputs_sha(s) -> str:
    h = hashlib.sha256()
    for m in s.mats:
        h.update(m.tobytes())
    return h.hexdigest()[:16]


def main():
    threads = int(sys.argv[1]) if len(sys.argv) > 1 else len(os.sched_getaffinity(0))
    s = synth.config4(n_proc=N_PROC, budget=BUDGET)
    t0 = time.time()
    ref = O.search_obj(s, n_threads=threads)
    dt = time.time() - t0
    lines = [f"# oracle results, {s.name} at {N_PROC} processes x {BUDGET} steps, interval {s.interval}, "
             f"permille {s.permille}, cap {s.cap}, seed {s.seed}, weights {list(s.weights)}",
             f"# written by tests/golden/make_cfg4_golden.py ({dt:.0f} s on {threads} threads)",
             f"inputs_sha256 {inputs_sha(s)}",
             f"params {N_PROC} {BUDGET} {s.interval} {s.permille} {s.cap} {s.seed}",
             "costs " + " ".join(str(c) for c in ref.cost)]
    for k, lst in enumerate(ref.lists):
        lines.append(f"list {k} " + " ".join(str(e) for e in lst))
    for k, cv in enumerate(ref.curve):
        lines.append(f"curve {k} " + " ".join(str(c) for c in cv))
    lines.append("# per process: " + " ".join(FIELDS) + " (hashes in hex)")
    for k in range(len(s.mats)):
        d = ref.digests[k]
        for p in range(N_PROC):
            vals = []
            for f in FIELDS:
                v = int(d[f][p])
                vals.append(f"{v:x}" if f.endswith("hash") else str(v))
            lines.append(f"p {k} {p} " + " ".join(vals))
    with open(OUT, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print(f"wrote {OUT} in {dt:.0f} s")


if __name__ == "__main__":
    main()
