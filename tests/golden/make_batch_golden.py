"""Writes the expected balanced / unbalanced totals of every member of the 4,096-graph
batched workload, from the CPU oracle.

Usage: python tests/golden/make_batch_golden.py [threads]

The only counting code this script runs is ``oracle.count`` (the plain CPU oracle), one
single-threaded call per graph spread over a thread pool (the oracle's ctypes calls
release the interpreter lock). The graphs come from the seeded generators
(``synth.batch_specs(4096, seed=0)``). The output holds, per member, its index, its
sizes and its two totals, and one SHA-256 digest over every member's edge list in index
order, so that a test can confirm it generated the same batch.
"""

from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2601_17707_gb300 import synth  # noqa: E402

N_GRAPHS = 4096
SEED = 0
OUT = os.path.join(HERE, "batch_4096_chung_lu.txt")


def batch_digest(gs) -> str:
    h = hashlib.sha256()
    for g in gs:
        h.update(np.ascontiguousarray(g.u, dtype="<i4").tobytes())
        h.update(np.ascontiguousarray(g.v, dtype="<i4").tobytes())
        h.update(np.ascontiguousarray(g.sign, dtype="i1").tobytes())
    return h.hexdigest()


def main() -> None:
    threads = int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1)
    specs = synth.batch_specs(N_GRAPHS, seed=SEED)
    gs = synth.batch_graphs(specs)
    t0 = time.time()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        counts = list(ex.map(lambda g: oracle.count(g, threads=1, per_vertex=False), gs))
    dt = time.time() - t0
    with open(OUT, "w") as f:
        f.write(f"# Expected totals of the {N_GRAPHS}-graph batched workload (synth.batch_specs, "
                f"seed {SEED}), written by\n")
        f.write("# tests/golden/make_batch_golden.py from the CPU oracle alone "
                f"({threads} threads, {dt:.0f} s).\n")
        f.write(f"graphs {N_GRAPHS}\nseed {SEED}\n")
        f.write(f"edges_sha256 {batch_digest(gs)}\n")
        f.write(f"balanced_sum {sum(c.balanced for c in counts)}\n")
        f.write(f"unbalanced_sum {sum(c.unbalanced for c in counts)}\n")
        f.write("# member index, n_u, n_v, n_edges, balanced, unbalanced\n")
        for i, (g, c) in enumerate(zip(gs, counts)):
            f.write(f"g {i} {g.n_u} {g.n_v} {g.n_edges} {c.balanced} {c.unbalanced}\n")
    print(OUT, dt)


if __name__ == "__main__":
    main()
