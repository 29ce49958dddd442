"""Writes tests/golden/*.json: CPU-oracle results on the full-size synthetic workloads.

Calls only the seeded generators (graphgen) and the CPU oracle (oracle/); nothing here touches the
GPU library.  Each record holds the CSR's SHA-256 (so a reader can check it regenerated the same
graph), the deterministic-schedule oracle's membership SHA-256, modularity (Eq. 1), pass count and
community count, and the sequential-oracle modularity as a second reference.

    python tests/golden/make_golden.py [rmat22 sbm10k ...]
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import graphgen as gg  # noqa: E402
import oracle  # noqa: E402

WORKLOADS = {
    "rmat22": lambda: gg.rmat(22, 16, 0.57, 0.19, 0.19, 22, gg.W_INT8),
    "rmat20": lambda: gg.rmat(20, 16, 0.57, 0.19, 0.19, 22, gg.W_INT8),
    "sbm10k": lambda: gg.sbm(10000, 100, 0.1, 0.0005, 1),
    # road-like: 4899 x 4899 lattice (~24.0M vertices), 10% of the edges deleted, 1% long links
    "grid24m": lambda: gg.grid(4899, 4899, 0.10, 0.01, 3),
    # R-MAT 22 without its 1,799,215 isolated vertices (which count toward |V'| in the pass loop's
    # aggregation-tolerance test and stop it after two passes on the full graph)
    "rmat22_noiso": lambda: gg.drop_isolated(gg.rmat(22, 16, 0.57, 0.19, 0.19, 22, gg.W_INT8)),
    # fp32 weights in (0, 1]; 172 rows over 4096 arcs (the giant-row path), maximum degree 25,238
    "rmat18_fp32": lambda: gg.rmat(18, 16, 0.57, 0.19, 0.19, 18, gg.W_FP32),
}


def csr_sha256(g) -> str:
    h = hashlib.sha256()
    for a in (g.offsets, g.targets, g.weights):
        h.update(a.tobytes())
    return h.hexdigest()


def main(names):
    for name in names:
        t0 = time.time()
        g = WORKLOADS[name]()
        t1 = time.time()
        mem, q, passes, stats = oracle.louvain(g.offsets, g.targets, g.weights, oracle.default_params())
        t2 = time.time()
        _, q_seq, _, _ = oracle.louvain(g.offsets, g.targets, g.weights, oracle.default_params(schedule=1))
        rec = {
            "workload": name, "n": g.n, "arcs": g.n_arcs, "csr_sha256": csr_sha256(g),
            "params": "oracle.default_params() (paper defaults, max_passes 10, seed 0, colour-synchronous)",
            "membership_sha256": hashlib.sha256(mem.astype("<i4").tobytes()).hexdigest(),
            "modularity": q, "passes": passes, "communities": int(mem.max()) + 1 if len(mem) else 0,
            "iterations": [s["iterations"] for s in stats],
            "sequential_modularity": q_seq,
            "oracle_seconds": round(t2 - t1, 2), "generate_seconds": round(t1 - t0, 2),
        }
        with open(os.path.join(HERE, f"{name}_oracle.json"), "w") as f:
            json.dump(rec, f, indent=1)
        print(json.dumps(rec))


if __name__ == "__main__":
    main(sys.argv[1:] or ["sbm10k", "rmat20", "rmat22"])
