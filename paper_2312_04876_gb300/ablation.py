"""Parameter study of the Louvain controls on the GPU path (host-side driver of louvain_run).

For each control of Section 4.1 the study runs the defaults and an alternative, and reports the
alternative's runtime and modularity relative to the defaults, as the paper's parameter study does
(Figure 3).  The workloads are the seeded synthetic graphs that stand in for the paper's
SuiteSparse set.

    python -m paper_2312_04876_gb300.ablation --workloads sbm10k rmat20 grid6m --mode fast \
        --reps 3 --md study.md [--json study.json]

Settings, each changing one control of the defaults:

* MAX_ITERATIONS: 20 against 100 and 10;
* tolerance drop rate: 10 against 1 (threshold scaling off) and 100;
* initial tolerance: 0.01 against 1e-6 and 0.1;
* aggregation tolerance: 0.8 against 1 (never stops early) and 0.6;
* vertex pruning: on against off;
* super-vertex graph: compacted against holey;
* hash-table sizing: 2 slots per key against 1 and 4 (table_factor).

Timing and aggregation:

* Each setting runs once untimed, since its first run builds its iteration graphs and buffers.
* It then runs `reps` timed times.  Runtime is the median of CUDA-event times on the run's
  stream.  Modularity is the mean, since fast mode varies from run to run.
* Across workloads, relative runtimes combine by geometric mean and relative modularities by
  arithmetic mean.
"""
from __future__ import annotations

import argparse
import json
import math
import statistics
import sys

# (control, alternative value); the defaults come from louvain_default_params
ALTERNATIVES = [
    ("max_iterations", 100), ("max_iterations", 10),
    ("tolerance_drop", 1.0), ("tolerance_drop", 100.0),
    ("tolerance", 1e-6), ("tolerance", 1e-1),
    ("aggregation_tolerance", 1.0), ("aggregation_tolerance", 0.6),
    ("pruning", 0),
    ("compact", 0),
    ("table_factor", 1), ("table_factor", 4),
]

def _rmat27_fp32():
    """R-MAT 27 with fp32 weights (134M vertices, 4.2B arcs), drawn on the device: (offsets,
    targets, weights) as CUDA tensors."""
    from graphgen import device
    return device.rmat(27, 16, 0.57, 0.19, 0.19, 22, fp_weights=True)


WORKLOADS = {
    "sbm10k": lambda gg: gg.sbm(10000, 100, 0.1, 0.0005, 1),
    "rmat20": lambda gg: gg.rmat(20, 16, 0.57, 0.19, 0.19, 22, gg.W_INT8),
    "rmat22": lambda gg: gg.rmat(22, 16, 0.57, 0.19, 0.19, 22, gg.W_INT8),
    "grid6m": lambda gg: gg.grid(2449, 2449, 0.10, 0.01, 3),
    "grid24m": lambda gg: gg.grid(4899, 4899, 0.10, 0.01, 3),
    "rmat27_fp32": lambda gg: _rmat27_fp32(),
}


def settings() -> list:
    """[(label, overrides)]: the defaults first, then one entry per alternative."""
    out = [("defaults", {})]
    for name, value in ALTERNATIVES:
        out.append((f"{name}={value:g}" if isinstance(value, float) else f"{name}={value}", {name: value}))
    return out


def measure(timed_run, reps: int) -> dict:
    """timed_run() -> (ms, result with .modularity, .passes, .total_iterations).  One untimed call,
    then `reps` timed ones."""
    timed_run()
    ms, q, passes, its = [], [], [], []
    for _ in range(max(reps, 1)):
        t, r = timed_run()
        ms.append(t)
        q.append(r.modularity)
        passes.append(r.passes)
        its.append(r.total_iterations)
    return {"ms": statistics.median(ms), "q": statistics.fmean(q), "passes": statistics.fmean(passes),
            "iterations": statistics.fmean(its), "reps": len(ms)}


def summarise(results: dict) -> list:
    """results[workload][label] = measure(...) -> rows of (label, relative runtime, relative
    modularity), combined over workloads (geometric / arithmetic mean), defaults first."""
    labels = [lab for lab, _ in settings()]
    rows = []
    for lab in labels:
        tr, qr = [], []
        for wl, per in results.items():
            if lab not in per or "defaults" not in per or "error" in per[lab] or "error" in per["defaults"]:
                continue
            base = per["defaults"]
            tr.append(per[lab]["ms"] / base["ms"])
            qr.append(per[lab]["q"] / base["q"] if base["q"] != 0 else float("nan"))
        if tr:
            rows.append((lab, math.exp(statistics.fmean(math.log(x) for x in tr)), statistics.fmean(qr)))
        else:  # failed on every workload: listed, with no ratios
            rows.append((lab, float("nan"), float("nan")))
    return rows


def markdown(results: dict, mode: str, command: str) -> str:
    rows = summarise(results)
    wls = list(results)
    out = [f"# Parameter study, {mode} mode", "", "Command:", "", "```", command, "```", "",
           "Runtime relative to the defaults (geometric mean over workloads) and modularity relative to the "
           "defaults (arithmetic mean); per workload the median ms and the mean Q.  The defaults are measured "
           "before and after the other settings and the faster median is the reference.", "",
           "| setting | rel. runtime | rel. modularity | " + " | ".join(f"{w} ms | {w} Q" for w in wls) + " |",
           "|---|---:|---:|" + "---:|---:|" * len(wls)]
    for lab, rt, rq in rows:
        cells = []
        for w in wls:
            m = results[w].get(lab)
            if m and "error" in m:
                cells += ["failed", ""]
            else:
                cells += [f"{m['ms']:.2f}", f"{m['q']:.5f}"] if m else ["", ""]
        out.append(f"| {lab} | {rt:.3f} | {rq:.4f} | " + " | ".join(cells) + " |")
    return "\n".join(out) + "\n"


def study(graphs: dict, make_timed_run, reps: int) -> dict:
    """graphs[name] = device CSR; make_timed_run(graph, overrides) -> timed_run for measure().
    The defaults are measured first and again after the other settings; the faster of the two
    medians is the reference (a one-off stall of the host or the box in the first calls of a
    process once put the defaults 7x above every other setting of a workload)."""
    def attempt(graph, ov):
        try:
            return measure(make_timed_run(graph, ov), reps)
        except Exception as e:  # a setting the library refuses (e.g. a table that overflows): recorded
            return {"ms": float("nan"), "q": float("nan"), "passes": float("nan"), "iterations": float("nan"),
                    "reps": 0, "error": f"{type(e).__name__}: {e}"[:160]}

    results = {}
    for wl, graph in graphs.items():
        results[wl] = {lab: attempt(graph, ov) for lab, ov in settings()}
        again = attempt(graph, {})
        if "error" in results[wl]["defaults"] or again["ms"] < results[wl]["defaults"]["ms"]:
            results[wl]["defaults"] = again
    return results


def _cuda_timed_run(L, graph, params, stream):
    import torch

    def run():
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        _, r = L.run(*graph, params, stream=stream)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), r

    return run


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workloads", nargs="+", default=["sbm10k", "rmat20", "grid6m"], choices=sorted(WORKLOADS))
    ap.add_argument("--mode", default="fast", choices=["fast", "deterministic"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--md", default=None)
    ap.add_argument("--json", default=None)
    a = ap.parse_args(argv)
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("the parameter study runs the CUDA path: no CUDA device is visible")
    import graphgen as gg

    import paper_2312_04876_gb300 as lv
    stream = torch.cuda.current_stream()
    results = {}
    for wl in a.workloads:  # one workload at a time, with its own handle
        g = WORKLOADS[wl](gg)
        graph = g if isinstance(g, tuple) else tuple(torch.from_numpy(x).cuda() for x in (g.offsets, g.targets, g.weights))
        del g
        torch.cuda.synchronize()
        torch.cuda.empty_cache()  # a device generator's scratch goes back before the runs
        L = lv.Louvain(0)

        def make(gr, ov, L=L):
            return _cuda_timed_run(L, gr, lv.default_params(mode=a.mode, validate=0, **ov), stream)

        results.update(study({wl: graph}, make, a.reps))
        L.close()
        del graph
        torch.cuda.empty_cache()
    command = "python -m paper_2312_04876_gb300.ablation " + " ".join(sys.argv[1:] if argv is None else argv)
    md = markdown(results, a.mode, command)
    if a.md:
        with open(a.md, "w") as f:
            f.write(md)
    if a.json:
        with open(a.json, "w") as f:
            json.dump({"mode": a.mode, "reps": a.reps, "results": results}, f, indent=1)
    print(md)
    return 0


if __name__ == "__main__":
    sys.exit(main())
