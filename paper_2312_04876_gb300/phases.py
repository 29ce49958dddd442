"""Where a Louvain run spends its time on the GPU path (host-side driver of louvain_run).

The report has three parts, the breakdowns the paper gives for its own runs (Figures 5 and 6):

* the split by phase (colouring, local moving, aggregation, other), summed over passes;
* the split by pass;
* the runtime per arc of the input.

The workloads are the seeded synthetic graphs that stand in for the paper's SuiteSparse set.

    python -m paper_2312_04876_gb300.phases --workloads sbm10k rmat20 rmat22 grid24m --mode fast \
        --reps 3 --md phases.md

Each workload runs once untimed, then `reps` times.  The run with the median device time
(`louvain_result.ms_total`) supplies the per-pass phase times (`louvain_pass_stats`, CUDA events
on the run's stream).
"""
from __future__ import annotations

import argparse
import sys

PHASES = ("ms_colour", "ms_move", "ms_aggregate", "ms_other")
PHASE_NAMES = {"ms_colour": "colouring", "ms_move": "local moving", "ms_aggregate": "aggregation",
               "ms_other": "other"}

def _rmat27_fp32():
    """R-MAT 27 with fp32 weights (134M vertices, 4.2B arcs), drawn on the device: (offsets,
    targets, weights) as CUDA tensors."""
    from graphgen import device
    return device.rmat(27, 16, 0.57, 0.19, 0.19, 22, fp_weights=True)


WORKLOADS = {
    "sbm10k": lambda gg: gg.sbm(10000, 100, 0.1, 0.0005, 1),
    "rmat20": lambda gg: gg.rmat(20, 16, 0.57, 0.19, 0.19, 22, gg.W_INT8),
    "rmat22": lambda gg: gg.rmat(22, 16, 0.57, 0.19, 0.19, 22, gg.W_INT8),
    "grid24m": lambda gg: gg.grid(4899, 4899, 0.10, 0.01, 3),
    "rmat27_fp32": lambda gg: _rmat27_fp32(),
}


def split(stats: list) -> dict:
    """Per-pass stats (dicts with the PHASES keys) -> phase totals and shares, and pass shares."""
    tot = {ph: sum(s[ph] for s in stats) for ph in PHASES}
    all_ms = sum(tot.values())
    per_pass = [sum(s[ph] for ph in PHASES) for s in stats]
    return {"phase_ms": tot,
            "phase_share": {ph: (tot[ph] / all_ms if all_ms > 0 else 0.0) for ph in PHASES},
            "pass_ms": per_pass,
            "pass_share": [(p / all_ms if all_ms > 0 else 0.0) for p in per_pass],
            "ms": all_ms}


def pick_median(runs: list):
    """runs: [(ms_total, stats)] -> the run whose time is the (lower) median."""
    order = sorted(range(len(runs)), key=lambda k: runs[k][0])
    return runs[order[(len(order) - 1) // 2]]


def markdown(results: dict, mode: str, command: str) -> str:
    """results[workload] = {"n_arcs": A, "ms": run ms, "split": split(...)}."""
    out = [f"# Phase and pass split, {mode} mode", "", "Command:", "", "```", command, "```", "",
           "| workload | arcs | run ms | ns per arc | " + " | ".join(PHASE_NAMES[p] for p in PHASES) +
           " | pass shares |",
           "|---|---:|---:|---:|" + "---:|" * len(PHASES) + "---|"]
    for wl, r in results.items():
        sp = r["split"]
        shares = " | ".join(f"{100 * sp['phase_share'][p]:.1f}%" for p in PHASES)
        passes = ", ".join(f"{100 * x:.1f}%" for x in sp["pass_share"])
        out.append(f"| {wl} | {r['n_arcs']:,} | {r['ms']:.2f} | {1e6 * r['ms'] / max(r['n_arcs'], 1):.3f} | "
                   f"{shares} | {passes} |")
    return "\n".join(out) + "\n"


def profile(run, n_arcs: int, reps: int) -> dict:
    """run() -> (ms_total, per-pass stats); one untimed call, then `reps`."""
    run()
    ms, stats = pick_median([run() for _ in range(max(reps, 1))])
    return {"n_arcs": n_arcs, "ms": ms, "split": split(stats)}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workloads", nargs="+", default=["sbm10k", "rmat20", "rmat22"], choices=sorted(WORKLOADS))
    ap.add_argument("--mode", default="fast", choices=["fast", "deterministic"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--md", default=None)
    a = ap.parse_args(argv)
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("the phase report runs the CUDA path: no CUDA device is visible")
    import graphgen as gg

    import paper_2312_04876_gb300 as lv
    params = lv.default_params(mode=a.mode, validate=0)
    results = {}
    for wl in a.workloads:
        g = WORKLOADS[wl](gg)
        if isinstance(g, tuple):  # drawn on the device
            o, t, w = g
        else:
            o, t, w = (torch.from_numpy(x).cuda() for x in (g.offsets, g.targets, g.weights))
        del g
        torch.cuda.synchronize()
        torch.cuda.empty_cache()  # the generator's scratch goes back before the run sizes its workspace
        L = lv.Louvain(0)  # a handle per workload: the previous one's workspace is released

        def run():
            _, r = L.run(o, t, w, params)
            return r.ms_total, r.stats

        results[wl] = profile(run, t.numel(), a.reps)
        L.close()
        del o, t, w
        torch.cuda.empty_cache()
    command = "python -m paper_2312_04876_gb300.phases " + " ".join(sys.argv[1:] if argv is None else argv)
    md = markdown(results, a.mode, command)
    if a.md:
        with open(a.md, "w") as f:
            f.write(md)
    print(md)
    return 0


if __name__ == "__main__":
    sys.exit(main())
