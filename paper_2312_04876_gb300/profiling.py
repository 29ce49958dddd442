"""Summaries of Nsight Compute launch lists of a Louvain run (host-side tooling, no GPU needed).

`ncu --csv --log-file F --metrics gpu__time_duration.sum[,dram__bytes_read.sum,dram__bytes_write.sum]`
writes one row per (launch, metric).  This module groups the rows by launch, maps every kernel to
the kernel class that louvain_kernel_profile reports (the local-move and merge kernels by degree
bucket, the giant-row kernels by phase), and writes

  * a Markdown table per kernel (launches, total time, share of the run's kernel time) and per
    class, with the command that produced the list;
  * a JSON file of DRAM bytes per class invocation, keyed by a hash of the CUDA sources, that the
    benchmark reads as the roofline's measured `traffic` (stale once the sources change).

    python -m paper_2312_04876_gb300.profiling launches.csv --workload rmat22 --mode fast \
        --command "<the ncu command>" --md profiles/x.md [--traffic-json profiles/traffic_rmat22_fast.json]

With --full, the csv is the raw page of one full capture (`ncu -i r.ncu-rep --page raw --csv`)
and the Markdown lists its key counters per launch (duration, DRAM bytes, occupancy, stalls).
"""
from __future__ import annotations

import argparse
import collections
import csv
import hashlib
import json
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (group lanes, log2 table slots) of the per-bucket kernels -> bucket
_BUCKET_OF = {("4", "3"): 0, ("8", "5"): 1, ("32", "8"): 2, ("32", "10"): 3, ("256", "12"): 4, ("256", "13"): 5}
_LM_NAMES = ["local_move_b0_g4", "local_move_b1_g8", "local_move_b2_warp", "local_move_b3_warp1k",
             "local_move_b4_block4k", "local_move_b5_block8k", "local_move_b6_giant"]
_MG_NAMES = ["merge_b0_g4", "merge_b1_g8", "merge_b2_warp", "merge_b3_warp1k", "merge_b4_block4k",
             "merge_b5_block8k", "merge_b6_giant"]
GIANT = 6
# kernel whose launch count is the number of invocations of each multi-kernel class
PRIMARY = {"local_move_b6_giant": "k_glm_scan", "merge_b6_giant": "k_giant_mg_emit"}


def strip_comments(src: str) -> str:
    """C/C++/CUDA source with its comments removed and every run of whitespace outside string and
    character literals collapsed to one newline (if it holds one) or one space: what the compiler
    and preprocessor see, so that editing a comment or re-indenting keeps a capture's counters
    valid."""
    out = []
    i, n = 0, len(src)
    gap = ""  # pending separator: "", " " or "\n"

    def sep(kind):
        return "\n" if "\n" in (gap, kind) else kind

    while i < n:
        ch = src[i]
        if src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j  # the newline itself is kept as whitespace
            gap = sep(" ")
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            body = src[i:n if j < 0 else j]
            i = n if j < 0 else j + 2
            gap = sep("\n" if "\n" in body else " ")
        elif ch.isspace():
            gap = sep("\n" if ch == "\n" else " ")
            i += 1
        else:
            if ch in "\"'":
                j = i + 1
                while j < n and src[j] != ch and src[j] != "\n":
                    j += 2 if src[j] == "\\" else 1
                tok = src[i:j + 1]
            else:
                tok = ch
            if gap and out:
                out.append(gap)
            gap = ""
            out.append(tok)
            i += len(tok)
    return "".join(out)


def source_sha256(root: str = ROOT) -> str:
    """Hash of the CUDA sources and the public header, comments and layout left out (same
    definition as the benchmark's)."""
    csrc = os.path.join(root, "paper_2312_04876_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(csrc, f), encoding="utf-8") as fh:
                h.update(f.encode() + b"\0" + strip_comments(fh.read()).encode())
    with open(os.path.join(root, "include", "louvain.h"), encoding="utf-8") as fh:
        h.update(strip_comments(fh.read()).encode())
    return h.hexdigest()


def short_name(full: str) -> str:
    """'void lm_kernel<IntMode, 32, 8, 0>(LmArgs<IntMode>)' -> 'lm_kernel<IntMode, 32, 8, 0>'."""
    s = re.sub(r"^void\s+", "", full.strip())
    depth = 0
    for k, ch in enumerate(s):
        if ch == "<":
            depth += 1
        elif ch == ">":
            depth -= 1
        elif ch == "(" and depth == 0:
            return s[:k].replace("lv::", "")
    return s.replace("lv::", "")


def kernel_class(name: str) -> str | None:
    """Kernel class of one launch, or None for kernels that belong to the sequence around them
    (the giant-row plan kernel, resolved by the caller from the next giant kernel)."""
    base = name.split("<")[0]
    args = [a.strip() for a in name[len(base) + 1:-1].split(",")] if "<" in name else []
    if base == "lm_kernel" and len(args) >= 3:
        return _LM_NAMES[_BUCKET_OF.get((args[1], args[2]), GIANT)]
    if base == "merge_kernel" and len(args) >= 3:
        return _MG_NAMES[_BUCKET_OF.get((args[1], args[2]), GIANT)]
    if base.startswith("k_glm_"):
        return _LM_NAMES[GIANT]
    if base.startswith("k_giant_mg_"):
        return _MG_NAMES[GIANT]
    if base.startswith("k_gplan_"):
        return None
    if base in ("k_compact", "k_compact_group", "k_giant_copy_chunks", "k_row_len"):
        return "compact"
    if base.startswith("k_mod_") or base == "k_giant_mod_chunks":
        return "modularity"
    if base.startswith("jp_") or base == "k_jp_reset":
        return "colour_jp"
    if base == "lm_apply":
        return "sigma_apply"
    return "other"


def read_launches(path: str) -> list[dict]:
    """Launches in ID order: {'id', 'name', 'grid', 'block', metric: value...} (times in ns)."""
    rows = []
    with open(path, newline="") as f:
        lines = [ln for ln in f if ln.startswith('"')]
    rd = csv.reader(lines)
    hdr = None
    by_id = collections.OrderedDict()
    for r in rd:
        if r and r[0] == "ID":
            hdr = r
            continue
        if not hdr or len(r) != len(hdr):
            continue
        d = dict(zip(hdr, r))
        lid = int(d["ID"])
        L = by_id.setdefault(lid, {"id": lid, "name": short_name(d["Kernel Name"]), "grid": d["Grid Size"],
                                   "block": d["Block Size"]})
        unit = d["Metric Unit"]
        v = float(d["Metric Value"].replace(",", ""))
        scale = {"us": 1e3, "usecond": 1e3, "ms": 1e6, "msecond": 1e6, "s": 1e9, "second": 1e9,
                 "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9}.get(unit, 1.0)
        L[d["Metric Name"]] = v * scale
    rows = list(by_id.values())
    # resolve the plan kernels to the class of the next giant-row kernel
    nxt = None
    for L in reversed(rows):
        c = kernel_class(L["name"])
        if c is None:
            c = nxt or "other"
        elif c in (_LM_NAMES[GIANT], _MG_NAMES[GIANT], "compact", "modularity"):
            nxt = c
        L["class"] = c
    return rows


def summarise(rows: list[dict]) -> dict:
    tot = sum(L.get("gpu__time_duration.sum", 0.0) for L in rows)
    ker = collections.OrderedDict()
    cls = collections.OrderedDict()
    for L in rows:
        t = L.get("gpu__time_duration.sum", 0.0)
        dram = L.get("dram__bytes_read.sum", 0.0) + L.get("dram__bytes_write.sum", 0.0)
        has_dram = "dram__bytes_read.sum" in L
        k = ker.setdefault(L["name"], {"launches": 0, "ns": 0.0, "dram": 0.0, "class": L["class"]})
        k["launches"] += 1
        k["ns"] += t
        k["dram"] += dram
        c = cls.setdefault(L["class"], {"launches": 0, "kernel_launches": 0, "ns": 0.0, "dram": 0.0,
                                        "has_dram": has_dram})
        c["kernel_launches"] += 1
        c["ns"] += t
        c["dram"] += dram
    for name, c in cls.items():
        prim = PRIMARY.get(name)
        if prim:
            c["launches"] = sum(k["launches"] for kn, k in ker.items() if kn.split("<")[0] == prim)
        else:
            c["launches"] = c["kernel_launches"]
    return {"total_ns": tot, "launches": len(rows), "kernels": ker, "classes": cls}


def markdown(s: dict, title: str, command: str) -> str:
    tot = s["total_ns"]
    out = [f"# {title}", "", "Command (run from the repository root on one GB300):", "", "```", command, "```", "",
           f"{s['launches']} kernel launches, {tot / 1e6:.3f} ms of kernel time (ncu serialises launches and "
           "runs them cold: compare shares, not absolute times).", "",
           "| kernel | class | launches | total ms | share | DRAM MB/launch |", "|---|---|---:|---:|---:|---:|"]
    for name, k in sorted(s["kernels"].items(), key=lambda kv: -kv[1]["ns"]):
        dram = f"{k['dram'] / k['launches'] / 1e6:.2f}" if k["dram"] else "-"
        out.append(f"| `{name}` | {k['class']} | {k['launches']} | {k['ns'] / 1e6:.3f} | "
                   f"{100 * k['ns'] / tot:.1f}% | {dram} |")
    out += ["", "| class | invocations | kernel launches | total ms | share | DRAM MB/invocation |",
            "|---|---:|---:|---:|---:|---:|"]
    for name, c in sorted(s["classes"].items(), key=lambda kv: -kv[1]["ns"]):
        dram = f"{c['dram'] / max(1, c['launches']) / 1e6:.2f}" if c["has_dram"] else "-"
        out.append(f"| {name} | {c['launches']} | {c['kernel_launches']} | {c['ns'] / 1e6:.3f} | "
                   f"{100 * c['ns'] / tot:.1f}% | {dram} |")
    return "\n".join(out) + "\n"


def traffic_json(s: dict, workload: str, mode: str, command: str, source_root: str = ROOT) -> dict:
    classes = {}
    for name, c in s["classes"].items():
        if c["has_dram"] and c["launches"]:
            classes[name] = {"dram_bytes_per_launch": c["dram"] / c["launches"], "invocations": c["launches"],
                             "kernel_launches": c["kernel_launches"], "ncu_ms": c["ns"] / 1e6}
    return {"workload": workload, "mode": mode, "source_sha256": source_sha256(source_root), "command": command,
            "note": "dram__bytes_read.sum + dram__bytes_write.sum per class invocation, one ncu pass "
                    "per launch; valid only while the CUDA sources (comments and layout left out) hash to source_sha256",
            "classes": classes}


# metrics of a full (`--set full`) report worth a line in a summary, with their labels
FULL_METRICS = [
    ("gpu__time_duration.sum", "duration"),
    ("dram__bytes_read.sum", "DRAM read"),
    ("dram__bytes_write.sum", "DRAM write"),
    ("gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed", "DRAM throughput % of peak"),
    ("lts__t_sector_hit_rate.pct", "L2 hit rate %"),
    ("lts__throughput.avg.pct_of_peak_sustained_elapsed", "L2 throughput % of peak"),
    ("sm__warps_active.avg.pct_of_peak_sustained_active", "warps active % of peak"),
    ("sm__maximum_warps_per_active_cycle_pct", "occupancy limit %"),
    ("launch__registers_per_thread", "registers/thread"),
    ("launch__shared_mem_per_block_dynamic", "dynamic shared memory/block"),
    ("launch__grid_size", "grid"),
    ("launch__block_size", "block"),
    ("smsp__inst_executed.sum", "warp instructions"),
    ("smsp__issue_active.avg.pct_of_peak_sustained_active", "issue active %"),
    ("smsp__average_warps_issue_stalled_long_scoreboard_per_issue_active.ratio", "stall long scoreboard / issue"),
    ("smsp__average_warps_issue_stalled_short_scoreboard_per_issue_active.ratio", "stall short scoreboard / issue"),
    ("smsp__average_warps_issue_stalled_barrier_per_issue_active.ratio", "stall barrier / issue"),
    ("smsp__average_warps_issue_stalled_wait_per_issue_active.ratio", "stall wait / issue"),
    ("smsp__average_warps_issue_stalled_mio_throttle_per_issue_active.ratio", "stall MIO throttle / issue"),
    ("sm__pipe_tensor_cycles_active.avg.pct_of_peak_sustained_active", "tensor pipe active %"),
]


def full_report_markdown(raw_csv: str, title: str, command: str, note: str = "") -> str:
    """Summary of `ncu -i <report> --page raw --csv` output: one column per captured launch."""
    rows = [r for r in csv.reader(raw_csv.splitlines()) if r]
    hdr, units, data = rows[0], rows[1], rows[2:]
    col = {name: k for k, name in enumerate(hdr)}
    out = [f"# {title}", "", "Command (run from the repository root on one GB300):", "", "```", command, "```", ""]
    if note:
        out += [note, ""]
    kname = col.get("Kernel Name")
    out += ["| metric | " + " | ".join(f"launch {k + 1}" for k in range(len(data))) + " | unit |",
            "|---|" + "---:|" * len(data) + "---|"]
    if kname is not None:
        out.append("| kernel | " + " | ".join(f"`{short_name(r[kname]).split('(')[0]}`" for r in data) + " | |")
    for metric, label in FULL_METRICS:
        k = col.get(metric)
        if k is None:
            continue
        out.append(f"| {label} | " + " | ".join(r[k] for r in data) + f" | {units[k]} |")
    return "\n".join(out) + "\n"


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("csv")
    ap.add_argument("--workload", required=True)
    ap.add_argument("--mode", required=True)
    ap.add_argument("--command", required=True)
    ap.add_argument("--md")
    ap.add_argument("--traffic-json")
    ap.add_argument("--source-root", default=ROOT,
                    help="tree whose CUDA sources ran under ncu (e.g. a checkout of the profiled commit)")
    ap.add_argument("--full", action="store_true",
                    help="csv is `ncu -i <report> --page raw --csv` of a full capture: write its summary to --md")
    ap.add_argument("--title", default="")
    ap.add_argument("--note", default="")
    a = ap.parse_args(argv)
    if a.full:
        with open(a.csv) as f:
            text = full_report_markdown(f.read(), a.title or a.workload, a.command, a.note)
        with open(a.md, "w") as f:
            f.write(text)
        return
    s = summarise(read_launches(a.csv))
    if a.md:
        with open(a.md, "w") as f:
            f.write(markdown(s, f"Kernel launch list: {a.workload}, {a.mode} mode", a.command))
    if a.traffic_json:
        with open(a.traffic_json, "w") as f:
            json.dump(traffic_json(s, a.workload, a.mode, a.command, a.source_root), f, indent=1)
    if not a.md:
        print(markdown(s, f"{a.workload} {a.mode}", a.command))


if __name__ == "__main__":
    main()
