"""Host-side ncu summaries (paper_2312_04876_gb300.profiling): kernel-class mapping, launch-list
grouping with DRAM bytes per class invocation, and the full-capture summary table."""
from __future__ import annotations

from paper_2312_04876_gb300 import profiling as P


def _launch_csv(rows):
    hdr = ['"ID"', '"Kernel Name"', '"Grid Size"', '"Block Size"', '"Metric Name"', '"Metric Unit"', '"Metric Value"']
    out = [",".join(hdr)]
    for lid, name, metric, unit, value in rows:
        out.append(",".join(f'"{x}"' for x in (lid, name, "(1, 1, 1)", "(256, 1, 1)", metric, unit, value)))
    return "\n".join(out) + "\n"


def test_kernel_classes():
    assert P.kernel_class("lm_kernel<IntMode, 32, 8, 0>") == "local_move_b2_warp"
    assert P.kernel_class("lm_kernel<IntMode, 256, 13, 0>") == "local_move_b5_block8k"
    assert P.kernel_class("merge_kernel<IntMode, 4, 3, 0>") == "merge_b0_g4"
    assert P.kernel_class("k_glm_scan<IntMode>") == "local_move_b6_giant"
    assert P.kernel_class("k_giant_mg_emit<IntMode>") == "merge_b6_giant"
    assert P.kernel_class("k_gplan_scan") is None
    assert P.kernel_class("k_mod_group<IntMode, 4>") == "modularity"
    assert P.short_name("void lv::lm_kernel<IntMode, 4, 3, 0>(LmArgs<IntMode>)") == "lm_kernel<IntMode, 4, 3, 0>"


def test_launch_list_summary(tmp_path):
    rows = []
    lid = 0
    # two giant local-move invocations (plan kernel + insert + scan each) and one warp launch
    for _ in range(2):
        for name, t, rd in (("k_gplan_counts", "1", "0"), ("k_glm_insert<IntMode>", "10", "1"),
                            ("k_glm_scan<IntMode>", "5", "2")):
            rows += [(lid, f"void {name}(int)", "gpu__time_duration.sum", "us", t),
                     (lid, f"void {name}(int)", "dram__bytes_read.sum", "MB", rd),
                     (lid, f"void {name}(int)", "dram__bytes_write.sum", "MB", "0")]
            lid += 1
    rows += [(lid, "void lm_kernel<IntMode, 32, 8, 0>(LmArgs<IntMode>)", "gpu__time_duration.sum", "us", "4"),
             (lid, "void lm_kernel<IntMode, 32, 8, 0>(LmArgs<IntMode>)", "dram__bytes_read.sum", "MB", "3"),
             (lid, "void lm_kernel<IntMode, 32, 8, 0>(LmArgs<IntMode>)", "dram__bytes_write.sum", "MB", "1")]
    f = tmp_path / "l.csv"
    f.write_text(_launch_csv(rows))
    s = P.summarise(P.read_launches(str(f)))
    assert s["launches"] == 7
    assert abs(s["total_ns"] - 36e3) < 1e-6
    g = s["classes"]["local_move_b6_giant"]
    assert g["launches"] == 2 and g["kernel_launches"] == 6  # the plan kernels join their invocation
    assert abs(g["dram"] - 6e6) < 1e-3
    w = s["classes"]["local_move_b2_warp"]
    assert w["launches"] == 1 and abs(w["dram"] - 4e6) < 1e-3
    md = P.markdown(s, "t", "cmd")
    assert "local_move_b6_giant" in md and "cmd" in md
    tj = P.traffic_json(s, "rmat22", "fast", "cmd")
    assert abs(tj["classes"]["local_move_b6_giant"]["dram_bytes_per_launch"] - 3e6) < 1e-3
    assert len(tj["source_sha256"]) == 64


def test_full_report_summary():
    hdr = ["ID", "Kernel Name", "gpu__time_duration.sum", "dram__bytes_read.sum", "launch__grid_size",
           "smsp__average_warps_issue_stalled_long_scoreboard_per_issue_active.ratio"]
    units = ["", "", "us", "Mbyte", "", "inst"]
    data = [["0", "void k_glm_insert<IntMode>(int)", "53.2", "22.3", "1216", "48.1"],
            ["1", "void k_glm_scan<IntMode>(int)", "44.1", "22.0", "1216", "25.8"]]
    raw = "\n".join(",".join(f'"{x}"' for x in r) for r in [hdr, units] + data) + "\n"
    md = P.full_report_markdown(raw, "title", "the command", "a note")
    lines = md.splitlines()
    assert lines[0] == "# title" and "the command" in md and "a note" in md
    assert "| kernel | `k_glm_insert<IntMode>` | `k_glm_scan<IntMode>` | |" in lines
    assert "| duration | 53.2 | 44.1 | us |" in lines
    assert "| stall long scoreboard / issue | 48.1 | 25.8 | inst |" in lines


def test_source_hash_ignores_comments_only(tmp_path):
    csrc = tmp_path / "paper_2312_04876_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "include").mkdir()
    (tmp_path / "include" / "louvain.h").write_text("int f(int);  /* public */\n")
    base = '#define W 4\nint g(int x) {  // doubles\n  return 2 * x + W; /* s */ }\nconst char* m = "a // b";\n'
    k = csrc / "k.cu"
    k.write_text(base)
    h0 = P.source_sha256(str(tmp_path))
    # comments edited, lines re-indented, a comment-only line added: same code, same hash
    k.write_text('#define W 4\n// new note\nint g(int x) {    // twice x\n    return 2 * x + W;   }\n'
                 'const char* m = "a // b";\n')
    assert P.source_sha256(str(tmp_path)) == h0
    # a change inside a string literal, to an operator, or a joined preprocessor line is a change
    for edit in (base.replace("a // b", "a  // b"), base.replace("2 * x", "3 * x"),
                 base.replace("#define W 4\nint", "#define W 4 int")):
        k.write_text(edit)
        assert P.source_sha256(str(tmp_path)) != h0
    assert P.strip_comments("a  =  1; // c\n  b /* d */ = '/';") == "a = 1;\nb = '/';"
