"""The source hash that keeps stored DRAM counters valid only for the sources they were captured
on (paper_2312_04876_gb300.sources)."""
from __future__ import annotations

from paper_2312_04876_gb300 import sources as P


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
