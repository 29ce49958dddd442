"""Hash of the library's CUDA sources and public header, with comments and layout left out.

The benchmark keeps DRAM counters captured by Nsight Compute beside the sources they were
captured on; it reports them only while this hash still matches, so any code change voids them
while a comment edit or a re-indent does not.
"""
from __future__ import annotations

import hashlib
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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
