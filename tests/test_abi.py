"""The C ABI library builds, loads and exports every entry point include/louvain.h declares
(no GPU needed; no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "louvain.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(louvain_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2312_04876_gb300 import build as b
    path = b.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("louvain_create", "louvain_run", "louvain_run_host", "louvain_modularity", "louvain_destroy",
                 "louvain_default_params", "louvain_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol():
    from paper_2312_04876_gb300 import _native
    assert set(_declared()) == set(_native.SIGNATURES)


def test_default_params_are_the_papers():
    from paper_2312_04876_gb300 import default_params
    p = default_params()
    assert (p.max_iterations, p.tolerance, p.tolerance_drop, p.aggregation_tolerance, p.pruning) == (20, 0.01, 10.0,
                                                                                                      0.8, 1)
    assert p.max_passes == 10 and p.mode == 0 and p.validate == 1 and p.compact == 1


def test_status_strings(lib):
    lib.louvain_status_string.restype = ctypes.c_char_p
    assert lib.louvain_status_string(0) == b"LOUVAIN_OK"
    assert lib.louvain_status_string(3) == b"LOUVAIN_ERR_OVERFLOW"


def test_create_without_gpu_returns_status(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    h = ctypes.c_void_p()
    lib.louvain_create.restype = ctypes.c_int32
    rc = lib.louvain_create(ctypes.byref(h), 0, ctypes.c_size_t(0))
    assert rc == 5 and not h.value  # LOUVAIN_ERR_CUDA, no handle


def test_null_handle_is_rejected(lib):
    lib.louvain_run.restype = ctypes.c_int32
    rc = lib.louvain_run(None, 0, 0, None, None, None, 0, None, None, None, None, None, 0, None)
    assert rc == 1


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """The product path has no CPU fallback: without the built library every entry point raises."""
    from paper_2312_04876_gb300 import _native
    monkeypatch.setattr(_native, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _native.load(str(tmp_path / "liblouvain.so"))


def test_scan_wrappers_refuse_bad_tensors_before_any_library_call(monkeypatch):
    """The scan kernels read values[0, n) and write out[0, n] through raw pointers: a CPU tensor,
    another dtype or a strided view is refused by the binding before the library is touched."""
    import torch
    import paper_2312_04876_gb300 as lv
    from paper_2312_04876_gb300 import _native

    def no_library(*a, **k):
        raise AssertionError("library called")

    monkeypatch.setattr(_native, "load", no_library)
    for bad in (torch.arange(10, dtype=torch.int64), torch.arange(10, dtype=torch.int32),
                torch.arange(20, dtype=torch.int64)[::2], [1, 2, 3]):
        with pytest.raises(ValueError):
            lv.exclusive_scan_static(bad)


_STRUCTS = {"louvain_params": "Params", "louvain_pass_stats": "PassStats", "louvain_result": "Result",
            "louvain_graph_result": "GraphResult", "louvain_serve_result": "ServeResult",
            "louvain_kernel_stat": "KernelStat"}


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every struct of include/louvain.h has the same size and field offsets in the ctypes binding as
    a C compiler gives it (a field added on one side only would shift every later field)."""
    import shutil
    import subprocess
    from paper_2312_04876_gb300 import _native
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include "louvain.h"', "int main(void) {"]
    for cname, pyname in _STRUCTS.items():
        st = getattr(_native, pyname)
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in st._fields_:
            c_field = f[0][:-1] if f[0].endswith("_") else f[0]  # pass_ in Python is pass in C
            lines.append(f'  printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {c_field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], capture_output=True,
                       text=True)
    assert r.returncode == 0, r.stderr  # a field the binding names but the header lacks fails here
    got = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], capture_output=True,
                                                             text=True).stdout.splitlines())
    for cname, pyname in _STRUCTS.items():
        st = getattr(_native, pyname)
        assert int(got[f"{cname} size"]) == ctypes.sizeof(st), cname
        for f in st._fields_:
            assert int(got[f"{cname} {f[0]}"]) == getattr(st, f[0]).offset, (cname, f[0])


def _declared_arities():
    src = open(os.path.join(ROOT, "include", "louvain.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    out = {}
    for m in re.finditer(r"\b(louvain_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", src):
        args = " ".join(m.group(2).split())
        out[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    return out


def test_binding_argument_counts_match_the_header():
    """Each entry point takes as many arguments in the ctypes binding as the header declares (one
    missing or extra argument would hand the library a shifted argument list)."""
    from paper_2312_04876_gb300 import _native
    arity = _declared_arities()
    assert set(arity) == set(_native.SIGNATURES)
    for name, (_, argtypes) in _native.SIGNATURES.items():
        assert len(argtypes) == arity[name], name
