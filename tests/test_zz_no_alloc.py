"""louvain_exclusive_scan_static -- the scan entry point that allocates nothing.

It serves callers that cannot call cudaMalloc (a host application whose memory manager owns all
device memory, or a latency-critical loop that cannot take cudaMalloc's device-wide
synchronisation): its scratch lives in a fixed __device__ array inside the library.  This file is
collected last so that a run stopping at the first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _static_scan(lib, x, out):
    tot = ctypes.c_int64()
    st = lib.louvain_exclusive_scan_static(x.data_ptr(), out.data_ptr(), x.numel(),
                                           torch.cuda.current_stream().cuda_stream, ctypes.byref(tot))
    return st, int(tot.value)


def test_static_scan_matches_handle_scan_twice(cuda_ok):
    import paper_2312_04876_gb300 as lv
    from paper_2312_04876_gb300 import _native
    lib = _native.load()
    L = lv.Louvain(0)
    rng = np.random.default_rng(123)
    # two calls in a row on different data and sizes (several tiles, ragged tails): the second
    # call must not see anything the first left behind in the shared scratch
    for n in (3_000_017, 4_097):
        x = torch.from_numpy(rng.integers(0, 1 << 24, size=n, dtype=np.int64)).cuda()
        out = torch.full((n + 1,), -7, dtype=torch.int64, device="cuda")
        st, tot = _static_scan(lib, x, out)
        assert st == _native.OK
        ref, ref_tot = L.exclusive_scan(x)  # the existing entry point (handle workspace)
        assert tot == ref_tot
        assert torch.equal(out, ref)
    L.close()


def test_static_scan_limits(cuda_ok):
    from paper_2312_04876_gb300 import _native, STATIC_SCAN_MAX
    lib = _native.load()
    x = torch.zeros(1, dtype=torch.int64, device="cuda")
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    tot = ctypes.c_int64()
    # a count beyond the fixed scratch is rejected before anything runs
    assert lib.louvain_exclusive_scan_static(x.data_ptr(), out.data_ptr(), STATIC_SCAN_MAX + 1,
                                             None, ctypes.byref(tot)) == _native.ERR_INVALID
    # an empty input writes the zero total
    assert lib.louvain_exclusive_scan_static(x.data_ptr(), out.data_ptr(), 0, None, ctypes.byref(tot)) == _native.OK
    assert tot.value == 0 and int(out[0]) == 0
