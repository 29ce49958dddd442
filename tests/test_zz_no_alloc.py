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


def _static_scan(lib, x_ptr, out_ptr, n):
    tot = ctypes.c_int64()
    st = lib.louvain_exclusive_scan_static(x_ptr, out_ptr, n, torch.cuda.current_stream().cuda_stream,
                                           ctypes.byref(tot))
    return st, int(tot.value)


def _cumsum_exclusive(x: np.ndarray) -> np.ndarray:
    return np.concatenate([[0], np.cumsum(x)]).astype(np.int64)


def test_static_scan_matches_handle_scan_twice(cuda_ok):
    import paper_2312_04876_gb300 as lv
    from paper_2312_04876_gb300 import _native
    lib = _native.load()
    L = lv.Louvain(0)
    rng = np.random.default_rng(123)
    # two calls in a row on different data and sizes (several tiles, ragged tails): the second
    # call must not see anything the first left behind in the shared scratch
    for n in (3_000_017, 4_097):
        xh = rng.integers(0, 1 << 24, size=n, dtype=np.int64)
        x = torch.from_numpy(xh).cuda()
        out = torch.full((n + 1,), -7, dtype=torch.int64, device="cuda")
        st, tot = _static_scan(lib, x.data_ptr(), out.data_ptr(), n)
        assert st == _native.OK
        ref, ref_tot = L.exclusive_scan(x)  # the existing entry point (handle workspace)
        assert tot == ref_tot
        assert torch.equal(out, ref)
        # and the definition itself, on the host
        assert np.array_equal(out.cpu().numpy(), _cumsum_exclusive(xh))
    L.close()


def test_static_scan_in_place_and_through_the_binding(cuda_ok):
    import paper_2312_04876_gb300 as lv
    from paper_2312_04876_gb300 import _native
    lib = _native.load()
    rng = np.random.default_rng(7)
    n = 1_234_567
    xh = rng.integers(-(1 << 30), 1 << 30, size=n, dtype=np.int64)
    ref = _cumsum_exclusive(xh)
    # in place: input in buf[0, n), result over the same buffer plus the total in buf[n]
    buf = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    buf[:n] = torch.from_numpy(xh).cuda()
    st, tot = _static_scan(lib, buf.data_ptr(), buf.data_ptr(), n)
    assert st == _native.OK and tot == int(ref[-1])
    assert np.array_equal(buf.cpu().numpy(), ref)
    # the Python wrapper, with and without a caller-provided output
    out, tot = lv.exclusive_scan_static(torch.from_numpy(xh).cuda())
    assert tot == int(ref[-1]) and np.array_equal(out.cpu().numpy(), ref)
    own = torch.full((n + 5,), 3, dtype=torch.int64, device="cuda")
    out, tot = lv.exclusive_scan_static(torch.from_numpy(xh).cuda(), own)
    assert out is own and np.array_equal(own[:n + 1].cpu().numpy(), ref) and int(own[n + 1]) == 3
    # arguments the kernels cannot take are refused before any library call
    x = torch.from_numpy(xh).cuda()
    with pytest.raises(ValueError):
        lv.exclusive_scan_static(x, torch.empty(n, dtype=torch.int64, device="cuda"))  # one short
    with pytest.raises(ValueError):
        lv.exclusive_scan_static(x.to(torch.int32))
    with pytest.raises(ValueError):
        lv.exclusive_scan_static(x[::2])


def test_static_scan_at_the_maximum_count(cuda_ok):
    """2^26 elements: the tile sums fill all 2^14 entries of the fixed scratch."""
    import paper_2312_04876_gb300 as lv
    n = lv.STATIC_SCAN_MAX
    x = torch.randint(0, 1 << 20, (n,), dtype=torch.int64, device="cuda")
    out, tot = lv.exclusive_scan_static(x)
    ref = torch.cumsum(x, 0)
    assert tot == int(ref[-1])
    assert int(out[0]) == 0 and torch.equal(out[1:], ref)
    del x, out, ref
    torch.cuda.empty_cache()


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
