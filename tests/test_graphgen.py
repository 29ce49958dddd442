"""Structural checks of the seeded generators (no GPU)."""
import numpy as np
import pytest

import graphgen as gg
from helpers import check_csr


def _symmetric(g):
    src = np.repeat(np.arange(g.n), np.diff(g.offsets))
    fwd = set(zip(src.tolist(), g.targets.tolist(), g.weights.tolist()))
    rev = set(zip(g.targets.tolist(), src.tolist(), g.weights.tolist()))
    return fwd == rev


@pytest.mark.parametrize("make", [
    lambda: gg.sbm(2000, 20, 0.1, 0.002, 9),
    lambda: gg.rmat(12, weights=gg.W_INT8),
    lambda: gg.rmat(11, weights=gg.W_FP32),
    lambda: gg.grid(40, 50),
    lambda: gg.batch_sbm(4, 3),
])
def test_csr_is_symmetric_sorted_loopfree(make):
    g = make()
    check_csr(g)
    src = np.repeat(np.arange(g.n), np.diff(g.offsets))
    assert not np.any(src == g.targets)
    for i in range(0, g.n, max(1, g.n // 200)):
        row = g.targets[g.offsets[i]:g.offsets[i + 1]]
        assert np.all(np.diff(row) > 0)
    assert _symmetric(g)
    assert np.all(g.weights > 0)


def test_generators_are_deterministic():
    a, b = gg.rmat(12, seed=5), gg.rmat(12, seed=5)
    assert np.array_equal(a.targets, b.targets) and np.array_equal(a.weights, b.weights)
    c = gg.rmat(12, seed=6)
    assert not (a.n_arcs == c.n_arcs and np.array_equal(a.targets, c.targets))


def test_sbm_density_matches_parameters():
    g = gg.sbm(10000, 100, 0.1, 0.0005, 1)
    planted = gg.planted_blocks(10000, 100)
    src = np.repeat(np.arange(g.n), np.diff(g.offsets))
    intra = np.count_nonzero(planted[src] == planted[g.targets]) / 2
    inter = (g.n_arcs / 2) - intra
    exp_intra = 100 * 100 * 99 / 2 * 0.1
    exp_inter = (10000 * 9999 / 2 - 100 * 100 * 99 / 2) * 0.0005
    assert abs(intra - exp_intra) < 5 * np.sqrt(exp_intra)
    assert abs(inter - exp_inter) < 5 * np.sqrt(exp_inter)


def test_rmat_weights_and_hubs():
    g = gg.rmat(14, weights=gg.W_INT8)
    assert g.weights.min() >= 1 and g.weights.max() <= 8
    deg = g.degrees()
    assert deg[0] == deg.max()  # no scrambling: vertex 0 is the top hub
    gf = gg.rmat(10, weights=gg.W_FP32)
    assert gf.weights.dtype == np.float32 and gf.weights.min() > 0 and gf.weights.max() <= 1.0


def test_grid_degree():
    g = gg.grid(100, 100, 0.10, 0.01, 3)
    # 2*rows*cols-ish lattice edges, 90% kept, plus 1% long links
    exp_edges = (2 * 100 * 99) * 0.9 * 1.01
    assert abs(g.n_arcs / 2 - exp_edges) < 0.03 * exp_edges


def test_batch_params_ranges():
    for gi in range(50):
        n, k, p_in, p_out, seed = gg.batch_sbm_params(4, gi)
        assert 1000 <= n <= 200000 and 2 <= k <= 64
        assert 0 < p_out < p_in <= 1 and abs(p_out / p_in - 0.02) < 1e-12


@pytest.mark.parametrize("scale,fp", [(9, False), (11, True), (12, False)])
def test_tensor_rmat_equals_c_generator(scale, fp):
    """The tensor R-MAT (used on the GPU for scale 27) draws exactly graphgen.rmat's CSR; run here
    on CPU tensors, in small chunks so the chunk loop is exercised."""
    torch = pytest.importorskip("torch")
    from graphgen import device as gd
    o, t, w = gd.rmat(scale, 16, 0.57, 0.19, 0.19, 30 + scale, fp_weights=fp, device="cpu", chunk=1 << 13)
    g = gg.rmat(scale, 16, 0.57, 0.19, 0.19, 30 + scale, gg.W_FP32 if fp else gg.W_INT8)
    assert np.array_equal(o.numpy(), g.offsets)
    assert np.array_equal(t.numpy(), g.targets)
    assert np.array_equal(w.numpy(), g.weights)


def test_tensor_hash3_equals_c_hash3():
    torch = pytest.importorskip("torch")
    from graphgen import device as gd
    for a, b, c in [(0, 0, 0), (22, 12345, 3), (2**63 + 5, 2**40, 7)]:
        x = gd.hash3(torch.tensor(gd._s64(a)), gd._s64(b), gd._s64(c))
        assert int(x) & ((1 << 64) - 1) == gg.hash3(a, b, c)


def test_drop_isolated_keeps_every_arc():
    g = gg.from_edges(7, [(1, 3), (3, 5), (5, 1), (6, 6)], [2, 3, 4, 5])
    h = gg.drop_isolated(g)
    assert h.n == 4  # vertices 0, 2 and 4 had no arc
    old = {1: 0, 3: 1, 5: 2, 6: 3}
    arcs_g = sorted((old[u], old[int(v)], int(w)) for u in range(g.n)
                    for v, w in zip(g.targets[g.offsets[u]:g.offsets[u + 1]], g.weights[g.offsets[u]:g.offsets[u + 1]]))
    arcs_h = sorted((u, int(v), int(w)) for u in range(h.n)
                    for v, w in zip(h.targets[h.offsets[u]:h.offsets[u + 1]], h.weights[h.offsets[u]:h.offsets[u + 1]]))
    assert arcs_g == arcs_h
