"""Graphs whose arcs do not fit in HBM (params.host_arcs = 1): the input's targets and weights are
read in place from host memory and the super-vertex graphs' arc buffers live in pinned host memory,
both reached by the kernels over NVLink-C2C; per-vertex state stays in HBM.  The results must be
those of the default placement -- identical to the CPU oracle in deterministic integer mode -- and
the run must fit under an HBM budget that the default placement cannot meet."""
from __future__ import annotations

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def rmat16():
    g = gg.rmat(16, weights=gg.W_INT8, seed=22)
    ref = oracle.louvain(g.offsets, g.targets, g.weights, oracle.default_params(seed=4))
    return g, ref


def test_host_input_and_host_arc_buffers_bit_exact(cuda_ok, rmat16):
    import paper_2312_04876_gb300 as lv
    g, (ref_mem, ref_q, ref_passes, ref_stats) = rmat16
    L = lv.Louvain(0)
    # input read in place from pageable host memory (registered for the call)
    m1, r1 = L.run_host(g.offsets, g.targets, g.weights, mode="deterministic", seed=4, host_arcs=1)
    assert np.array_equal(m1, ref_mem) and r1.modularity == ref_q and r1.passes == ref_passes
    # input already pinned (left registered as it was)
    po, pt, pw = (torch.from_numpy(a).pin_memory() for a in (g.offsets, g.targets, g.weights))
    m2, r2 = L.run_host(po, pt, pw, mode="deterministic", seed=4, host_arcs=1)
    assert np.array_equal(m2, ref_mem) and r2.modularity == ref_q
    # device-resident input, super-vertex graphs in host memory
    o, t, w = (torch.from_numpy(a).to(DEV) for a in (g.offsets, g.targets, g.weights))
    m3, r3 = L.run(o, t, w, mode="deterministic", seed=4, host_arcs=1)
    assert np.array_equal(m3.cpu().numpy(), ref_mem)
    assert [s["iterations"] for s in r3.stats] == [s["iterations"] for s in ref_stats]
    # and back to the default placement on the same handle
    m4, _ = L.run(o, t, w, mode="deterministic", seed=4)
    assert np.array_equal(m4.cpu().numpy(), ref_mem)
    L.close()


def test_host_arcs_fit_a_budget_the_default_placement_cannot(cuda_ok):
    import paper_2312_04876_gb300 as lv
    g = gg.rmat(18, weights=gg.W_INT8, seed=22)
    ref_mem, ref_q, _, _ = oracle.louvain(g.offsets, g.targets, g.weights, oracle.default_params())
    L = lv.Louvain(0)
    L.run_host(g.offsets, g.targets, g.weights, mode="deterministic")
    full = L.workspace_bytes()
    L.close()
    budget = int(full * 0.55)
    L = lv.Louvain(0, hbm_budget_bytes=budget)
    with pytest.raises(lv.LouvainError) as e:
        L.run_host(g.offsets, g.targets, g.weights, mode="deterministic")
    assert e.value.status == 2  # LOUVAIN_ERR_OOM
    m, r = L.run_host(g.offsets, g.targets, g.weights, mode="deterministic", host_arcs=1)
    assert np.array_equal(m, ref_mem) and r.modularity == ref_q
    assert L.workspace_bytes() <= budget
    # fast mode under the same budget: a valid partition within 0.005 of the oracle
    m, r = L.run_host(g.offsets, g.targets, g.weights, mode="fast", host_arcs=1, validate=0)
    assert m.min() == 0 and m.max() == r.n_communities - 1 and r.modularity >= ref_q - 0.005
    L.close()


def test_host_arcs_fp32(cuda_ok):
    import paper_2312_04876_gb300 as lv
    g = gg.rmat(14, weights=gg.W_FP32, seed=8)
    _, ref_q, _, _ = oracle.louvain(g.offsets, g.targets, g.weights, oracle.default_params())
    L = lv.Louvain(0)
    m, r = L.run_host(g.offsets, g.targets, g.weights, mode="deterministic", host_arcs=1)
    assert abs(r.modularity - ref_q) <= 1e-4
    assert abs(oracle.modularity(g.offsets, g.targets, g.weights, m) - r.modularity) <= 1e-10
    L.close()
