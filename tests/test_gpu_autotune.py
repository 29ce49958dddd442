"""Autotuning (louvain_autotune / louvain_autotune_batch): the knobs it picks change only the
speed -- in deterministic mode the tuned run returns exactly the default run's membership -- and
every knob value it may pick is itself exact against the oracle (giant threshold 2048 moves rows
of 2049..4096 arcs to the multi-block giant path)."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(g):
    d = torch.device("cuda:0")
    return tuple(torch.from_numpy(a).to(d) for a in (g.offsets, g.targets, g.weights))


@pytest.fixture(scope="module")
def L(cuda_ok):
    import paper_2312_04876_gb300 as lv
    h = lv.Louvain(0)
    yield h
    h.close()


def test_autotune_keeps_the_result(L):
    g = gg.rmat(16, weights=gg.W_INT8, seed=22)  # hubs of 2049..4096 arcs and giants
    o, t, w = _dev(g)
    tuned, ms = L.autotune(o, t, w, mode="deterministic", reps=1)
    assert ms > 0.0
    assert tuned.giant_min_degree in (2048, 4096) and tuned.lm_blocks_per_sm in (4, 16) and tuned.compact in (0, 1)
    assert tuned.table_factor in (2, 4)
    m0, r0 = L.run(o, t, w, mode="deterministic")
    m1, r1 = L.run(o, t, w, params=tuned)
    assert torch.equal(m0, m1) and r0.modularity == r1.modularity


@pytest.mark.parametrize("giant_min", [2048, 4096])
def test_giant_threshold_is_exact(L, giant_min):
    g = gg.rmat(16, weights=gg.W_INT8, seed=22)
    o, t, w = _dev(g)
    mem, r = L.run(o, t, w, mode="deterministic", giant_min_degree=giant_min)
    ref_mem, ref_q, _, _ = oracle.louvain(g.offsets, g.targets, g.weights, oracle.default_params())
    assert np.array_equal(mem.cpu().numpy(), ref_mem) and r.modularity == ref_q


def test_autotune_batch(L):
    graphs = [gg.batch_sbm(4, k, n_lo=500.0, n_hi=4000.0) for k in range(12)]
    vo, offs, tg, wt = gg.concat(graphs)
    d = torch.device("cuda:0")
    o, t, w = (torch.from_numpy(a).to(d) for a in (offs, tg, wt))
    tuned, ms = L.autotune_batch(vo, o, t, w, mode="deterministic")
    assert ms > 0.0
    m0, per0, _ = L.run_batch(vo, o, t, w, mode="deterministic")
    m1, per1, _ = L.run_batch(vo, o, t, w, params=tuned)
    assert torch.equal(m0, m1)
