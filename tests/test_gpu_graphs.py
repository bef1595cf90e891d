"""CUDA-graph replay of step pairs (lb_step, lb_step_batch) against direct
launches: the same kernels with the same arguments, so every population,
field and FP64 total is bit-identical."""
import numpy as np
import pytest

from paper_0912_4230_gb300 import lb, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _same(a, b):
    fa, ha = a.populations()
    fb, hb = b.populations()
    assert np.array_equal(fa, fb)
    if ha is not None:
        assert np.array_equal(ha, hb)
    assert np.array_equal(a.reduce(), b.reduce())
    for x, y in zip(a.fields(), b.fields()):
        assert np.array_equal(x, y)
    assert a.t == b.t


@pytest.mark.parametrize("storage", ["fp32", "fp64", "fp16"])
@pytest.mark.parametrize("check_every", [1, 0])
def test_step_graph_equals_direct_launches(storage, check_every):
    """Solids, walls, solute inlet/outlet, full K: 1 + 37 + 6 steps (an odd
    start parity, pairs from the graph, the exporting last step direct)."""
    p = W.random_medium(19, 13, 11, seed=5)
    g = lb.Lattice(p, storage=storage, check_every=check_every)
    d = lb.Lattice(p, storage=storage, check_every=check_every)
    d.set_graphs(False)
    for n in (1, 37, 6):
        g.step(n)
        d.step(n)
        _same(g, d)
    assert lb.lb_debug_graphs(g.ctx) & 1
    assert lb.lb_debug_graphs(d.ctx) == 0


def test_step_graph_after_autotune_and_reinit():
    """The graph is dropped when the autotuner changes the launch shape and
    stays valid across lb_init."""
    p = W.miscible(64, 48, 40, seed=2)
    g = lb.Lattice(p, storage="fp32")
    d = lb.Lattice(p, storage="fp32")
    d.set_graphs(False)
    g.step(11)
    d.step(11)
    lb.lb_autotune(g.ctx, 2)
    lb.lb_autotune(d.ctx, 2)
    g.step(21)
    d.step(21)
    _same(g, d)
    g.init()
    d.init()
    g.step(15)
    d.step(15)
    _same(g, d)


def test_time_dependent_law_is_not_replayed():
    """The hardening law reads t, so its steps are launched directly."""
    p = W.wood(nx=30, ny=40, wood_depth=30)
    g = lb.Lattice(p, storage="fp32")
    g.step(9)
    assert lb.lb_debug_graphs(g.ctx) == 0


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_batch_graph_equals_direct_launches(storage):
    """A batch with a lattice on its own launch and several sharing the
    persistent launch; then a different membership (the graph is captured
    again) and a changed order."""
    torch = pytest.importorskip("torch")
    s = torch.cuda.Stream()
    probs = [W.miscible(40, 36, 30, seed=1), W.miscible(64, 20, 17, seed=2),
             W.miscible(33, 48, 21, seed=3), W.miscible(128, 64, 20, seed=4),
             W.miscible(16, 16, 16, seed=5)]
    g = [lb.Lattice(q, storage=storage, kernel="cell", stream=s.cuda_stream) for q in probs]
    d = [lb.Lattice(q, storage=storage, kernel="cell", stream=s.cuda_stream) for q in probs]
    for x in d:
        x.set_graphs(False)
    lb.lb_step_batch([x.ctx for x in g], 25)
    lb.lb_step_batch([x.ctx for x in d], 25)
    assert lb.lb_debug_graphs(g[0].ctx) & 2
    assert lb.lb_debug_graphs(d[0].ctx) == 0
    for a, b in zip(g, d):
        _same(a, b)
    sub = [4, 0, 2]
    lb.lb_step_batch([g[i].ctx for i in sub], 12)
    lb.lb_step_batch([d[i].ctx for i in sub], 12)
    lb.lb_step_batch([g[i].ctx for i in reversed(sub)], 8)
    lb.lb_step_batch([d[i].ctx for i in reversed(sub)], 8)
    for i in range(len(probs)):
        _same(g[i], d[i])


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_free_surface_steps_from_the_graph(storage):
    """The free-surface step (five passes over device-side tile lists, the
    stamp counter on the device) replayed from a graph: cell types, liquid
    mass and populations bit-identical to direct launches."""
    p = W.drop(nx=24, ny=24, nz=28, R=5.0, gap=6.0, seed=3)
    g = lb.Lattice(p, storage=storage)
    d = lb.Lattice(p, storage=storage)
    d.set_graphs(False)
    for n in (1, 31, 40):
        g.step(n)
        d.step(n)
        ta, ma = g.free_surface_state()
        tb, mb = d.free_surface_state()
        assert np.array_equal(ta, tb) and np.array_equal(ma, mb)
        fa, _ = g.populations()
        fb, _ = d.populations()
        assert np.array_equal(fa, fb)
        assert g.t == d.t
    assert lb.lb_debug_graphs(g.ctx) & 1
