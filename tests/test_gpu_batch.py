"""Batched persistent launch and the serving loop on the GPU."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0912_4230_gb300 import lb, serve, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _lat(p, storage="fp32", stream=None):
    return lb.Lattice(p, storage=storage, kernel="cell", check_every=1, stream=stream)


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_batched_step_equals_separate_steps(storage):
    torch = pytest.importorskip("torch")
    s = torch.cuda.Stream()
    # the first three share the persistent launch; the 128 x 64 x 20 lattice
    # (1280 blocks, more than one resident wave) takes its own launch
    probs = [W.miscible(40, 36, 30, seed=1), W.miscible(64, 20, 17, seed=2),
             W.miscible(33, 48, 21, seed=3), W.miscible(128, 64, 20, seed=4)]
    sep = [_lat(p, storage) for p in probs]
    bat = [_lat(p, storage, stream=s.cuda_stream) for p in probs]
    for g in sep:
        g.step(70)
    lb.lb_step_batch([g.ctx for g in bat], 70)
    for p, a, b in zip(probs, sep, bat):
        fa, ha = a.populations()
        fb, hb = b.populations()
        assert np.array_equal(fa, fb) and np.array_equal(ha, hb)
        ra, rb = a.reduce(), b.reduce()
        assert np.array_equal(ra, rb)
        ua, ub = a.fields()[1], b.fields()[1]
        assert np.array_equal(ua, ub)
        assert a.t == b.t == 70


def test_batch_of_more_lattices_than_one_launch_holds():
    """70 lattices: two launches per step (64 + 6 lattices), each lattice
    bit-identical to stepping it alone; an odd step count leaves every
    context on the other buffer."""
    torch = pytest.importorskip("torch")
    s = torch.cuda.Stream()
    probs = [W.miscible(8 + (i % 5), 6 + (i % 3), 5 + (i % 4), seed=100 + i) for i in range(70)]
    sep = [_lat(p) for p in probs]
    bat = [_lat(p, stream=s.cuda_stream) for p in probs]
    for g in sep:
        g.step(9)
    lb.lb_step_batch([g.ctx for g in bat], 9)
    for a, b in zip(sep, bat):
        fa, ha = a.populations()
        fb, hb = b.populations()
        assert np.array_equal(fa, fb) and np.array_equal(ha, hb)
        assert np.array_equal(a.reduce(), b.reduce())
        assert np.array_equal(a.fields()[1], b.fields()[1])
        assert a.t == b.t == 9
    for g in sep + bat:
        g.close()


def test_batched_step_parity_with_oracle():
    p = W.miscible(24, 20, 18, seed=7)
    g = _lat(p)
    lb.lb_step_batch([g.ctx], 40)
    o = O.Oracle(p)
    o.step(40)
    _, u, C, _ = g.fields()
    _, ru, rC, _ = o.fields()
    assert np.abs(u - ru).max() <= 1e-5 * np.abs(ru).max()
    assert np.abs(C - rC).max() <= 1e-5


def test_serving_results_same_alone_and_in_the_mix():
    stream = W.requests(n=6, rate=200.0, seed=11, sides=(32, 48), steps_range=(60, 140))
    reqs = serve.make_requests(stream)
    be = serve.LibraryBackend("fp32")
    mixed = serve.Server(be, budget_bytes=2 * 10 ** 9, chunk=32).run(reqs)
    assert mixed["requests"] == 6 and mixed["max_resident"] >= 2
    for r in reqs:
        alone_req = serve.make_requests([q for q in stream if q["id"] == r.id])
        serve.Server(be, budget_bytes=2 * 10 ** 9, chunk=32).run(alone_req)
        a, b = r.result, alone_req[0].result
        for k in ("rho", "u", "C", "nu"):
            assert np.array_equal(a[k], b[k]), (r.id, k)
        assert np.array_equal(a["totals"], b["totals"])


def test_serving_in_a_packed_arena():
    """All lattices of the mix sub-allocated from one arena inside a torch
    tensor: the results equal those of lattices from cudaMalloc, the arena is
    empty afterwards, and its peak stays inside the budget."""
    torch = pytest.importorskip("torch")
    stream = W.requests(n=6, rate=200.0, seed=11, sides=(32, 48), steps_range=(60, 140))
    plain = serve.make_requests(stream)
    serve.Server(serve.LibraryBackend("fp32"), budget_bytes=2 * 10 ** 9, chunk=32).run(plain)
    budget = 2 * 10 ** 9
    region = torch.empty(budget, dtype=torch.uint8, device="cuda")
    arena = lb.Arena(budget, region.data_ptr())
    arena.use()
    try:
        reqs = serve.make_requests(stream)
        st = serve.Server(serve.LibraryBackend("fp32"), budget_bytes=budget, chunk=32).run(reqs)
    finally:
        lb.Arena.use_none()
    assert st["requests"] == 6
    stats = arena.stats()
    assert stats["used"] == 0 and stats["blocks"] == 0 and 0 < stats["peak"] <= budget
    for a, b in zip(plain, reqs):
        for k in ("rho", "u", "C", "nu"):
            assert np.array_equal(a.result[k], b.result[k]), (a.id, k)
        assert np.array_equal(a.result["totals"], b.result["totals"])
    arena.close()
