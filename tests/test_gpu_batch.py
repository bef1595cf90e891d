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


@pytest.mark.parametrize("storage", ["fp16", "fp32"])
def test_serving_same_alone_and_in_the_mix_as_timed(storage):
    """The serving configuration the benchmark times: lattices sub-allocated
    from one packed arena, created and initialised on an admission thread and
    stream while the resident ones step on the step stream, step pairs
    replayed from CUDA graphs, only the oldest requests stepped each chunk
    (fill_cells), FP16 and FP32 storage. Every request's fields and totals
    are bit-identical to the same request served alone the same way."""
    torch = pytest.importorskip("torch")
    stream = W.requests(n=8, rate=400.0, seed=13, sides=(32, 48, 64), steps_range=(60, 180))
    budget = 3 * 10 ** 9
    region = torch.empty(budget, dtype=torch.uint8, device="cuda")
    arena = lb.Arena(budget, region.data_ptr())
    step_s, admit_s = torch.cuda.Stream(), torch.cuda.Stream()

    def serve_all(reqs):
        be = serve.LibraryBackend(storage, keep_fields=True, batched=True,
                                  admit_stream=admit_s, step_stream=step_s)
        srv = serve.Server(be, budget_bytes=budget, chunk=24, fill_cells=120000,
                           admit_in_thread=True)
        st = srv.run(reqs)
        torch.cuda.synchronize()
        return st, srv

    arena.use()
    try:
        mixed = serve.make_requests(stream, storage=storage)
        st, srv = serve_all(mixed)
        assert st["requests"] == 8 and st["max_resident"] >= 2
        assert any(e["stepped"] < e["resident"] for e in srv.log)   # fill_cells took a subset
        for r in mixed:
            alone = serve.make_requests([q for q in stream if q["id"] == r.id], storage=storage)
            serve_all(alone)
            a, b = r.result, alone[0].result
            for k in ("rho", "u", "C", "nu"):
                assert np.array_equal(a[k], b[k]), (storage, r.id, k)
            assert np.array_equal(a["totals"], b["totals"]), (storage, r.id)
    finally:
        lb.Arena.use_none()
    assert arena.stats()["used"] == 0
    arena.close()


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


def test_release_callback_waits_for_the_stream():
    """A caller's allocator may reuse a released block at once (the packed
    arena does): when the leader's batch work list grows, its old list is
    released only after the launches queued on the leader's stream, which may
    still read it, have finished. The release callback sees an idle stream
    every time, and the grown batch still computes what separate steps do."""
    torch = pytest.importorskip("torch")
    s = torch.cuda.Stream()
    busy = []

    def alloc(n):
        return torch.cuda.caching_allocator_alloc(n, stream=s)

    def release(p):
        busy.append(not s.query())
        torch.cuda.caching_allocator_delete(p)

    lb.lb_set_allocator(alloc, release)
    try:
        probs = [W.miscible(48, 40, 36, seed=20 + i) for i in range(3)]
        bat = [_lat(p, stream=s.cuda_stream) for p in probs]
    finally:
        lb.lb_set_allocator(None, None)
    ref = [_lat(p) for p in probs]
    # one lattice queues 200 steps on s, then the work list grows to three
    lb.lb_step_batch([bat[0].ctx], 200)
    lb.lb_step_batch([g.ctx for g in bat], 5)
    ref[0].step(200)
    for g in ref:
        g.step(5)
    assert busy and not any(busy)
    for a, b in zip(ref, bat):
        fa, ha = a.populations()
        fb, hb = b.populations()
        assert np.array_equal(fa, fb) and np.array_equal(ha, hb)
    for g in bat + ref:
        g.close()


@pytest.mark.parametrize("storage,which", [("fp32", "miscible"), ("fp16", "precision"),
                                           ("fp64", "miscible")])
def test_bytes_required_is_the_arena_peak(storage, which):
    """The admission size (lb_bytes_required through serve.device_bytes) is
    the packed arena's peak for one lattice that is created, initialised,
    stepped, exported and reduced, less its share of a batch work list (not
    taken when it steps alone): the query and the allocation share one
    layout."""
    torch = pytest.importorskip("torch")
    p = (W.miscible(40, 36, 30, seed=1) if which == "miscible"
         else W.precision(32, 32, 32, seed=2))
    need = serve.device_bytes(p, storage)
    region = torch.empty(need + (1 << 20), dtype=torch.uint8, device="cuda")
    arena = lb.Arena(need + (1 << 20), region.data_ptr())
    arena.use()
    try:
        g = _lat(p, storage)
    finally:
        lb.Arena.use_none()
    g.step(3)
    g.fields()
    g.reduce()
    dom = lb.make_domain(p)
    gx = -(-p.nx // 64) if p.nx > 32 else 1
    blocks = gx * -(-p.ny // (128 // (64 if p.nx > 32 else 32))) * p.nz
    share = -(-8 * blocks // 256) * 256
    assert arena.stats()["peak"] == need - share, (arena.stats(), need, share)
    assert lb.lb_bytes_required(dom, lb.make_params(p, storage), 6) >= need
    g.close()
    assert arena.stats()["used"] == 0
    arena.close()
