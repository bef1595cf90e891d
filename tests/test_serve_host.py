"""Host-side logic of the serving loop (CPU only, fake stepping backend):
admission by HBM budget in arrival order, continuous batching in chunks,
memory released at completion, latency statistics."""
import numpy as np
import pytest

from paper_0912_4230_gb300 import serve, workloads as W


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += dt


class FakeBackend:
    """Each step of each resident lattice costs N * 1e-9 s on the fake clock."""

    def __init__(self, clock, per_lup=1e-9):
        self.clock, self.per_lup = clock, per_lup
        self.resident = set()
        self.batches = []

    def bytes(self, prob):
        return prob.N * 100

    def admit(self, prob):
        h = object()
        self.resident.add(h)
        return (h, prob.N)

    def step(self, handles, n):
        self.batches.append(len(handles))
        self.clock.t += n * sum(N for _, N in handles) * self.per_lup

    def finish(self, handle):
        self.resident.discard(handle[0])
        return "ok"


def _reqs(specs):
    out = []
    for i, (arr, side, steps) in enumerate(specs):
        p = W.gaussian_pulse(side, side, side)  # any problem: only its size matters here
        out.append(serve.Request(id=i, arrival=arr, steps=steps, problem=p))
    return out


def test_admission_respects_budget_and_order():
    clk = FakeClock()
    be = FakeBackend(clk)
    reqs = _reqs([(0.0, 10, 300), (0.0, 10, 300), (0.0, 10, 300)])
    srv = serve.Server(be, budget_bytes=2 * 1000 * 100, chunk=100, clock=clk, sleep=clk.sleep)
    st = srv.run(reqs)
    assert st["requests"] == 3
    assert st["max_resident"] == 2          # the third waits for memory
    assert all(e["used"] <= 2 * 1000 * 100 for e in srv.log)
    assert reqs[2].admitted >= reqs[0].done  # admitted only after one finished
    assert not be.resident                  # everything released


def test_late_arrivals_join_running_batches():
    clk = FakeClock()
    be = FakeBackend(clk)
    # the first request runs 1000 steps; the second arrives while it runs
    reqs = _reqs([(0.0, 10, 1000), (2e-6 * 300, 10, 200)])
    srv = serve.Server(be, budget_bytes=10 ** 9, chunk=100, clock=clk, sleep=clk.sleep)
    st = srv.run(reqs)
    assert 2 in be.batches                  # both lattices advanced in one batch
    assert reqs[1].done < reqs[0].done      # the short late request finished first
    assert st["p99_s"] >= st["p50_s"] > 0


def test_idle_server_waits_for_arrivals():
    clk = FakeClock()
    be = FakeBackend(clk)
    reqs = _reqs([(5.0, 8, 10)])
    st = serve.Server(be, budget_bytes=10 ** 9, chunk=10, clock=clk, sleep=clk.sleep).run(reqs)
    assert reqs[0].admitted >= 5.0 and st["requests"] == 1


def test_request_above_budget_is_refused():
    clk = FakeClock()
    be = FakeBackend(clk)
    with pytest.raises(ValueError):
        serve.Server(be, budget_bytes=10, clock=clk, sleep=clk.sleep).run(_reqs([(0.0, 8, 10)]))


def test_device_bytes_scale():
    """The library's size query, through the serving estimate: 16-bit storage
    takes less than FP32 and more than half of it; a 128^3 lattice holds at
    least its two FP32 buffers of f and h."""
    p = W.miscible(64, 64, 64)
    b32, b16 = serve.device_bytes(p, "fp32"), serve.device_bytes(p, "fp16")
    assert b16 < b32 < 2 * b16 + 64 ** 3 * 100
    assert serve.device_bytes(W.miscible(128, 128, 128)) > 2 * 2 * 19 * 4 * 128 ** 3


def test_request_stream_matches_the_serving_workload():
    rs = W.requests(n=256, rate=50.0, seed=5)
    gaps = np.diff([0.0] + [r["arrival"] for r in rs])
    assert len(rs) == 256 and abs(gaps.mean() - 1 / 50.0) < 0.3 / 50.0
    assert {r["nx"] for r in rs} <= {32, 48, 64, 96, 128, 160}
    assert all(r["nx"] <= r["nz"] <= 2 * r["nx"] + 1 for r in rs)
    assert all(2000 <= r["steps"] <= 20000 for r in rs)


def test_fill_policy_steps_oldest_first():
    clk = FakeClock()
    be = FakeBackend(clk)
    # three 1000-cell lattices resident together; fill_cells = 1500 steps two at a time
    reqs = _reqs([(0.0, 10, 200), (0.0, 10, 200), (0.0, 10, 200)])
    srv = serve.Server(be, budget_bytes=10 ** 9, chunk=100, clock=clk, sleep=clk.sleep,
                       fill_cells=1500)
    st = srv.run(reqs)
    assert st["requests"] == 3
    assert max(be.batches) == 2
    assert reqs[2].done > reqs[0].done and reqs[2].done > reqs[1].done


class SleepBackend:
    """Real-time fake: admission and steps take wall time."""

    def __init__(self):
        import threading
        self.lock = threading.Lock()
        self.resident = 0
        self.max_resident = 0

    def bytes(self, prob):
        return prob.N * 100

    def admit(self, prob):
        import time
        time.sleep(0.002)
        with self.lock:
            self.resident += 1
            self.max_resident = max(self.max_resident, self.resident)
        return prob.N

    def step(self, handles, n):
        import time
        time.sleep(1e-5 * n)

    def finish(self, handle):
        with self.lock:
            self.resident -= 1
        return "ok"


def test_admission_thread_overlaps_and_respects_budget():
    be = SleepBackend()
    reqs = _reqs([(0.0, 10, 300), (0.001, 10, 200), (0.002, 10, 100), (0.05, 10, 100)])
    srv = serve.Server(be, budget_bytes=2 * 1000 * 100, chunk=50, admit_in_thread=True)
    st = srv.run(reqs)
    assert st["requests"] == 4
    assert be.max_resident <= 2 and be.resident == 0
    assert all(r.done >= r.admitted >= r.arrival for r in reqs)


class ArenaBackend(FakeBackend):
    """Device memory from a fixed arena (the library's first-fit arena on a
    host region): admit raises MemoryError when the lattice does not fit, even
    if the estimate said it would."""

    def __init__(self, clock, arena, scale=1.5):
        super().__init__(clock)
        self.arena, self.scale = arena, scale
        self.blocks = {}

    def admit(self, prob):
        p = self.arena.alloc(int(self.bytes(prob) * self.scale))   # estimate too low
        if p is None:
            raise MemoryError("arena full")
        h, N = super().admit(prob)
        self.blocks[h] = p
        return (h, N)

    def finish(self, handle):
        self.arena.free(self.blocks.pop(handle[0]))
        return super().finish(handle)


@pytest.mark.parametrize("threaded", [False, True])
def test_admission_waits_when_the_arena_is_short(threaded):
    """The estimate admits three requests under the budget but the arena
    holds two: the third is admitted after one finishes, every request
    completes, and the arena is empty at the end."""
    import time
    from paper_0912_4230_gb300 import lb
    buf = np.zeros((1 << 20) + 256, np.uint8)
    base = (buf.ctypes.data + 255) // 256 * 256
    side = 10                                  # 1000 cells: estimate 100 000 bytes
    arena = lb.Arena(2 * 150_000 + 4096, base)
    if threaded:
        clock, sleep = time.perf_counter, time.sleep
        be = ArenaBackend(None, arena)
        be.step = lambda handles, n: None
    else:
        clk = FakeClock()
        clock, sleep = clk, clk.sleep
        be = ArenaBackend(clk, arena)
    reqs = _reqs([(0.0, side, 300), (0.0, side, 300), (0.0, side, 300)])
    srv = serve.Server(be, budget_bytes=10 ** 7, chunk=100, clock=clock, sleep=sleep,
                       admit_in_thread=threaded)
    st = srv.run(reqs)
    assert st["requests"] == 3
    assert reqs[2].admitted >= min(reqs[0].done, reqs[1].done)
    assert arena.stats()["used"] == 0
    arena.close()


def test_admission_fails_when_nothing_can_free_memory():
    from paper_0912_4230_gb300 import lb
    buf = np.zeros((1 << 16) + 256, np.uint8)
    base = (buf.ctypes.data + 255) // 256 * 256
    arena = lb.Arena(1 << 16, base)
    clk = FakeClock()
    be = ArenaBackend(clk, arena)
    srv = serve.Server(be, budget_bytes=10 ** 7, chunk=100, clock=clk, sleep=clk.sleep)
    with pytest.raises(MemoryError):
        srv.run(_reqs([(0.0, 10, 100)]))       # 150 000 bytes > the 64 KiB arena
    arena.close()


def test_admission_thread_failure_ends_the_run():
    """An error while admitting on the background thread (here an invalid
    request) is raised by run() instead of leaving it waiting."""
    import time

    class Failing(FakeBackend):
        def admit(self, prob):
            if prob.N > 500:
                raise ValueError("invalid request")
            return super().admit(prob)

    be = Failing(None)
    be.step = lambda handles, n: None
    srv = serve.Server(be, budget_bytes=10 ** 9, chunk=10, clock=time.perf_counter,
                       sleep=time.sleep, admit_in_thread=True)
    with pytest.raises(ValueError):
        srv.run(_reqs([(0.0, 5, 20), (0.0, 10, 20)]))


def test_device_bytes_counts_references_and_the_larger_staging():
    """The library's layout arithmetic (lb_bytes_required), checked block by
    block against what each storage and permeability choice must add: 16-bit
    storage halves the four population buffers of f and h and adds a 32-bit
    reference pair per cell and buffer; a full permeability tensor keeps three
    more rows of K^-1; without K the creation staging loses its six K rows,
    and the initialisation staging (larger then) takes its place."""
    from paper_0912_4230_gb300 import lb
    N = 32 ** 3
    p = W.miscible(32, 32, 32)
    dom = lb.make_domain(p)

    def req(storage, k_rows):
        return lb.lb_bytes_required(dom, lb.make_params(p, storage), k_rows)

    def g(b):   # 256-byte granule
        return -(-b // 256) * 256

    b32, b16 = req("fp32", 3), req("fp16", 3)
    assert b32 - b16 == 2 * (g(19 * N * 4 * 2) - g(19 * N * 2 * 2)) - 2 * g(4 * N)
    assert req("bf16", 3) == b16
    assert req("fp32", 6) - b32 == g(6 * 4 * N) - g(3 * 4 * N)
    create = g(4 * N + 24 * N + N + 64 + 256)
    init = g(4 * N * 5 + 4 * N + N + 256)
    assert create > init
    assert b32 - req("fp32", 0) == g(3 * 4 * N) + create - max(g(4 * N + N + 64 + 256), init)
    assert req("fp64", 3) > b32 > b16
    with pytest.raises(lb.LbError) as e:
        lb.lb_bytes_required(dom, lb.make_params(p, "fp32"), 4)
    assert e.value.code == lb.LB_EINVAL and "k_rows" in lb.lb_last_error(None)
