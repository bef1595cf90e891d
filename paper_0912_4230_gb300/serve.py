"""Serving loop for penetration solves: continuous batching under an HBM budget.

Requests (a porous medium, a lattice size and a number of steps) arrive over
time. A request is admitted as soon as it has arrived and its device memory
fits the budget next to the lattices already resident; admitted lattices stay
on the device and are advanced together, ``chunk`` steps at a time, by one
batched launch per step (``lb_step_batch``). Between chunks finished requests
export their fields and release their memory, and newly arrived requests
join, so work that arrives while others run overlaps with them on the GPU.
Each lattice is computed independently by the same per-cell arithmetic, so a
result does not depend on what else is in the batch.

The stepping backend is pluggable: :class:`LibraryBackend` drives the CUDA
library; tests of the host-side logic use a fake backend on the CPU.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time
from typing import Callable, List, Optional

import numpy as np



def device_bytes(prob, storage: str = "fp32") -> int:
    """Device memory one lattice of this problem takes, as the library
    allocates it (lb_bytes_required: the library's own allocation layout,
    each block in the packed arena's 256-byte granules, the larger of the
    creation and initialisation staging, and the lattice's share of a batch
    work list). A permeability field keeps 6 rows of K^-1 when any cell has
    an off-diagonal entry, else 3."""
    from . import lb
    kr = 0
    if prob.K6 is not None:
        kr = 6 if np.any(np.asarray(prob.K6).reshape(-1, 6)[:, 3:] != 0) else 3
    return lb.lb_bytes_required(lb.make_domain(prob), lb.make_params(prob, storage), kr,
                                prob.f_scale is not None)


@dataclasses.dataclass
class Request:
    id: int
    arrival: float               # seconds after the start of the run
    steps: int
    problem: object              # workloads.Problem
    bytes: int = 0
    admitted: Optional[float] = None
    done: Optional[float] = None
    remaining: int = 0
    handle: object = None
    result: object = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival

    @property
    def wait(self) -> float:
        return self.admitted - self.arrival


class LibraryBackend:
    """Resident lattices on the GPU through the C ABI.

    With torch streams given, a new lattice is created and initialised on
    ``admit_stream`` while earlier lattices step on ``step_stream``; the step
    stream waits for the admission work before the lattice's first step."""

    def __init__(self, storage: str = "fp32", stream=None, keep_fields: bool = True,
                 batched: bool = True, admit_stream=None, step_stream=None):
        from . import lb
        self.lb = lb
        self.storage = storage
        self.stream = stream
        self.keep_fields = keep_fields
        self.batched = batched
        self.admit_stream = admit_stream
        self.step_stream = step_stream

    def bytes(self, prob) -> int:
        return device_bytes(prob, self.storage)

    def admit(self, prob):
        """Create and initialise a lattice (may run on a background thread).
        Raises MemoryError when its device memory does not fit (for example
        in a packed arena that is full or fragmented)."""
        try:
            return self._admit(prob)
        except self.lb.LbError as e:
            if e.code == self.lb.LB_ENOMEM:
                raise MemoryError(str(e)) from None
            raise

    def _admit(self, prob):
        if self.admit_stream is None:
            return self.lb.Lattice(prob, storage=self.storage, kernel="cell", stream=self.stream)
        import torch
        self.lb.lb_set_stream(None, self.admit_stream.cuda_stream)
        h = self.lb.Lattice(prob, storage=self.storage, kernel="cell",
                            stream=self.admit_stream.cuda_stream)
        h.ready_event = torch.cuda.Event()
        h.ready_event.record(self.admit_stream)
        return h

    def activate(self, handle):
        """Before a lattice's first step (on the stepping thread, outside any
        graph capture): the step stream waits for its initialisation."""
        ev = getattr(handle, "ready_event", None)
        if ev is not None:
            self.step_stream.wait_event(ev)
            self.lb.lb_set_stream(handle.ctx, self.step_stream.cuda_stream)
            handle.ready_event = None

    def step(self, handles, n: int):
        """Enqueue n steps of every handle; returns an event recorded after
        them on the step stream (None without torch streams)."""
        if self.batched:
            self.lb.lb_step_batch([h.ctx for h in handles], n)
        else:
            for h in handles:   # the plain per-lattice path: one launch per lattice and step
                h.step(n)
        if self.step_stream is None:
            return None
        import torch
        ev = torch.cuda.Event()
        ev.record(self.step_stream)
        return ev

    def finish(self, handle, after=None):
        """Export (keep_fields) and release a finished lattice. With `after`
        (the event of the chunk that finished it) the lattice moves to a
        stream of its own that waits for that event, so the export and the
        release wait for its own last step only, not for the chunks enqueued
        for the other lattices since."""
        if after is not None:
            import torch
            if not hasattr(self, "_finish_stream"):
                self._finish_stream = torch.cuda.Stream()
            self._finish_stream.wait_event(after)
            self.lb.lb_set_stream(handle.ctx, self._finish_stream.cuda_stream)
        out = None
        if self.keep_fields:
            rho, u, C, nu = handle.fields()
            out = dict(rho=rho, u=u, C=C, nu=nu, totals=handle.reduce())
        else:
            handle.sync()
        handle.close()
        return out


class Server:
    """Admission by HBM budget, continuous batching in chunks of steps."""

    def __init__(self, backend, budget_bytes: int, chunk: int = 200,
                 clock: Callable[[], float] = time.perf_counter, sleep=time.sleep,
                 max_resident: Optional[int] = None, fill_cells: Optional[int] = None,
                 admit_in_thread: bool = False):
        """fill_cells: step, each chunk, only the oldest resident requests
        whose lattices together reach this many cells (enough to fill the
        GPU); the younger ones stay resident and join as the older finish.
        None steps every resident request together.
        admit_in_thread: create lattices on a background thread while the
        resident ones step (the library calls release the GIL)."""
        self.backend = backend
        self.budget = int(budget_bytes)
        self.chunk = int(chunk)
        self.max_resident = max_resident
        self.fill_cells = fill_cells
        self.admit_in_thread = admit_in_thread
        self.clock = clock
        self.sleep = sleep
        self.log: List[dict] = []

    def _finish(self, finishing, finished, lock, t0):
        for r, ev in finishing:
            r.result = (self.backend.finish(r.handle, ev) if ev is not None
                        else self.backend.finish(r.handle))
            r.handle = None
            r.done = self.clock() - t0
            with lock:
                self._used -= r.bytes
                self._released += 1
                lock.notify_all()
            finished.append(r)
        finishing.clear()

    def run(self, requests: List[Request]) -> dict:
        pending = sorted(requests, key=lambda r: (r.arrival, r.id))
        for r in pending:
            r.bytes = self.backend.bytes(r.problem)
            r.remaining = r.steps
            if r.bytes > self.budget:
                raise ValueError(f"request {r.id} needs {r.bytes} bytes, above the whole budget")
        active: List[Request] = []
        finished: List[Request] = []
        finishing: List[tuple] = []   # (request, event of the chunk that finished it)
        inflight = collections.deque()
        self._used = 0
        self._released = 0       # requests finished so far (wakes a waiting admission)
        self._admit_error = None
        t0 = self.clock()
        lups = 0
        lock = threading.Condition()
        ready: List[Request] = []
        admitter = None
        if self.admit_in_thread:
            def admit_loop():
                while pending:
                    r = pending[0]
                    wait = r.arrival - (self.clock() - t0)
                    if wait > 0:
                        self.sleep(wait)
                    with lock:
                        while (self._used + r.bytes > self.budget or
                               (self.max_resident is not None and
                                len(active) + len(ready) >= self.max_resident)):
                            lock.wait(0.01)
                        self._used += r.bytes
                    while True:
                        try:
                            r.handle = self.backend.admit(r.problem)
                            break
                        except MemoryError as e:
                            # device memory is short of the estimate (a full or
                            # fragmented arena): wait for a request to finish
                            with lock:
                                if not active and not ready:
                                    self._used -= r.bytes
                                    self._admit_error = e
                                    lock.notify_all()
                                    return
                                seen = self._released
                                while self._released == seen:
                                    lock.wait(0.01)
                    r.admitted = self.clock() - t0
                    with lock:
                        pending.pop(0)
                        ready.append(r)
                        lock.notify_all()
            def admit_guarded():
                # any failure of the admission thread ends the run with that
                # error (the stepping loop checks _admit_error each pass)
                try:
                    admit_loop()
                except BaseException as e:  # noqa: BLE001
                    with lock:
                        self._admit_error = e
                        lock.notify_all()

            admitter = threading.Thread(target=admit_guarded, daemon=True)
            admitter.start()
        while True:
            now = self.clock() - t0
            if admitter is not None:
                with lock:
                    if self._admit_error is not None:
                        raise self._admit_error
                    for r in ready:
                        if hasattr(self.backend, "activate"):
                            self.backend.activate(r.handle)
                    active.extend(ready)
                    ready.clear()
                    if not active:
                        if not pending and not ready:
                            break
                        lock.wait(0.005)
                        continue
            else:
                if not pending and not active:
                    break
                # admit, in arrival order, every arrived request that fits
                while (pending and pending[0].arrival <= now
                       and self._used + pending[0].bytes <= self.budget
                       and (self.max_resident is None or len(active) < self.max_resident)):
                    try:
                        handle = self.backend.admit(pending[0].problem)
                    except MemoryError:
                        if not active:
                            raise      # nothing resident will free memory
                        break          # retry after the next chunk
                    r = pending.pop(0)
                    r.handle = handle
                    if hasattr(self.backend, "activate"):
                        self.backend.activate(r.handle)
                    r.admitted = self.clock() - t0
                    self._used += r.bytes
                    active.append(r)
                if not active:
                    # nothing resident: wait for the next arrival
                    self.sleep(max(0.0, pending[0].arrival - now))
                    continue
            stepping = active
            if self.fill_cells is not None:
                stepping, cells = [], 0
                for r in active:          # arrival order
                    stepping.append(r)
                    cells += r.problem.N
                    if cells >= self.fill_cells:
                        break
            n = min(self.chunk, min(r.remaining for r in stepping))
            ev = self.backend.step([r.handle for r in stepping], n)
            if ev is not None:
                # at most two chunks queued ahead of the GPU, so that requests
                # admitted meanwhile join soon
                inflight.append(ev)
                while len(inflight) > 2:
                    inflight.popleft().synchronize()
            for r in stepping:
                r.remaining -= n
                lups += n * r.problem.N
            # requests finished by an earlier chunk are exported and released
            # now, after this chunk is enqueued, so the GPU has work while
            # the host waits for them
            self._finish(finishing, finished, lock, t0)
            still = []
            for r in active:
                if r.remaining == 0:
                    finishing.append((r, ev))
                else:
                    still.append(r)
            self.log.append(dict(t=self.clock() - t0, resident=len(active), stepped=len(stepping),
                                 stepped_cells=sum(r.problem.N for r in stepping),
                                 steps=n, used=self._used))
            with lock:
                active[:] = still
            if not still:
                self._finish(finishing, finished, lock, t0)
        if admitter is not None:
            admitter.join()
        wall = self.clock() - t0
        lat = np.array([r.latency for r in finished])
        wait = np.array([r.wait for r in finished])
        return dict(
            requests=len(finished), wall_s=wall, lups=lups, mlups=lups / wall / 1e6 if wall else 0.0,
            p50_s=float(np.percentile(lat, 50)), p99_s=float(np.percentile(lat, 99)),
            wait_p50_s=float(np.percentile(wait, 50)), wait_p99_s=float(np.percentile(wait, 99)),
            max_resident=max((e["resident"] for e in self.log), default=0),
        )


def make_requests(stream, storage="fp32", steps_scale: float = 1.0) -> List[Request]:
    """Requests of a serving workload (workloads.requests): the miscible medium
    at each request's size, seeded by its id; steps scaled by steps_scale."""
    from . import workloads as W
    out = []
    for q in stream:
        p = W.request_problem(q, storage=storage)
        steps = max(1, int(round(q["steps"] * steps_scale)))
        out.append(Request(id=q["id"], arrival=q["arrival"], steps=steps, problem=p))
    return out
