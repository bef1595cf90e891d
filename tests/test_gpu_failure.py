"""Failure detection on the GPU without a fault: a bounded wait that runs out
is reported as LB_ETIMEOUT and leaves the context usable; a non-finite state
is reported as LB_ENONFINITE."""
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_0912_4230_gb300 import lb, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def test_bounded_wait_gives_up_and_context_recovers():
    p = W.miscible(24, 20, 18, seed=7)
    g = lb.Lattice(p, storage="fp32", check_every=1)
    g.step(5)
    t0 = time.perf_counter()
    with pytest.raises(lb.LbError) as e:
        lb.lb_debug_wait_timeout(g.ctx, 50_000_000)   # 50 ms on a barrier nothing completes
    dt = time.perf_counter() - t0
    assert e.value.code == lb.LB_ETIMEOUT
    assert 0.04 < dt < 5.0
    # the status stays set until re-initialisation; afterwards the context steps normally
    with pytest.raises(lb.LbError) as e2:
        g.sync()
    assert e2.value.code == lb.LB_ETIMEOUT
    g.init()
    g.step(40)
    o = O.Oracle(p)
    o.step(40)
    _, u, C, _ = g.fields()
    _, ru, rC, _ = o.fields()
    assert np.abs(u - ru).max() <= 1e-5 * np.abs(ru).max()
    assert np.abs(C - rC).max() <= 1e-5


def test_wait_limit_is_validated():
    p = W.miscible(16, 8, 8, seed=1)
    g = lb.Lattice(p, storage="fp32")
    for bad in (0, -1, 3_000_000_000):
        with pytest.raises(lb.LbError) as e:
            lb.lb_debug_wait_timeout(g.ctx, bad)
        assert e.value.code == lb.LB_EINVAL
