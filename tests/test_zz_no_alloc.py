"""lb_totals_noalloc: the allocation-free variant of the totals behind
lb_reduce, for callers that cannot allocate device memory where they need
the totals. Checked through the C ABI against an FP64 host sum of the same
device arrays and against lb_reduce on the same state, twice in a row (the
second call reuses the library's fixed scratch array).
Collected last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

from paper_0912_4230_gb300 import lb, workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_totals_match_lb_reduce_twice():
    torch = pytest.importorskip("torch")
    import __graft_entry__
    __graft_entry__.build()
    p = W.random_medium(23, 17, 13, seed=12, solid_frac=0.15)
    g = lb.Lattice(p, storage="fp32")
    g.step(7)
    mass, solute, _, _ = g.reduce()
    f, h = g.populations()
    w = _weights()
    # the library's FP32 storage form: f_q - w_q (an exact round trip of the state)
    f32 = (f - w[:, None]).astype(np.float32)
    h32 = h.astype(np.float32)
    dev = torch.device("cuda:0")
    fd = torch.from_numpy(f32.ravel()).to(dev)
    hd = torch.from_numpy(h32.ravel()).to(dev)
    sd = torch.from_numpy(np.ascontiguousarray(p.solid, np.uint8)).to(dev)
    stream = torch.cuda.current_stream().cuda_stream
    # lb_reduce sums each cell's 19 stored values in FP32 before its FP64
    # sum over cells: a sequential FP32 sum of 19 terms is off by at most
    # 18 * 2^-24 * sum_q |term_q| per cell, this path widens every value
    live = p.solid == 0
    bound_m = 18 * 2.0 ** -24 * np.abs(f32[:, live]).sum()
    bound_s = 18 * 2.0 ** -24 * np.abs(h32[:, live]).sum()
    # an independent check: the FP64 sum on the host of the same device
    # arrays, copied back, every value widened as the call widens it. Both
    # are FP64 sums of the same ~2e5 terms in different orders (tree sums of
    # O(log n) depth): they agree to ~1e-14 of the sum of magnitudes.
    fh = fd.cpu().numpy().reshape(19, p.N).astype(np.float64) + w[:, None]
    hh = hd.cpu().numpy().reshape(19, p.N).astype(np.float64)
    host_m, host_s = fh[:, live].sum(), hh[:, live].sum()
    for _ in range(2):
        out = np.zeros(2)
        lb.lb_totals_noalloc(fd, hd, sd, p.N, out, stream)
        assert abs(out[0] - host_m) <= 1e-13 * np.abs(fh[:, live]).sum()
        assert abs(out[1] - host_s) <= 1e-13 * np.abs(hh[:, live]).sum()
        assert abs(out[0] - mass) <= bound_m + 1e-13 * abs(mass)
        assert abs(out[1] - solute) <= bound_s + 1e-13 * abs(solute)
    # device output buffer, solid mask omitted (all cells counted)
    outd = torch.zeros(2, dtype=torch.float64, device=dev)
    lb.lb_totals_noalloc(fd, hd, None, p.N, outd, stream)
    assert abs(outd[0].item() - (mass + f[:, ~live].sum())) <= bound_m + 1e-13 * abs(mass)
    g.close()


def test_noalloc_rejects_sizes_beyond_its_limit():
    pytest.importorskip("torch")
    with pytest.raises(lb.LbError) as e:
        lb.lb_totals_noalloc(np.zeros(19, np.float32), None, None, (1 << 24) + 1, np.zeros(2))
    assert e.value.code == lb.LB_EINVAL
    # the reason reaches the caller (lb_last_error(NULL) on this thread)
    assert "16777216" in str(e.value) and "16777216" in lb.lb_last_error(None)


def _weights():
    """D3Q19 weights in the library's direction order: rest 1/3, then per
    plane four diagonals (1/36) and two axis directions (1/18)."""
    return np.array([1 / 3] + ([1 / 36] * 4 + [1 / 18] * 2) * 3)
