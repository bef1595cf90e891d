"""Packed lattice arena bookkeeping (lb_arena_*) on a host region: the
allocator never touches the region's bytes, so its policy is checked here
against a plain Python model of first-fit over an address-ordered free list
with 256-byte blocks and merging of free neighbours."""
import threading

import numpy as np
import pytest

from paper_0912_4230_gb300 import lb

ALIGN = 256


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _region(nbytes):
    buf = np.zeros(nbytes + ALIGN, np.uint8)
    return buf, (buf.ctypes.data + ALIGN - 1) // ALIGN * ALIGN


class Model:
    """First fit, lowest address first; blocks rounded up to 256 bytes."""

    def __init__(self, nbytes):
        self.free = [(0, nbytes // ALIGN * ALIGN)]
        self.live = {}

    def alloc(self, n):
        need = -(-n // ALIGN) * ALIGN
        for i, (off, ln) in enumerate(self.free):
            if ln >= need:
                if ln == need:
                    self.free.pop(i)
                else:
                    self.free[i] = (off + need, ln - need)
                self.live[off] = need
                return off
        return None

    def release(self, off):
        ln = self.live.pop(off)
        self.free.append((off, ln))
        self.free.sort()
        merged = []
        for o, l in self.free:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + l)
            else:
                merged.append((o, l))
        self.free = merged


def test_blocks_are_aligned_rounded_and_merged():
    buf, base = _region(1 << 16)
    a = lb.Arena(1 << 16, base)
    p = [a.alloc(n) for n in (1, 256, 257, 1000)]
    assert [x - base for x in p] == [0, 256, 512, 1024]
    assert a.stats()["used"] == 256 + 256 + 512 + 1024
    a.free(p[1])
    a.free(p[2])        # merges with the freed block before it
    q = a.alloc(700)    # first fit: the merged 768-byte hole
    assert q - base == 256
    for x in (p[0], q, p[3]):
        a.free(x)
    st = a.stats()
    assert st["used"] == 0 and st["blocks"] == 0 and st["largest_free"] == 1 << 16
    assert st["peak"] == 2048
    a.close()


def test_full_arena_returns_null_and_recovers():
    buf, base = _region(4096)
    a = lb.Arena(4096, base)
    ps = [a.alloc(1024) for _ in range(4)]
    assert all(ps) and a.alloc(1) is None
    a.free(ps[2])
    assert a.alloc(1024) == ps[2]
    a.close()


def test_random_sequence_matches_the_model():
    rng = np.random.default_rng(3)
    nbytes = 1 << 22
    buf, base = _region(nbytes)
    a = lb.Arena(nbytes, base)
    m = Model(nbytes)
    held = []
    for _ in range(3000):
        if held and rng.random() < 0.45:
            off = held.pop(int(rng.integers(len(held))))
            a.free(base + off)
            m.release(off)
        else:
            n = int(rng.integers(1, 200_000))
            got = a.alloc(n)
            want = m.alloc(n)
            assert (got is None) == (want is None)
            if want is not None:
                assert got - base == want
                held.append(want)
        st = a.stats()
        assert st["used"] == sum(m.live.values())
        assert st["largest_free"] == max((l for _, l in m.free), default=0)
        assert st["blocks"] == len(m.live)
    a.close()


def test_concurrent_allocations_do_not_overlap():
    nbytes = 1 << 24
    buf, base = _region(nbytes)
    a = lb.Arena(nbytes, base)
    got = [[] for _ in range(8)]

    def worker(k):
        rng = np.random.default_rng(k)
        for _ in range(400):
            n = int(rng.integers(1, 8192))
            p = a.alloc(n)
            if p is not None:
                got[k].append((p - base, -(-n // ALIGN) * ALIGN))
            if got[k] and rng.random() < 0.3:
                off, _ = got[k].pop(0)
                a.free(base + off)

    ts = [threading.Thread(target=worker, args=(k,)) for k in range(8)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    blocks = sorted(b for g in got for b in g)
    for (o1, l1), (o2, _) in zip(blocks, blocks[1:]):
        assert o1 + l1 <= o2
    assert a.stats()["used"] == sum(l for _, l in blocks)
    a.close()


def test_invalid_regions_are_refused():
    buf, base = _region(4096)
    with pytest.raises(lb.LbError) as e:
        lb.Arena(4096, base + 16)      # not 256-byte aligned
    assert e.value.code == lb.LB_EINVAL
    with pytest.raises(lb.LbError):
        lb.Arena(100, base)            # smaller than one block


def test_foreign_pointers_are_ignored_on_release():
    """Releasing a pointer outside the region, or inside it but not at the
    start of a live block, leaves the bookkeeping unchanged."""
    buf, base = _region(1 << 14)
    a = lb.Arena(1 << 14, base)
    p = a.alloc(1000)
    before = a.stats()
    for q in (base - ALIGN, base + (1 << 14), base + (1 << 20), p + ALIGN, 1):
        a.free(q)
        assert a.stats() == before
    a.free(p)
    assert a.stats()["used"] == 0 and a.stats()["largest_free"] == 1 << 14
    a.close()


def test_requests_larger_than_the_region_get_nothing():
    """A request above the region's size fails without touching the free
    list, including sizes so close to 2^64 that rounding them up to a
    256-byte block would wrap around to zero."""
    buf, base = _region(1 << 14)
    a = lb.Arena(1 << 14, base)
    for n in ((1 << 14) + 1, 2 ** 64 - 1, 2 ** 64 - 255, 2 ** 63):
        assert a.alloc(n) is None
    st = a.stats()
    assert st["used"] == 0 and st["blocks"] == 0 and st["largest_free"] == 1 << 14
    p = a.alloc(1 << 14)          # the whole region still fits
    assert p == base and a.alloc(1) is None
    a.free(p)
    a.close()
