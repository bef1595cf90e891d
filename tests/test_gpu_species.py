"""Several solute species on the GPU (the fused step for the fluid and
species 0, the species pass for the others) against the FP64 oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0912_4230_gb300 import lb, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_identical_species_are_bit_identical(storage):
    p = W.random_medium(19, 11, 9, seed=31)
    ps = W.with_species(p, tau_D=(p.params["tau_D"],), C_in=(p.params["C_in"],))
    g = lb.Lattice(ps, storage=storage, check_every=1)
    g.step(20)
    C0, t0, h0 = g.species_state(0)
    C1, t1, h1 = g.species_state(1)
    assert np.array_equal(h0, h1) and np.array_equal(C0, C1) and np.array_equal(t0, t1)


def test_passive_species_leave_fluid_and_species_zero_unchanged():
    p = W.random_medium(19, 11, 9, seed=32, visc_law=2)
    rng = np.random.default_rng(5)
    ps = W.with_species(p, tau_D=(1.3, 0.55), C_in=(0.2, 2.0),
                        C0=(rng.uniform(0, 1, p.N), rng.uniform(0, 2, p.N)))
    a = lb.Lattice(p, storage="fp32", check_every=1)
    b = lb.Lattice(ps, storage="fp32", check_every=1)
    a.step(30)
    b.step(30)
    fa, ha = a.populations()
    fb, hb = b.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ha, hb)
    assert np.array_equal(a.reduce(), b.reduce())


@pytest.mark.parametrize("storage", ["fp64", "fp32", "fp16"])
def test_species_against_the_oracle(storage):
    """Solids, walls, full K, solute inlet/outlet: every species' field,
    totals and (FP64/FP32) populations."""
    p = W.random_medium(19, 13, 11, seed=33)
    rng = np.random.default_rng(9)
    ps = W.with_species(p, tau_D=(1.25, 0.6), C_in=(0.3, 1.7),
                        C0=(rng.uniform(0, 1, p.N), np.zeros(p.N)))
    g = lb.Lattice(ps, storage=storage, check_every=1)
    g.step(25)
    o = O.Oracle(ps)
    o.step(25)
    live = p.solid == 0
    tolC = {"fp64": 1.2e-7, "fp32": 1e-5, "fp16": 1e-3}[storage]
    for s in range(3):
        C, tot, h = g.species_state(s)
        rC, rtot, rh = o.species_state(s)
        assert np.abs(C[live] - rC[live]).max() <= tolC
        assert tot[0] == pytest.approx(rtot[0], rel=1e-6 if storage != "fp16" else 1e-4)
        relf = 2e-3 if storage == "fp16" else 1e-4   # FP16: the 1e-3 field bound
        assert tot[1] == pytest.approx(rtot[1], rel=relf, abs=1e-9)
        assert tot[2] == pytest.approx(rtot[2], rel=relf, abs=1e-9)
        if storage != "fp16":
            # FP32: each step rounds every population to 2^-24 of its size;
            # 25 steps accumulate at most ~25 x 2^-24 = 1.5e-6 of max |h|
            scale = max(1.0, float(np.abs(rh[:, live]).max()))
            tolp = 1e-13 if storage == "fp64" else 1.5e-6 * scale
            assert np.abs(h[:, live] - rh[:, live]).max() < tolp


def test_species_medium_full_size_first_steps():
    """128^3, three species, 3 steps, every cell of every species against
    the oracle, in the benchmark's configuration (autotuned launch)."""
    p = W.miscible_species(128, 128, 128, seed=0)
    g = lb.Lattice(p, storage="fp32")
    lb.lb_autotune(g.ctx, 2)
    g.step(3)
    o = O.Oracle(p)
    o.step(3)
    _, u, _, _ = g.fields()
    _, ru, _, _ = o.fields()
    assert np.abs(u - ru).max() <= 1e-5 * np.abs(ru).max()
    for s in range(3):
        assert np.abs(g.species_state(s)[0] - o.species_state(s)[0]).max() <= 1e-5


def test_species_use_the_per_cell_kernel_only():
    p = W.miscible_species(64, 8, 8, seed=1)
    with pytest.raises(lb.LbError) as e:
        lb.Lattice(p, storage="fp32", kernel="staged")
    assert e.value.code == lb.LB_EUNSUPPORTED


def test_species_lattice_in_a_batch_equals_its_own_steps():
    torch = pytest.importorskip("torch")
    s = torch.cuda.Stream()
    probs = [W.miscible(16, 12, 10, seed=1), W.miscible_species(16, 12, 10, seed=2)]
    sep = [lb.Lattice(p, storage="fp32", kernel="cell", check_every=1) for p in probs]
    bat = [lb.Lattice(p, storage="fp32", kernel="cell", check_every=1, stream=s.cuda_stream)
           for p in probs]
    for g in sep:
        g.step(12)
    lb.lb_step_batch([g.ctx for g in bat], 12)
    for a, b in zip(sep, bat):
        fa, ha = a.populations()
        fb, hb = b.populations()
        assert np.array_equal(fa, fb) and np.array_equal(ha, hb)
    for sp in range(3):
        assert np.array_equal(sep[1].species_state(sp)[2], bat[1].species_state(sp)[2])
