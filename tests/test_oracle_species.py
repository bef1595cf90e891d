"""Oracle pins for several solute species (reading R24: the paper keeps the
solute on its own lattice "to simplify a later extension to various
species"; each species has its own tau_D and inlet concentration, all share
V', species 0's concentration sets the viscosity).

* a species identical to species 0 evolves bit-identically to it;
* passive species change nothing of the fluid or of species 0 (bit-exact
  against the single-species run);
* each species' Gaussian pulse spreads with its own D = (tau_D - 1/2)/3;
* each species' solute balance with inlet and outlet faces holds step by
  step.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0912_4230_gb300 import workloads as W


def test_identical_species_evolve_identically():
    p = W.random_medium(9, 7, 6, seed=11)
    ps = W.with_species(p, tau_D=(p.params["tau_D"],) * 2, C_in=(p.params["C_in"],) * 2)
    o = O.Oracle(ps)
    o.step(40)
    C0, t0, h0 = o.species_state(0)
    for s in (1, 2):
        C, t, h = o.species_state(s)
        assert np.array_equal(h, h0) and np.array_equal(C, C0) and np.array_equal(t, t0)


def test_passive_species_leave_fluid_and_species_zero_unchanged():
    p = W.random_medium(9, 7, 6, seed=12, visc_law=2)
    rng = np.random.default_rng(3)
    ps = W.with_species(p, tau_D=(1.3, 0.55), C_in=(0.2, 2.0),
                        C0=(rng.uniform(0, 1, p.N), rng.uniform(0, 2, p.N)))
    a, b = O.Oracle(p), O.Oracle(ps)
    a.step(35)
    b.step(35)
    fa, ha = a.populations()
    fb, hb = b.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ha, hb)
    for x, y in zip(a.fields(), b.fields()):
        assert np.array_equal(x, y)
    assert np.array_equal(a.reduce(), b.reduce())


def test_each_species_diffuses_with_its_own_coefficient():
    taus = (0.8, 1.4, 0.6)
    p = W.with_species(W.gaussian_pulse(128, sigma0=4.0, tau_D=taus[0]), tau_D=taus[1:])
    o = O.Oracle(p)
    x = np.arange(128, dtype=float)
    var = {}
    for t in (20, 120):
        o.step(t - o.t)
        for s in range(3):
            C = o.species_state(s)[0]
            m = C.sum()
            xb = (C * x).sum() / m
            var[(s, t)] = (C * (x - xb) ** 2).sum() / m
    for s, tau in enumerate(taus):
        D = (tau - 0.5) / 3.0
        assert (var[(s, 120)] - var[(s, 20)]) / 100 == pytest.approx(2 * D, rel=1e-4)


def test_each_species_porosity_gradient_correction():
    """Eq. diffusionporous with V' = 0 and uniform C is stationary only with
    each species' own D in V* = V' + D grad(eps)/eps: species of different
    tau_D all stay uniform (to the second-order error of the single-species
    pin), and the deviation converges at second order for each."""
    dev = {}
    for nx in (32, 64):
        p = W.with_species(W.eps_bands(nx, 2, 2, C=0.5), tau_D=(1.4, 0.6), C0=())
        o = O.Oracle(p)
        o.step(2000)
        for s in range(3):
            dev[(s, nx)] = np.abs(o.species_state(s)[0] - 0.5).max()
    for s in range(3):
        assert dev[(s, 64)] < 1e-3
        assert 3.0 < dev[(s, 32)] / dev[(s, 64)] < 6.5


def test_each_species_balances_inlet_and_outlet_fluxes():
    p = W.with_species(W.random_medium(8, 7, 6, seed=6), tau_D=(1.1, 0.65), C_in=(0.4, 3.0))
    o = O.Oracle(p)
    prev = [o.species_state(s)[1] for s in range(3)]
    for _ in range(30):
        o.step(1)
        for s in range(3):
            cur = o.species_state(s)[1]
            d = cur[0] - prev[s][0]
            flux = (cur[1] - prev[s][1]) - (cur[2] - prev[s][2])
            assert d == pytest.approx(flux, abs=1e-12 * max(1.0, cur[0]))
            prev[s] = cur
    # species 2 enters at C = 3, above every initial value: its inlet injects
    assert o.species_state(2)[1][1] > 0 and o.species_state(1)[1][1] != 0


def test_species_count_is_validated():
    p = W.random_medium(5, 4, 4, seed=1)
    bad = p.replace(params=dict(p.params, species=9))
    with pytest.raises(ValueError):
        O.Oracle(bad)
    bad = W.with_species(p, tau_D=(0.5,))   # tau_D must exceed 1/2
    with pytest.raises(ValueError):
        O.Oracle(bad)
