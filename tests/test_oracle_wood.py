"""The wood-penetration workload (Section 5.5; reading R25: miscible
displacement of solvent by adhesive pressed in by P_ext, the free surface
left out) — input pins and behaviour pins on the oracle.

Inputs: Eq. wooddensityfunc at the ring ends and its monotone rise for
c < 0, the anisotropy ratios of Eq. Ktensor, a symmetric positive-definite
tensor whose radial axis lies across the rings at the ring angle, periodicity
over the ring width. Behaviour: the solute balance with inlet and outlet
holds step by step, and hardening (Eq. nuall) stops the inflow while it goes
on without it ("the simulation was stopped when the adhesive could not
penetrate further due to hardening").
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0912_4230_gb300 import workloads as W


def test_density_law_end_points_and_rise():
    r = W.wood_density([0.0, 0.5, 1.0 - 1e-12])
    assert r[0] == pytest.approx(310.0)
    assert r[2] == pytest.approx(310.0 * (1.0 + 2 * 0.62 * np.exp(0.2)), rel=1e-9)
    xs = np.linspace(0, 0.999, 200)
    assert np.all(np.diff(W.wood_density(xs)) > 0)


def test_tensor_ratios_and_porosity_range():
    rho = W.wood_density(np.linspace(0, 0.999, 50))
    eps, k = W.wood_tensor(rho)
    assert np.allclose(k[:, 1] / k[:, 0], 51470 / 8.2) and np.allclose(k[:, 2] / k[:, 0], 0.1)
    assert 0.45 < eps.min() < eps.max() < 0.8      # rho_max = 1500 kg/m^3 (reading)
    assert np.all(np.diff(k[:, 0]) < 0)               # denser latewood is less permeable


@pytest.mark.parametrize("angle", [45.0, 0.0])
def test_tensor_orientation_and_ring_periodicity(angle):
    p = W.wood(nx=60, ny=40, wood_depth=30, angle=angle)
    K = p.K6.reshape(-1, 6).astype(np.float64)
    y = np.arange(p.N) // p.nx % p.ny
    wood = y < 30
    th = np.deg2rad(angle)
    r_dir = np.array([np.cos(th), np.sin(th), 0.0])
    for n in np.flatnonzero(wood)[::97]:
        M = np.array([[K[n, 0], K[n, 3], K[n, 5]], [K[n, 3], K[n, 1], K[n, 4]],
                      [K[n, 5], K[n, 4], K[n, 2]]])
        w, v = np.linalg.eigh(M)
        assert w.min() > 0
        # the in-plane principal axis with the larger permeability is radial
        inplane = [i for i in range(3) if abs(v[2, i]) < 1e-6]
        big = max(inplane, key=lambda i: w[i])
        assert abs(abs(v[:, big] @ r_dir) - 1.0) < 1e-5
        assert w[big] / min(w[i] for i in inplane) == pytest.approx(10.0, rel=1e-5)
    if angle == 0.0:   # rings across x: porosity periodic with the ring width
        eps = p.eps.reshape(p.ny, p.nx)
        assert np.allclose(eps[:30, :30], eps[:30, 30:60])


def test_solute_balance_through_the_sample():
    p = W.wood(nx=30, ny=30, wood_depth=20, delta=10.0)
    o = O.Oracle(p)
    prev = o.reduce()
    for _ in range(40):
        o.step(1)
        cur = o.reduce()
        d = cur[1] - prev[1]
        flux = (cur[2] - prev[2]) - (cur[3] - prev[3])
        assert d == pytest.approx(flux, abs=1e-12 * max(1.0, cur[1]))
        prev = cur


def test_hardening_stops_the_flow():
    """a e^(alpha t) passes 1 near t = 2500 (alpha = 8e-3): the inflow stops
    (the largest velocity falls a hundredfold) while it goes on unchanged
    without hardening. The law grows without bound: past nu ~ 1e2 (tau ~ 3e2)
    the forcing scheme with the implicit drag breaks down, so the check stays
    at t <= 3200 (the paper stops its run when the adhesive no longer moves)."""
    base = dict(nx=30, ny=40, wood_depth=30, delta=10.0, K_scale=2e-2)
    hard, soft = W.wood(alpha=8e-3, **base), W.wood(alpha=0.0, **base)
    oh, os_ = O.Oracle(hard), O.Oracle(soft)
    umax = {}
    for t in (2000, 3200):
        oh.step(t - oh.t)
        os_.step(t - os_.t)
        umax[t] = (np.abs(oh.fields()[1]).max(), np.abs(os_.fields()[1]).max())
    assert umax[3200][0] < 1e-2 * umax[2000][0]
    assert umax[3200][1] == pytest.approx(umax[2000][1], rel=0.05)
    nu = oh.fields()[3]
    assert nu.max() > 100 * 0.15
