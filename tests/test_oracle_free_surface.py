"""Pins of the oracle's free-surface and surface-tension parts (CPU only):
exact liquid-mass conservation (Section 3, Eqs. eq:massmacro to
eq:deltamass; the paper reports < 1 % error, Section 5.3), smoothing of a
square liquid patch (Section 5.4) and Laplace's law for static drops."""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_0912_4230_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_square_patch_mass_conserved_and_rounded():
    """Section 5.4: a square liquid patch (A = 1e-3, tau = 0.7) rounds off
    under surface tension; the liquid mass is conserved exactly (P10)."""
    n, R = 64, 10
    p = W.thin_drop(n, R=R, A=1e-3, shape="square")
    o = O.Oracle(p)
    m0 = o.reduce()[0]

    def extents():
        t, m = o.free_surface_state()
        live = (m.reshape(n, n) > 0.5)
        y, x = np.nonzero(live)
        c = (n - 1) / 2
        ax = max(np.abs(x - c).max(), np.abs(y - c).max())
        dg = max(np.abs((x - c) + (y - c)).max(), np.abs((x - c) - (y - c)).max()) / np.sqrt(2)
        return dg / ax

    r0 = extents()
    o.step(2000)
    r1 = extents()
    assert o.reduce()[0] == pytest.approx(m0, rel=1e-12)
    assert r0 > 1.35          # a square: diagonal reach ~ sqrt(2) x axis reach
    assert r1 < 1.15          # rounded
    t, _ = o.free_surface_state()
    assert set(np.unique(t)) <= {W.LIQUID, W.INTERFACE, W.EMPTY}


def test_falling_drop_mass_conserved():
    """Section 5.3 analogue: a drop falls onto a solid wall; the total liquid
    mass stays constant to rounding, far inside the paper's 1 % bound (P10)."""
    p = W.drop(nx=24, ny=24, nz=28, R=5.0, gap=6.0, steps=500, seed=3)
    o = O.Oracle(p)
    m0 = o.reduce()[0]
    z0 = None
    for _ in range(5):
        o.step(100)
        assert abs(o.reduce()[0] / m0 - 1) < 1e-12
        t, m = o.free_surface_state()
        zc = (np.arange(p.N) // (p.nx * p.ny) * m).sum() / m.sum()
        z0 = zc if z0 is None else z0
    assert abs(o.reduce()[0] / m0 - 1) < GOLD["falling_drop"]["max_relative_mass_error"]
    assert zc < z0            # the drop moved down
    rho, u, _, _ = o.fields()
    t, _ = o.free_surface_state()
    assert np.all(rho[(t != W.EMPTY) & (p.solid == 0)] > 0.9)
    assert np.all(rho[t == W.EMPTY] == 0)


def test_laplace_law():
    """Static 2D drops: the pressure jump (rho_in - rho_gas)/3 with gas
    density 1 scales as 1/R (Laplace's law in 2D), with zero intercept (P9).
    The surface tension sigma itself has no printed value to compare to."""
    Rs = np.array([8.0, 12.0, 16.0, 24.0])
    dps = []
    for R in Rs:
        n = int(2 * R + 24)
        p = W.thin_drop(n, R=R, A=1e-3, shape="disc")
        o = O.Oracle(p)
        o.step(1000)
        rho, _, _, _ = o.fields()
        c = (n - 1) / 2
        y, x = np.mgrid[0:n, 0:n]
        inner = (((x - c) ** 2 + (y - c) ** 2) <= (R / 2) ** 2).ravel()
        dps.append((rho[inner].mean() - 1.0) / 3.0)
    dps = np.array(dps)
    assert np.all(dps > 0)
    sigma = dps * Rs
    assert sigma.max() / sigma.min() < 1.06
    A = np.vstack([1 / Rs, np.ones_like(Rs)]).T
    (slope, icpt), *_ = np.linalg.lstsq(A, dps, rcond=None)
    assert abs(icpt) < 0.05 * dps.max()
    pred = A @ np.array([slope, icpt])
    r2 = 1 - ((dps - pred) ** 2).sum() / ((dps - dps.mean()) ** 2).sum()
    assert r2 > 0.99
