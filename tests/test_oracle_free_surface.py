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


def _neighbours(p):
    """D3Q19 neighbours of every cell (N x 18 indices, -1 across a wall face
    or onto a solid cell), from the box and its face kinds alone."""
    vel = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    vel += [(a, b, 0) for a in (1, -1) for b in (1, -1)]
    vel += [(a, 0, b) for a in (1, -1) for b in (1, -1)]
    vel += [(0, a, b) for a in (1, -1) for b in (1, -1)]
    n = np.arange(p.N)
    x, y, z = n % p.nx, (n // p.nx) % p.ny, n // (p.nx * p.ny)
    out = np.full((p.N, 18), -1, np.int64)
    dims = (p.nx, p.ny, p.nz)
    for k, c in enumerate(vel):
        ok = np.ones(p.N, bool)
        coords = []
        for axis, (v, d) in enumerate(zip((x, y, z), dims)):
            w = v + c[axis]
            if p.bc[axis][0] == W.PERIODIC:
                w = w % d
            else:
                ok &= (w >= 0) & (w < d)
                w = np.clip(w, 0, d - 1)
            coords.append(w)
        m = coords[0] + p.nx * (coords[1] + p.ny * coords[2])
        ok &= p.solid[m] == 0
        out[:, k] = np.where(ok, m, -1)
    return out


def _check_layers(p, o, nb, prev):
    """The interface layer separates liquid from gas (no liquid cell next to
    an empty one) and empty cells hold no mass; a cell liquid before and
    after the step keeps m - rho (its mass exchange equals its density
    change: its links reach no empty cell, and bounce-back links cancel)."""
    t, m = o.free_surface_state()
    rho = o.fields()[0]
    live = p.solid == 0
    liquid = live & (t == W.LIQUID)
    nbt = np.where(nb >= 0, t[np.maximum(nb, 0)], W.LIQUID)
    assert not np.any(liquid[:, None] & (nbt == W.EMPTY)), "liquid cell next to an empty cell"
    assert np.all(m[live & (t == W.EMPTY)] == 0.0)
    d = m - rho
    if prev is not None:
        t0, d0 = prev
        both = liquid & (t0 == W.LIQUID)
        assert np.abs(d[both] - d0[both]).max(initial=0.0) < 1e-12
    return (t, d), int(np.sum(live & (t == W.INTERFACE)))


def test_conversions_keep_the_interface_layer_closed():
    """Reading R18 (conversion of filled and emptied cells): while the drop
    falls, fills and empties, every step leaves an interface layer between
    liquid and gas, no mass in the gas, and m - rho unchanged in cells that
    stay liquid. A filled cell whose empty neighbours were not made
    interface, or an emptied cell whose liquid neighbours stayed liquid,
    breaks the first property; excess mass left in an emptied cell the
    second; an exchange term dropped between liquid and interface cells the
    third."""
    p = W.drop(nx=24, ny=24, nz=28, R=5.0, gap=6.0, steps=400, seed=3)
    o = O.Oracle(p)
    nb = _neighbours(p)
    o.step(1)   # the exported density of lb_init is rho0, not that of the perturbed populations
    prev, n0 = _check_layers(p, o, nb, None)
    n_if = [n0]
    changed = 0
    for _ in range(200):
        o.step(1)
        t_prev = prev[0]
        prev, k = _check_layers(p, o, nb, prev)
        n_if.append(k)
        changed += int(np.sum(prev[0] != t_prev))
    assert changed > 50            # cells did fill and empty along the way
    assert min(n_if) > 0


def test_contact_angle_sweep_is_reproduced_and_ordered():
    """The stored sweep of the wetting reading (R16, written by
    tests/golden/contact_angle.py from the oracle): the angle falls as the
    wall looks more like liquid, a wall with wall_rho = 1 wets at about 90
    degrees, and the drop workload's 0.6 case relaxed from a half disc is
    reproduced."""
    import importlib.util
    here = os.path.join(os.path.dirname(__file__), "golden")
    sweep = json.load(open(os.path.join(here, "contact_angle.json")))
    for angles in sweep["angles_deg"].values():
        assert all(a >= b for a, b in zip(angles, angles[1:]))
    k = sweep["wall_rho"].index(1.0)
    assert all(abs(v[k] - 90.0) < 10.0 for v in sweep["angles_deg"].values())
    spec = importlib.util.spec_from_file_location("contact_angle", os.path.join(here, "contact_angle.py"))
    ca = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(ca)
    i = sweep["wall_rho"].index(0.6)
    assert ca.run(0.6, -7.0) == pytest.approx(sweep["angles_deg"]["from_90deg"][i], abs=0.05)


def test_falling_drop_follows_free_fall():
    """Section 5.3's falling drop: with the gas carrying no momentum, a
    drop under the body force G falls freely until it meets the wall; its
    centre of mass moves by G t^2 / 2 (within 1.5 %: the interface cells'
    fill and the drop's small deformation), and the liquid mass stays
    constant. At the paper's G = 1e-6 this is the printed impact after about
    10 600 steps for a drop whose lowest point starts 56 cells above the
    wall (sqrt(2 * 56 / 1e-6) = 10 583)."""
    G = 1e-5
    p = W.drop(nx=48, ny=1, nz=80, R=8.0, gap=30.0, u_drop=0.0, perturb=0.0)
    p = p.replace(params=dict(p.params, G=(0.0, 0.0, -G), A=0.0))
    o = O.Oracle(p)
    z = np.arange(p.N) // (p.nx * p.ny)

    def zcm():
        _, m = o.free_surface_state()
        return (m * z).sum() / m.sum(), m.sum()

    z0, m0 = zcm()
    for k in range(1, 11):              # to t = 2000, before the impact at sqrt(2 * 30 / G) = 2449
        o.step(200)
        zc, m = zcm()
        t = 200 * k
        assert (z0 - zc) == pytest.approx(0.5 * G * t * t, rel=0.015)
        assert m == pytest.approx(m0, rel=1e-12)
