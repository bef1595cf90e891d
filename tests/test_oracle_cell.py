"""Pins of the oracle's single-cell pieces against what the paper and the
mathematics fix (CPU only).

Each test checks a property that a dropped term, a wrong sign, a wrong index
or a transposed operand in the oracle would break: moment identities of the
equilibria and forcing terms (Section 2, Eqs. equilc1, equilc2, coeffforce1,
equild), the continuum surface-tension tensor (Eq. eqsurftens), the implicit
velocity correction (Eqs. forcement, expandV) and the viscosity laws.
"""
import itertools
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_0912_4230_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _c():
    c, w, opp = O.velocity_set()
    return c.astype(float), w, opp


def test_velocity_set_is_d3q19():
    c, w, opp = O.velocity_set()
    # brute force: every integer vector in {-1,0,1}^3 of squared length <= 2
    brute = {v for v in itertools.product((-1, 0, 1), repeat=3) if sum(x * x for x in v) <= 2}
    assert len(brute) == 19
    assert {tuple(v) for v in c.tolist()} == brute
    g = GOLD["d3q19_weights"]
    for q in range(19):
        s = int((c[q] ** 2).sum())
        expect = {0: g["w0"], 1: g["w_axis"], 2: g["w_diagonal"]}[s]
        assert w[q] == pytest.approx(expect, abs=1e-15)
    for q in range(19):
        assert (c[opp[q]] == -c[q]).all()


def test_velocity_set_plane_reading():
    """Reading of the missing figure: q = 1 + 6p + (i-1); orientation i = 1..4
    are diagonals and 5, 6 the first axis of plane p (x-y, y-z, z-x)."""
    c, _, _ = O.velocity_set()
    planes = [(0, 1), (1, 2), (2, 0)]
    for p, (a0, a1) in enumerate(planes):
        other = 3 - a0 - a1
        for i in range(1, 7):
            v = c[1 + 6 * p + i - 1]
            assert v[other] == 0
            if i <= 4:
                assert abs(v[a0]) == 1 and abs(v[a1]) == 1
            else:
                assert v[a0] == (1 if i == 5 else -1) and v[a1] == 0
        # diagonals run counter-clockwise in the (a0, a1) plane
        d = [c[1 + 6 * p + k][[a0, a1]] for k in range(4)]
        for k in range(4):
            cross = d[k][0] * d[(k + 1) % 4][1] - d[k][1] * d[(k + 1) % 4][0]
            assert cross > 0


def test_velocity_set_isotropy():
    c, w, _ = _c()
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.allclose(w @ c, 0.0, atol=1e-16)
    assert np.allclose(np.einsum("q,qa,qb->ab", w, c, c), np.eye(3) / 3.0, atol=1e-15)
    assert np.allclose(np.einsum("q,qa,qb,qc->abc", w, c, c, c), 0.0, atol=1e-16)
    I = np.eye(3)
    iso4 = (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I)
            + np.einsum("ad,bc->abcd", I, I)) / 9.0
    assert np.allclose(np.einsum("q,qa,qb,qc,qd->abcd", w, c, c, c, c), iso4, atol=1e-15)


def _surface_tension_tensor(A, tau, F):
    """Eq. eqsurftens written out entry by entry as printed."""
    Fx, Fy, Fz = F
    M = np.array([[-Fy ** 2 - Fz ** 2, Fx * Fy, Fx * Fz],
                  [Fx * Fy, -Fx ** 2 - Fz ** 2, Fy * Fz],
                  [Fz * Fx, Fz * Fy, -Fx ** 2 - Fy ** 2]])
    return 2.0 * A * tau / (9.0 * np.linalg.norm(F)) * M


@pytest.mark.parametrize("seed", range(6))
def test_feq_moments(seed):
    rng = np.random.default_rng(seed)
    c, w, _ = _c()
    rho = rng.uniform(0.8, 1.2)
    u = rng.uniform(-0.05, 0.05, 3)
    eps = rng.uniform(0.2, 1.0)
    tau = rng.uniform(0.55, 1.5)
    A = rng.uniform(1e-4, 1e-2) if seed % 2 else 0.0
    F = rng.uniform(-1, 1, 3)
    fe = O.feq(rho, u, eps, tau, A, F)
    # zeroth and first moments: rho and rho V' (Eqs. macros1, macros)
    assert fe.sum() == pytest.approx(rho, rel=1e-14)
    assert np.allclose(fe @ c, rho * u, rtol=0, atol=1e-15)
    # second moment: rho c_s^2 I + rho u u / eps (porous Navier-Stokes, Eq.
    # momentum) plus eps*S from the surface-tension terms (Eq. eqsurftens)
    P = np.einsum("q,qa,qb->ab", fe, c, c)
    expect = rho / 3.0 * np.eye(3) + rho * np.outer(u, u) / eps
    if A:
        expect = expect + eps * _surface_tension_tensor(A, tau, F)
    assert np.allclose(P, expect, rtol=0, atol=1e-14)


def test_feq_without_gradient_has_no_surface_term():
    u = np.array([0.01, -0.02, 0.03])
    a = O.feq(1.1, u, 0.7, 0.9, 0.0, (0, 0, 0))
    b = O.feq(1.1, u, 0.7, 0.9, 5e-3, (0, 0, 0))
    assert np.array_equal(a, b)
    # at rest and without gradient f^eq reduces to w_q rho
    _, w, _ = _c()
    assert np.allclose(O.feq(1.3, np.zeros(3), 0.4, 0.8), 1.3 * w, rtol=1e-15)


@pytest.mark.parametrize("seed", range(6))
def test_forcing_moments(seed):
    rng = np.random.default_rng(100 + seed)
    c, w, _ = _c()
    rho, tau, eps = rng.uniform(0.8, 1.2), rng.uniform(0.55, 2.0), rng.uniform(0.2, 1.0)
    u = rng.uniform(-0.05, 0.05, 3)
    Fe = rng.uniform(-1e-3, 1e-3, 3)
    T = O.forcing(rho, tau, eps, u, Fe)
    pre = 1.0 - 0.5 / tau
    assert abs(T.sum()) < 1e-18
    assert np.allclose(T @ c, pre * rho * Fe, rtol=1e-13, atol=0)
    M2 = np.einsum("q,qa,qb->ab", T, c, c)
    assert np.allclose(M2, pre * rho * (np.outer(u, Fe) + np.outer(Fe, u)) / eps,
                       rtol=1e-12, atol=1e-20)


def _spd(rng, scale):
    A = rng.standard_normal((3, 3))
    return scale * (A @ A.T + 0.5 * np.eye(3))


@pytest.mark.parametrize("seed", range(8))
def test_velocity_solve_satisfies_implicit_equations(seed):
    """V' = V + F^ext/2 (Eq. expandV) with F^ext = -eps nu K^-1 V' + eps G
    (Eq. forcement): the solver output must satisfy both equations."""
    rng = np.random.default_rng(200 + seed)
    K = _spd(rng, 10 ** rng.uniform(-4, 0))
    Kinv = np.linalg.inv(K)
    V = rng.uniform(-0.05, 0.05, 3)
    G = rng.uniform(-1e-3, 1e-3, 3)
    eps, nu = rng.uniform(0.2, 1.0), rng.uniform(0.02, 0.4)
    Vp, Fe = O.velocity_solve(V, eps, nu, Kinv, G)
    assert np.allclose(Vp - 0.5 * Fe, V, rtol=0, atol=1e-15)
    assert np.allclose(Fe, -eps * nu * Kinv @ Vp + eps * G, rtol=1e-12, atol=1e-18)


def test_velocity_solve_without_medium():
    V = np.array([0.01, 0.02, -0.03])
    G = np.array([1e-3, 0, 2e-3])
    Vp, Fe = O.velocity_solve(V, 0.5, 0.1, None, G)
    assert np.allclose(Fe, 0.5 * G)
    assert np.allclose(Vp, V + 0.25 * G)


@pytest.mark.parametrize("seed", range(4))
def test_heq_moments(seed):
    rng = np.random.default_rng(300 + seed)
    c, w, _ = _c()
    eps, C = rng.uniform(0.2, 1.0), rng.uniform(0, 1)
    Vs = rng.uniform(-0.05, 0.05, 3)
    he = O.heq(eps, C, Vs)
    assert he.sum() == pytest.approx(eps * C, rel=1e-14)
    assert np.allclose(he @ c, eps * C * Vs, atol=1e-16)
    assert np.allclose(np.einsum("q,qa,qb->ab", he, c, c), eps * C / 3 * np.eye(3), atol=1e-16)


def test_viscosity_laws():
    p = W.random_medium()
    k = p.params
    # law 1: linear in the clamped concentration
    p1 = p.replace(params=dict(k, visc_law=1))
    assert O.tau_of(p1, 0.0, 5) == pytest.approx(k["tau0"])
    assert O.tau_of(p1, 1.0, 5) == pytest.approx(k["tau1"])
    assert O.tau_of(p1, 0.25, 5) == pytest.approx(k["tau0"] + 0.25 * (k["tau1"] - k["tau0"]))
    assert O.tau_of(p1, -3.0, 5) == pytest.approx(k["tau0"])
    assert O.tau_of(p1, 7.0, 5) == pytest.approx(k["tau1"])
    # law 2 (Eq. nuall): nu = (tau - 1/2)/3 factorises into a time factor and
    # a concentration factor with ratio exp(beta) between C = 0 and C = 1
    p2 = p.replace(params=dict(k, visc_law=2))
    nu = lambda C, t: (O.tau_of(p2, C, t) - 0.5) / 3.0
    assert nu(1.0, 0) == pytest.approx(k["nu_g"] * (1 + k["a"]), rel=1e-14)
    assert nu(0.0, 7) / nu(1.0, 7) == pytest.approx(np.exp(k["beta"]), rel=1e-14)
    assert nu(0.3, 40) / nu(0.3, 0) == pytest.approx(
        (1 + k["a"] * np.exp(k["alpha"] * 40)) / (1 + k["a"]), rel=1e-14)
    # law 0 is constant
    p0 = p.replace(params=dict(k, visc_law=0))
    assert O.tau_of(p0, 0.9, 100) == k["tau"]
