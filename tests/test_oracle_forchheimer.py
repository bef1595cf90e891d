"""Oracle pins for the Forchheimer drag (reading R21: the porous-flow model of
Guo and Zhao that the paper builds on, F_eps = cF 1.75 / sqrt(150 eps^3)).

* isotropic K: the velocity solve equals Guo and Zhao's closed form
  u = v / (c0 + sqrt(c0^2 + c1 |v|)), c0 = (1 + eps nu / (2K)) / 2,
  c1 = eps F_eps / (2 sqrt(K)), v = V + eps G / 2;
* diagonal K: V' = V + F^ext / 2 and the root is unique (bisection bracket);
* cF = 0 is the Darcy solve; no medium means no drag;
* lattice: the steady velocity of a uniform periodic medium balances the body
  force, nu K^-1 V' + F_eps |V'| K^-1/2 V' = G, solved independently here by a
  scalar root finder (isotropic: a quadratic);
* a full (non-diagonal) K with Forchheimer drag is refused.
"""
import numpy as np
import pytest
from scipy.optimize import brentq

from oracle import oracle as O
from paper_0912_4230_gb300 import workloads as W


def ergun(eps, cF=1.0):
    return cF * 1.75 / np.sqrt(150.0 * eps ** 3)


@pytest.mark.parametrize("seed", range(6))
def test_isotropic_solve_is_guo_zhao_closed_form(seed):
    rng = np.random.default_rng(seed)
    for _ in range(50):
        V = rng.normal(size=3) * 10 ** rng.uniform(-5, -1)
        G = rng.normal(size=3) * 10 ** rng.uniform(-6, -2)
        eps, nu = rng.uniform(0.3, 1.0), rng.uniform(0.02, 0.4)
        K = 10 ** rng.uniform(-3, 2)
        cF = 10 ** rng.uniform(-1, 1)
        Vp, Fe = O.velocity_solve(V, eps, nu, np.eye(3) / K, G, cF)
        v = V + 0.5 * eps * G
        c0 = 0.5 * (1.0 + 0.5 * eps * nu / K)
        c1 = 0.5 * eps * ergun(eps, cF) / np.sqrt(K)
        u = v / (c0 + np.sqrt(c0 * c0 + c1 * np.linalg.norm(v)))
        assert np.abs(Vp - u).max() <= 1e-13 * np.abs(u).max()


@pytest.mark.parametrize("seed", range(4))
def test_diagonal_solve_half_force_velocity(seed):
    rng = np.random.default_rng(100 + seed)
    for _ in range(50):
        V = rng.normal(size=3) * 10 ** rng.uniform(-5, -1)
        G = rng.normal(size=3) * 10 ** rng.uniform(-6, -2)
        eps, nu = rng.uniform(0.3, 1.0), rng.uniform(0.02, 0.4)
        k = 10 ** rng.uniform(-2, 3, 3)
        cF = 10 ** rng.uniform(-1, 1)
        Vp, Fe = O.velocity_solve(V, eps, nu, np.diag(k), G, cF)
        # the half-force velocity
        assert np.abs(Vp - (V + 0.5 * Fe)).max() <= 1e-14 * max(np.abs(Vp).max(), 1e-30) + 1e-18
        # drag: Darcy part plus the Forchheimer part along each principal axis
        drag = eps * nu * k * Vp + eps * ergun(eps, cF) * np.sqrt(k) * np.linalg.norm(Vp) * Vp
        scale = max(np.abs(eps * G).max(), np.abs(drag).max())
        assert np.abs(Fe - (eps * G - drag)).max() <= 1e-15 * scale


def test_zero_coefficient_is_darcy_and_no_medium_no_drag():
    rng = np.random.default_rng(7)
    V, G = rng.normal(size=3) * 1e-2, rng.normal(size=3) * 1e-4
    k = np.diag([3.0, 0.5, 20.0])
    a = O.velocity_solve(V, 0.6, 0.1, k, G, 0.0)
    b = O.velocity_solve(V, 0.6, 0.1, k, G)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    Vp, Fe = O.velocity_solve(V, 0.6, 0.1, None, G, 2.0)
    assert np.allclose(Vp, V + 0.5 * 0.6 * G, rtol=1e-15) and np.allclose(Fe, 0.6 * G, rtol=1e-15)


def _steady(p, steps):
    o = O.Oracle(p)
    o.step(steps)
    _, u, _, _ = o.fields()
    return u


def test_isotropic_bulk_balances_body_force():
    K, eps, tau, G, cF = 10.0, 0.5, 0.8, 1.5e-3, 3.0
    p = W.forchheimer_bulk(K=(K, K, K), eps=eps, tau=tau, G=(G, 0.0, 0.0), cF=cF)
    u = _steady(p, 2000)
    nu = (tau - 0.5) / 3
    a, b = ergun(eps, cF) / np.sqrt(K), nu / K
    ux = (-b + np.sqrt(b * b + 4 * a * G)) / (2 * a)
    assert np.abs(u[:, 0] - ux).max() <= 1e-10 * ux
    assert np.abs(u[:, 1:]).max() <= 1e-14
    # the Forchheimer drag matters here: the Darcy velocity would be ~3x larger
    assert G * K / nu > 2 * ux


def test_anisotropic_bulk_balances_oblique_body_force():
    K, eps, tau, cF = (2.0, 0.25, 8.0), 0.6, 0.7, 2.0
    G = np.array([2e-3, -1e-3, 1.5e-3])
    p = W.forchheimer_bulk(K=K, eps=eps, tau=tau, G=tuple(G), cF=cF)
    u = _steady(p, 3000)
    nu = (tau - 0.5) / 3
    k = 1.0 / np.array(K, dtype=np.float64)
    Fe = ergun(float(p.eps[0]), cF)  # the porosity as stored (float32)

    def vel(s):
        return G / (nu * k + Fe * np.sqrt(k) * s)

    s = brentq(lambda s: np.linalg.norm(vel(s)) - s, 0.0, np.linalg.norm(G / (nu * k)), xtol=1e-16)
    want = vel(s)
    assert np.abs(u - want).max() <= 1e-12 * np.abs(want).max()
    # not parallel to G: the anisotropic drag turns the flow
    cosang = u[0] @ G / (np.linalg.norm(u[0]) * np.linalg.norm(G))
    assert cosang < 0.99


def test_full_tensor_with_forchheimer_is_refused():
    p = W.random_medium(6, 5, 4, seed=2, spd=True)
    p = p.replace(params=dict(p.params, forchheimer=1.0))
    with pytest.raises(Exception):
        O.Oracle(p)
