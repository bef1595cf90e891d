"""Oracle pins for the pressure and velocity faces (reading R23: the paper
lists pressure and flow-rate boundary conditions without a method; pressure
faces hold the face density 3 eps P of P = rho c_s^2 / eps by anti-bounce-back
on the even part of the porous equilibrium, velocity faces are moving-wall
bounce-back).

* pressure-driven flow through a uniform medium: the steady mass flux is
  K (rho_in - rho_out) / (3 eps nu L) (from -grad(rho c_s^2)/rho = eps nu V / K,
  the porous momentum equation in one dimension) and the density falls
  linearly between the face densities;
* porous Couette flow from a moving face: Brinkman's profile
  u_b sinh(r (L - z)) / sinh(r L), r = sqrt(eps / K), converging at second
  order;
* a flow rate imposed by a normal velocity face: mass flux rho u_in, and the
  pressure gradient of Darcy's law up to the outlet face density;
* surface tension or a free surface with open fluid faces is refused.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0912_4230_gb300 import workloads as W


def test_pressure_driven_darcy_flux_and_profile():
    p = W.pressure_darcy()
    o = O.Oracle(p)
    o.step(3000)
    rho, u, _, _ = o.fields()
    eps, K, nu, n = float(p.eps[0]), 1.0, (0.8 - 0.5) / 3, p.nx
    P_in, P_out = p.params["face_P"][0]
    rin, rout = 3 * eps * P_in, 3 * eps * P_out
    J = rho * u[:, 0]
    assert J.std() <= 1e-9 * J.mean()
    assert J.mean() == pytest.approx(K * (rin - rout) / (3 * eps * nu * n), rel=1e-6)
    x = np.arange(n) + 0.5
    assert np.abs(rho - (rin + (rout - rin) * x / n)).max() <= 1e-5 * (rin - rout)
    assert np.abs(u[:, 1:]).max() <= 1e-15


def _couette_error(nz, K):
    p = W.velocity_couette(nz=nz, K=K)
    o = O.Oracle(p)
    o.step({32: 8000, 64: 30000}[nz])
    _, u, _, _ = o.fields()
    eps, u_b = float(p.eps[0]), 1e-3
    r = np.sqrt(eps / K)
    zeta = np.arange(nz) + 0.5
    want = u_b * np.sinh(r * (nz - zeta)) / np.sinh(r * nz)
    return np.sqrt(((u[:, 0] - want) ** 2).sum() / (want ** 2).sum())


def test_moving_face_couette_profile_second_order():
    e32 = _couette_error(32, 16.0)
    e64 = _couette_error(64, 64.0)   # r L fixed
    assert e32 <= 2.5e-3
    assert 3.5 <= e32 / e64 <= 4.5


def test_flow_rate_face_mass_flux_and_gradient():
    p = W.inflow_darcy()
    o = O.Oracle(p)
    o.step(8000)
    rho, u, _, _ = o.fields()
    eps, K, nu, n = float(p.eps[0]), 1.0, (0.8 - 0.5) / 3, p.nx
    u_in = p.params["face_u"][0][0][0]
    J = rho * u[:, 0]
    assert J.std() <= 1e-9 * J.mean()
    assert J.mean() == pytest.approx(rho[0] * u_in, rel=1e-6)
    # Darcy: d rho / dx = -3 eps nu J / K; the line reaches 3 eps P_out at the face
    slope = np.polyfit(np.arange(n), rho, 1)[0]
    assert slope == pytest.approx(-3 * eps * nu * J.mean() / K, rel=1e-4)
    rout = 3 * eps * p.params["face_P"][0][1]
    assert rho[-1] + 0.5 * slope == pytest.approx(rout, abs=1e-4 * (rho[0] - rout))


@pytest.mark.parametrize("extra", [dict(A=1e-3), dict(free_surface=1)])
def test_open_faces_refuse_surface_tension_and_free_surface(extra):
    p = W.random_medium(5, 4, 6, seed=1, open_faces=True, solute=False)
    p = p.replace(K6=None, params=dict(p.params, **extra))
    with pytest.raises(Exception):
        O.Oracle(p)
