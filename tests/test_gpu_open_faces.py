"""Pressure and velocity faces of the fluid lattice on the GPU, against the
FP64 oracle (bit-exact boundary classes, fields and populations) and against
the closed forms the oracle is pinned to."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0912_4230_gb300 import lb, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("dims", [(3, 4, 5), (19, 7, 6)])
def test_open_face_classes_bit_exact(dims):
    p = W.random_medium(*dims, seed=4, solid_frac=0.2, open_faces=True)
    g = lb.Lattice(p, storage="fp32")
    o = O.Oracle(p)
    for lattice in (0, 1):
        assert np.array_equal(g.neighbors(lattice), o.neighbors(lattice))


@pytest.mark.parametrize("storage", ["fp64", "fp32", "fp16"])
def test_random_medium_with_open_faces(storage):
    """Velocity and pressure faces along x, pressure faces along z (with
    solute inlet/outlet on the same faces), walls along y, solids, full K."""
    p = W.random_medium(19, 13, 11, seed=23, open_faces=True)
    g = lb.Lattice(p, storage=storage, check_every=1)
    g.step(25)
    o = O.Oracle(p)
    o.step(25)
    rho, u, C, nu = g.fields()
    r_rho, r_u, r_C, r_nu = o.fields()
    live = p.solid == 0
    umax = np.abs(r_u[live]).max()
    tol = {"fp64": (1.2e-7, 1.2e-7, 1.2e-7), "fp32": (1e-5, 1e-6, 1e-5),
           "fp16": (1e-3, 2e-5, 1e-3)}[storage]
    assert np.abs(u[live] - r_u[live]).max() <= tol[0] * umax
    assert np.abs(rho[live] - r_rho[live]).max() <= tol[1]
    assert np.abs(C[live] - r_C[live]).max() <= tol[2]
    if storage != "fp16":
        f, h = g.populations()
        rf, rh = o.populations()
        tolp = 1e-13 if storage == "fp64" else 2e-7
        assert np.abs(f[:, live] - rf[:, live]).max() < tolp
        assert np.abs(h[:, live] - rh[:, live]).max() < tolp


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_pressure_driven_darcy_flux(storage):
    p = W.pressure_darcy()
    g = lb.Lattice(p, storage=storage)
    g.step(3000)
    rho, u, _, _ = g.fields()
    eps, K, nu, n = float(p.eps[0]), 1.0, (0.8 - 0.5) / 3, p.nx
    P_in, P_out = p.params["face_P"][0]
    rin, rout = 3 * eps * P_in, 3 * eps * P_out
    J = rho.astype(np.float64) * u[:, 0]
    want = K * (rin - rout) / (3 * eps * nu * n)
    assert J.mean() == pytest.approx(want, rel=1e-6 if storage == "fp64" else 2e-4)


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_moving_face_couette(storage):
    nz, K = 32, 16.0
    p = W.velocity_couette(nz=nz, K=K)
    g = lb.Lattice(p, storage=storage)
    g.step(8000)
    _, u, _, _ = g.fields()
    eps, u_b = float(p.eps[0]), 1e-3
    r = np.sqrt(eps / K)
    zeta = np.arange(nz) + 0.5
    want = u_b * np.sinh(r * (nz - zeta)) / np.sinh(r * nz)
    err = np.sqrt(((u[:, 0] - want) ** 2).sum() / (want ** 2).sum())
    assert err <= 2.5e-3


def test_flow_rate_face_mass_flux():
    p = W.inflow_darcy()
    g = lb.Lattice(p, storage="fp64")
    g.step(8000)
    rho, u, _, _ = g.fields()
    J = rho.astype(np.float64) * u[:, 0]
    assert J.mean() == pytest.approx(float(rho[0]) * p.params["face_u"][0][0][0], rel=1e-6)


def test_open_faces_use_the_per_cell_kernel_only():
    p = W.random_medium(64, 8, 8, seed=2, open_faces=True)
    with pytest.raises(lb.LbError) as e:
        lb.Lattice(p, storage="fp32", kernel="staged")
    assert e.value.code == lb.LB_EUNSUPPORTED
    g = lb.Lattice(p, storage="fp32")
    choice = lb.lb_autotune(g.ctx, 2)
    assert choice in (32, 64, 128)


def test_open_face_lattice_in_a_batch_equals_its_own_steps():
    torch = pytest.importorskip("torch")
    s = torch.cuda.Stream()
    probs = [W.random_medium(12, 9, 8, seed=50 + i, open_faces=(i == 1), spd=False) for i in range(3)]
    sep = [lb.Lattice(p, storage="fp32", kernel="cell", check_every=1) for p in probs]
    bat = [lb.Lattice(p, storage="fp32", kernel="cell", check_every=1, stream=s.cuda_stream)
           for p in probs]
    for g in sep:
        g.step(15)
    lb.lb_step_batch([g.ctx for g in bat], 15)
    for a, b in zip(sep, bat):
        fa, ha = a.populations()
        fb, hb = b.populations()
        assert np.array_equal(fa, fb) and np.array_equal(ha, hb)
