"""Forchheimer drag on the GPU (permeability mode with a diagonal K and the
Guo-Zhao inertial term) against the FP64 oracle and the Darcy-Forchheimer
closed form."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0912_4230_gb300 import lb, workloads as W

pytestmark = pytest.mark.gpu

TOL32 = dict(u=1e-5, rho=1e-6, C=1e-5, nu=3.4e-6)


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _fields_close(g, o, p, storage):
    rho, u, C, nu = g.fields()
    r_rho, r_u, r_C, r_nu = o.fields()
    live = p.solid == 0
    umax = np.abs(r_u[live]).max()
    if storage == "fp64":
        tol = dict(u=1.2e-7, rho=1.2e-7, C=1.2e-7, nu=1.2e-7)
    else:
        tol = TOL32
    assert np.abs(u[live] - r_u[live]).max() <= tol["u"] * umax
    assert np.abs(rho[live] - r_rho[live]).max() <= tol["rho"]
    assert np.abs(C[live] - r_C[live]).max() <= tol["C"]
    assert np.abs(nu[live] - r_nu[live]).max() <= tol["nu"]


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
@pytest.mark.parametrize("law", [1, 2])
def test_random_medium_with_forchheimer(storage, law):
    """Solids, walls, solute inlet/outlet, random diagonal K, strong drag
    (cF = 5); 19-cell rows with a ragged tail."""
    p = W.random_medium(19, 13, 11, seed=31, spd=False, visc_law=law, u_amp=0.05)
    p = p.replace(params=dict(p.params, forchheimer=5.0))
    g = lb.Lattice(p, storage=storage, check_every=1)
    g.step(30)
    o = O.Oracle(p)
    o.step(30)
    _fields_close(g, o, p, storage)
    f, h = g.populations()
    rf, rh = o.populations()
    live = p.solid == 0
    tolp = 1e-13 if storage == "fp64" else 2e-7
    assert np.abs(f[:, live] - rf[:, live]).max() < tolp
    assert np.abs(h[:, live] - rh[:, live]).max() < tolp


def test_forchheimer_medium_small_parity_and_balances():
    p = W.forchheimer(40, 36, 30, seed=3)
    g = lb.Lattice(p, storage="fp32", check_every=1)
    m0 = g.reduce()
    g.step(300)
    o = O.Oracle(p)
    o.step(300)
    _fields_close(g, o, p, "fp32")
    r, ro = g.reduce(), o.reduce()
    assert r[0] == pytest.approx(m0[0], rel=1e-9)
    assert r[2] == pytest.approx(ro[2], rel=1e-5)
    assert (r[1] - m0[1]) == pytest.approx(r[2] - r[3], rel=1e-4)


def test_forchheimer_medium_full_size_first_steps():
    """128^3 in the benchmark's configuration (autotuned launch), 3 steps,
    every cell against the oracle."""
    p = W.forchheimer(128, 128, 128, seed=0)
    g = lb.Lattice(p, storage="fp32")
    lb.lb_autotune(g.ctx, 2)
    g.step(3)
    o = O.Oracle(p)
    o.step(3)
    _fields_close(g, o, p, "fp32")


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_bulk_velocity_matches_darcy_forchheimer_closed_form(storage):
    K, eps, tau, G, cF = 10.0, 0.5, 0.8, 1.5e-3, 3.0
    p = W.forchheimer_bulk(K=(K, K, K), eps=eps, tau=tau, G=(G, 0.0, 0.0), cF=cF)
    g = lb.Lattice(p, storage=storage)
    g.step(2000)
    _, u, _, _ = g.fields()
    nu = (tau - 0.5) / 3
    a, b = cF * 1.75 / np.sqrt(150.0 * eps ** 3) / np.sqrt(K), nu / K
    ux = (-b + np.sqrt(b * b + 4 * a * G)) / (2 * a)
    tol = 2e-7 if storage == "fp64" else 2e-5   # fields are exported as float32
    assert np.abs(u[:, 0] - ux).max() <= tol * ux


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_row_staged_kernel_with_forchheimer(storage):
    p = W.forchheimer(40, 36, 30, seed=5)
    st = lb.Lattice(p, storage=storage, kernel="staged", check_every=1)
    cell = lb.Lattice(p, storage=storage, kernel="cell", check_every=1)
    st.step(20)
    cell.step(20)
    fs, hs = st.populations()
    fc, hc = cell.populations()
    tol = 1e-14 if storage == "fp64" else 5e-7
    assert np.abs(fs - fc).max() <= tol and np.abs(hs - hc).max() <= tol


def test_batched_forchheimer_lattices_equal_separate_steps():
    torch = pytest.importorskip("torch")
    s = torch.cuda.Stream()
    probs = [W.forchheimer(24, 20, 18, seed=i) for i in range(3)]
    sep = [lb.Lattice(p, storage="fp32", kernel="cell", check_every=1) for p in probs]
    bat = [lb.Lattice(p, storage="fp32", kernel="cell", check_every=1, stream=s.cuda_stream)
           for p in probs]
    for g in sep:
        g.step(25)
    lb.lb_step_batch([g.ctx for g in bat], 25)
    for a, b in zip(sep, bat):
        fa, ha = a.populations()
        fb, hb = b.populations()
        assert np.array_equal(fa, fb) and np.array_equal(ha, hb)


def test_full_tensor_with_forchheimer_is_unsupported():
    p = W.random_medium(8, 6, 5, seed=2, spd=True)
    p = p.replace(params=dict(p.params, forchheimer=1.0))
    with pytest.raises(lb.LbError) as e:
        lb.Lattice(p, storage="fp32")
    assert e.value.code == lb.LB_EUNSUPPORTED
