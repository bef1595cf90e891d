"""The seeded input recipes (CPU only): the workloads have the structure the
benchmark configurations state, and a seed fixes every array."""
import numpy as np
import pytest

from paper_0912_4230_gb300 import workloads as W


def test_miscible_medium_structure():
    """Porosity bands of period 16 along x (0.35 / 0.85 +- 0.05), diagonal K
    with K_zz = 100 K_xx and K_xx log-uniform in [1e-4, 1e-2], solute inlet
    and outlet on the z faces, the linear hardening law."""
    p = W.miscible(32, 8, 8, seed=0)
    eps = p.eps.reshape(p.nz, p.ny, p.nx)
    low, high = eps[:, :, (np.arange(32) % 16) < 8], eps[:, :, (np.arange(32) % 16) >= 8]
    assert np.all(np.abs(low - 0.35) <= 0.05 + 1e-6) and np.all(np.abs(high - 0.85) <= 0.05 + 1e-6)
    K = p.K6.reshape(p.N, 6)
    assert np.all(K[:, 3:] == 0)
    assert np.allclose(K[:, 2], 100 * K[:, 0], rtol=1e-6) and np.array_equal(K[:, 0], K[:, 1])
    assert 1e-4 * (1 - 1e-6) <= K[:, 0].min() and K[:, 0].max() <= 1e-2 * (1 + 1e-6)
    assert p.sbc[2] == (W.INLET, W.OUTLET) and p.bc == W.ALL_PERIODIC
    assert p.params["visc_law"] == 1 and (p.params["tau0"], p.params["tau1"]) == (0.6, 1.5)


def test_precision_tensors_are_rotated_diagonals_per_block():
    """K = R_b diag(K_xx, K_xx, 100 K_xx) R_b^T: SPD with those eigenvalues in
    every cell, one rotation per block (the eigenvector of the large
    eigenvalue is the same throughout a block and differs between blocks)."""
    p = W.precision(16, 16, 16, block=8, storage="fp32")
    K6 = p.K6.reshape(p.N, 6).astype(np.float64)
    K = np.zeros((p.N, 3, 3))
    K[:, 0, 0], K[:, 1, 1], K[:, 2, 2] = K6[:, 0], K6[:, 1], K6[:, 2]
    K[:, 0, 1] = K[:, 1, 0] = K6[:, 3]
    K[:, 1, 2] = K[:, 2, 1] = K6[:, 4]
    K[:, 2, 0] = K[:, 0, 2] = K6[:, 5]
    lam, vec = np.linalg.eigh(K)
    kxx = W.miscible(16, 16, 16, seed=0).K6.reshape(p.N, 6)[:, 0].astype(np.float64)
    assert np.allclose(lam[:, 0], kxx, rtol=1e-5) and np.allclose(lam[:, 1], kxx, rtol=1e-5)
    assert np.allclose(lam[:, 2], 100 * kxx, rtol=1e-5)
    axis = vec[:, :, 2] * np.sign(vec[:, 2:3, 2] + 1e-30)
    n = np.arange(p.N)
    x, y, z = n % 16, (n // 16) % 16, n // 256
    block = (x // 8) + 2 * ((y // 8) + 2 * (z // 8))
    for b in range(8):
        a = axis[block == b]
        assert np.allclose(np.abs(a @ a[0]), 1.0, atol=1e-4)
    firsts = np.array([axis[block == b][0] for b in range(8)])
    assert np.abs(firsts @ firsts.T - np.eye(8)).max() > 0.05   # the blocks are rotated differently


@pytest.mark.parametrize("factory", [lambda s: W.miscible(16, 8, 8, seed=s),
                                     lambda s: W.random_medium(8, 6, 5, seed=s),
                                     lambda s: W.drop(nx=16, ny=16, nz=16, R=4.0, gap=3.0, seed=s)])
def test_a_seed_fixes_every_array(factory):
    a, b, c = factory(3), factory(3), factory(4)
    for name in ("eps", "K6", "solid", "rho0", "u0", "C0", "f_scale"):
        x, y, z = getattr(a, name), getattr(b, name), getattr(c, name)
        if x is None:
            continue
        assert np.array_equal(x, y), name
    assert any(getattr(a, n) is not None and not np.array_equal(getattr(a, n), getattr(c, n))
               for n in ("eps", "K6", "u0", "f_scale", "solid") if getattr(a, n) is not None)


def test_request_stream_statistics():
    """Poisson arrivals at 50 per second, sides from {32, ..., 160}, z-aspect
    between 1 and 2, steps between 2000 and 20000."""
    reqs = W.requests(n=256, rate=50.0, seed=5)
    arr = np.array([r["arrival"] for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], arr]))
    assert np.all(gaps >= 0) and 0.015 < gaps.mean() < 0.025
    assert {r["nx"] for r in reqs} <= {32, 48, 64, 96, 128, 160}
    assert all(r["nx"] == r["ny"] and r["nx"] <= r["nz"] <= 2 * r["nx"] for r in reqs)
    assert all(2000 <= r["steps"] <= 20000 for r in reqs)
