"""Pins of the oracle's lattice-level behaviour (CPU only): streaming and
boundary classes by brute force, exact conservation, the Brinkman and Darcy
closed forms (Section 5.1), the viscous and Darcy decay of a shear wave and of a
standing sound wave, the
paper's printed anisotropic-channel numbers
(Section 5.2), Gaussian diffusion and the porosity-gradient correction of the
solute lattice (Section 2.2), and the viscosity laws (Section 5.5)."""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_0912_4230_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
Q = 19


def brute_sources(p, kinds):
    """Pull sources by direct coordinate arithmetic: the population along c_q
    at x comes from x - c_q, wrapped modulo n on periodic faces."""
    c, _, _ = O.velocity_set()
    nx, ny, nz = p.nx, p.ny, p.nz
    dims = (nx, ny, nz)
    out = np.zeros((Q, p.N), np.int64)
    for n in range(p.N):
        X = (n % nx, (n // nx) % ny, n // (nx * ny))
        for q in range(Q):
            if p.solid[n]:
                out[q, n] = -1
                continue
            s = [X[a] - c[q][a] for a in range(3)]
            crossed = set()
            for a in range(3):
                if 0 <= s[a] < dims[a]:
                    continue
                kind = kinds[a][0 if s[a] < 0 else 1]
                if kind == W.PERIODIC:
                    s[a] %= dims[a]
                else:
                    crossed.add(kind)
            if W.WALL in crossed:
                out[q, n] = -2
            elif W.VELOCITY in crossed:
                out[q, n] = -7
            elif W.PRESSURE in crossed:
                out[q, n] = -6
            elif W.INLET in crossed:
                out[q, n] = -3
            elif W.OUTLET in crossed:
                out[q, n] = -4
            else:
                idx = s[0] + nx * (s[1] + ny * s[2])
                out[q, n] = -2 if p.solid[idx] else idx
    return out


@pytest.mark.parametrize("dims", [(3, 4, 5), (4, 3, 5), (1, 2, 3)])
@pytest.mark.parametrize("seed", [0, 1])
def test_neighbor_table_brute_force(dims, seed):
    p = W.random_medium(*dims, seed=seed, solid_frac=0.2)
    o = O.Oracle(p)
    for lattice, kinds in ((0, p.bc), (1, p.sbc)):
        assert np.array_equal(o.neighbors(lattice), brute_sources(p, kinds))


@pytest.mark.parametrize("dims", [(3, 4, 5), (5, 3, 4)])
def test_neighbor_table_brute_force_open_faces(dims):
    """Pressure and velocity faces, with their precedence on edges."""
    p = W.random_medium(*dims, seed=4, solid_frac=0.2, open_faces=True)
    o = O.Oracle(p)
    for lattice, kinds in ((0, p.bc), (1, p.sbc)):
        assert np.array_equal(o.neighbors(lattice), brute_sources(p, kinds))
    src = o.neighbors(0)
    assert (src == -6).any() and (src == -7).any()


def test_periodic_streaming_is_a_permutation():
    p = W.random_medium(5, 4, 3, walls=False, solute=False, solid_frac=0.0)
    src = O.Oracle(p).neighbors(0)
    for q in range(Q):
        assert sorted(src[q].tolist()) == list(range(p.N))


def test_one_step_moments_are_streamed_sums():
    """rho(x) = sum_q f_q(x - c_q) and rho V = sum_q f_q(x - c_q) c_q after one
    stream (flowchart steps f, h; Eqs. macros1, macros); with no medium and no
    force V' = V. Same for C = sum_q h_q(x - c_q)/eps."""
    p = W.random_medium(5, 4, 6, seed=3, solid_frac=0.15, spd=False)
    p = p.replace(K6=None, params=dict(p.params, G=(0.0, 0.0, 0.0), visc_law=0))
    rng = np.random.default_rng(7)
    f = rng.uniform(0.01, 0.1, (Q, p.N))
    h = rng.uniform(0.0, 0.05, (Q, p.N))
    o = O.Oracle(p)
    o.set_populations(f.ravel(), h.ravel())
    o.step(1)
    rho, u, C, _ = o.fields()
    c, _, opp = O.velocity_set()
    src = brute_sources(p, p.bc)
    ssrc = brute_sources(p, p.sbc)
    for n in range(p.N):
        if p.solid[n]:
            continue
        fs = np.array([f[opp[q], n] if src[q, n] == -2 else f[q, src[q, n]] for q in range(Q)])
        assert rho[n] == pytest.approx(fs.sum(), rel=1e-14)
        assert np.allclose(u[n], fs @ c / fs.sum(), rtol=1e-12, atol=1e-16)
        if (ssrc[:, n] < -2).any():
            continue  # inlet/outlet cells are pinned by the solute-balance test
        hs = np.array([h[opp[q], n] if ssrc[q, n] == -2 else h[q, ssrc[q, n]] for q in range(Q)])
        assert C[n] == pytest.approx(hs.sum() / p.eps[n], rel=1e-13)


@pytest.mark.parametrize("A", [0.0, 2e-3])
def test_mass_conservation(A):
    """sum_q f^eq_q = rho and sum_q T_q = 0, and bounce-back returns every
    population: the total mass stays constant to rounding (P4)."""
    p = W.random_medium(8, 7, 6, seed=5, A=A)
    o = O.Oracle(p)
    m0 = o.reduce()[0]
    for _ in range(5):
        o.step(20)
        assert o.reduce()[0] == pytest.approx(m0, rel=1e-13)


def test_solute_balance_with_inlet_and_outlet():
    """Sum h(t+1) - sum h(t) = flux_in - flux_out, step by step (P5)."""
    p = W.random_medium(8, 7, 6, seed=6)
    o = O.Oracle(p)
    prev = o.reduce()
    for _ in range(30):
        o.step(1)
        cur = o.reduce()
        d = cur[1] - prev[1]
        flux = (cur[2] - prev[2]) - (cur[3] - prev[3])
        assert d == pytest.approx(flux, abs=1e-12 * max(1.0, cur[1]))
        prev = cur
    assert cur[2] > 0  # the inlet really injects


def test_solute_conserved_when_periodic():
    p = W.random_medium(6, 5, 7, seed=8, inlet=False)
    o = O.Oracle(p)
    s0 = o.reduce()[1]
    o.step(50)
    assert o.reduce()[1] == pytest.approx(s0, rel=1e-13)


def _brinkman_error(nz, K, steps, tau=0.8, solute_C=None):
    p = W.brinkman(nz=nz, K=K, tau=tau)
    nu = (tau - 0.5) / 3.0
    if solute_C is not None:
        # uniform concentration with the linear law reduces to a constant tau
        N = p.N
        p = p.replace(params=dict(p.params, solute=1, visc_law=1, tau0=0.6, tau1=1.5, tau_D=0.8),
                      C0=np.full(N, solute_C, np.float32))
        nu = (0.6 + 0.9 * float(np.float32(solute_C)) - 0.5) / 3.0
    o = O.Oracle(p)
    o.step(steps)
    _, u, _, _ = o.fields()
    eps, Kf, G = float(p.eps[0]), float(p.K6[0]), p.params["G"][0]
    r = np.sqrt(eps / Kf)   # r = sqrt(nu eps / (K nu_e)) with nu = nu_e
    y = np.arange(nz) + 0.5  # halfway bounce-back: walls at y = 0 and y = L
    exact = G * Kf / nu * (1 - np.cosh(r * (y - nz / 2)) / np.cosh(r * nz / 2))
    return np.linalg.norm(u[:, 0] - exact) / np.linalg.norm(exact)


@pytest.mark.parametrize("tau", [0.55, 0.8, 0.5 + np.sqrt(3.0 / 16.0), 1.2, 2.0])
def test_poiseuille_exact_discrete_solution(tau):
    """Plane Poiseuille flow (eps = 1, no medium, body force G between two
    halfway bounce-back walls a distance L apart): the steady BGK solution
    on the lattice is the parabola plus a uniform slip fixed by tau alone,
    u(y) = G/(2 nu) [y (L - y) + (16 (tau - 1/2)^2 - 3)/12]
    (He, Zou, Luo and Dembo, J. Stat. Phys. 87 (1997): the halfway wall sits
    exactly at the link midpoint only for (tau - 1/2)^2 = 3/16). Reached to
    rounding for every tau; a misplaced wall, a dropped half force or a
    wrong viscosity would leave an error of order one in the slip term."""
    nz, G = 16, 1e-6
    p = W.brinkman(nz=nz, K=1.0, eps=1.0, tau=tau, G=G).replace(K6=None)
    o = O.Oracle(p)
    nu = (tau - 0.5) / 3.0
    o.step(int(np.ceil(40.0 * nz * nz / (np.pi ** 2 * nu))))   # 40 e-folds of the slowest mode
    _, u, _, _ = o.fields()
    y = np.arange(nz) + 0.5
    exact = G / (2 * nu) * (y * (nz - y) + (16 * (tau - 0.5) ** 2 - 3) / 12)
    assert np.abs(u[:, 0] - exact).max() <= 1e-9 * np.abs(exact).max()
    assert np.abs(u[:, 1:]).max() <= 1e-9 * np.abs(exact).max()


def test_brinkman_closed_form_and_convergence():
    """Eq. eq:darcy with the boundary layer resolved (1/r = 5.2 cells at
    L = 64): relative L2 error below 1e-2, second order under refinement at
    fixed Darcy number (P1)."""
    e64 = _brinkman_error(64, 16.0, 4000)
    e128 = _brinkman_error(128, 64.0, 12000)
    assert e64 < 1e-2
    assert 3.0 < e64 / e128 < 5.0


def test_brinkman_with_uniform_concentration_and_linear_viscosity():
    """With uniform C the hardening law is a constant tau and the channel is
    again the Brinkman profile with nu = (tau(C) - 1/2)/3 (P8)."""
    assert _brinkman_error(64, 16.0, 4000, solute_C=0.3) < 1e-2


def test_plain_channel_bulk_darcy_velocity():
    """16x16x64 plain channel, 2000 steps: away from the walls the flow is
    the Darcy velocity G K / nu (F^ext = 0), far below the FP64 noise floor;
    the cells next to the walls carry the decaying discrete boundary layer of
    the under-resolved (r = 7.75 per cell) profile (P2)."""
    p = W.plain_channel()
    o = O.Oracle(p)
    o.step(p.steps)
    _, u, _, _ = o.fields()
    ux = u[:, 0].reshape(p.shape)
    darcy = p.params["G"][0] * float(p.K6[0]) / ((0.8 - 0.5) / 3.0)
    bulk = ux[20:-20]
    assert np.abs(bulk / darcy - 1).max() < 1e-10
    assert np.abs(u[:, 1:]).max() < 1e-9 * darcy
    # the wall-layer deviation decays away from each wall
    dev = np.abs(ux[:, 0, 0] / darcy - 1)
    assert all(dev[k + 1] < dev[k] for k in range(10))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_darcy_bulk_full_spd_tensor(seed):
    """Uniform periodic medium at steady state: F^ext = 0, so V' = K G / nu
    exactly, also for a full SPD tensor (P2)."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((3, 3))
    K = 0.02 * (A @ A.T + np.eye(3))
    G = rng.uniform(-1e-5, 1e-5, 3)
    p = W.random_medium(2, 2, 2, seed=seed, solid_frac=0.0, walls=False, solute=False)
    N = p.N
    K6 = np.tile(np.array([K[0, 0], K[1, 1], K[2, 2], K[0, 1], K[1, 2], K[2, 0]], np.float32), N)
    p = p.replace(eps=np.full(N, 0.6, np.float32), K6=K6, rho0=np.ones(N, np.float32),
                  u0=np.zeros(3 * N, np.float32), params=dict(tau=0.8, G=tuple(G)))
    o = O.Oracle(p)
    o.step(3000)
    _, u, _, _ = o.fields()
    K64 = np.array([[K6[0], K6[3], K6[5]], [K6[3], K6[1], K6[4]], [K6[5], K6[4], K6[2]]], float)
    expect = K64 @ G / 0.1
    assert np.allclose(u, expect, rtol=1e-9, atol=1e-9 * np.abs(expect).max())


@pytest.mark.parametrize("direction,key,gold", [(0, "vx_max", "vx_max"), (1, "vy_max", "vy_max")])
def test_anisotropic_channel_paper_values(direction, key, gold):
    """Section 5.2: tau = 0.6, eps = 0.3, G = 0.1, K = diag(1e-3, 1e-5):
    the paper prints v_x,max = 3e-3 and v_y,max = 3e-5 (P3)."""
    g = GOLD["aniso_channel"]
    p = W.aniso_channel(direction=direction, n=g["lattice"][0], eps=g["porosity"], tau=g["tau"],
                        G=g["G"], Kxx=g["K_xx"], Kyy=g["K_yy"])
    o = O.Oracle(p)
    # the discrete wall layer of flow along y (r = 173 per cell) decays by a
    # factor of about 0.7 per cell and takes longer to settle at the centre
    o.step(300 if direction == 0 else 3000)
    _, u, _, _ = o.fields()
    comp = u[:, direction].reshape(p.ny, p.nx)
    centre = comp[p.ny // 2, p.nx // 2]
    assert centre == pytest.approx(g[gold], rel=1e-6)
    # cross-flow vanishes
    assert np.abs(u[:, 1 - direction]).max() < 1e-15


@pytest.mark.parametrize("dims", [(64, 1, 1), (1, 64, 1), (1, 1, 64)])
def test_gaussian_pulse_diffusion(dims):
    """Eq. diffusionporous with eps = 1 and V' = 0 is the diffusion equation
    with D = (tau_D - 1/2)/3: the variance grows by 2 D per step and the
    profile stays the analytic Gaussian (P6)."""
    tau_D = 0.8
    D = (tau_D - 0.5) / 3.0
    p = W.gaussian_pulse(*dims, sigma0=4.0, tau_D=tau_D)
    o = O.Oracle(p)
    axis = int(np.argmax(dims))
    n = dims[axis]
    x = np.arange(n, dtype=float)
    var = {}
    for t in (20, 120):
        o.step(t - o.t)
        _, _, C, _ = o.fields()
        m = C.sum()
        xb = (C * x).sum() / m
        var[t] = (C * (x - xb) ** 2).sum() / m
    assert (var[120] - var[20]) / 100 == pytest.approx(2 * D, rel=1e-4)
    s2 = 16.0 + 2 * D * 120
    exact = 4.0 / np.sqrt(s2) * np.exp(-(x - (n - 1) / 2) ** 2 / (2 * s2))
    assert np.linalg.norm(C - exact) / np.linalg.norm(exact) < 1e-2
    # total solute is conserved exactly
    assert C.sum() == pytest.approx(p.C0.astype(float).sum(), rel=1e-12)


def test_gaussian_pulse_isotropy_and_advection():
    """3D pulse advected by a uniform V': the centroid moves with V' t and the
    three variances grow alike (P6)."""
    u = (0.02, -0.01, 0.015)
    n = 40
    p = W.gaussian_pulse(n, n, n, sigma0=2.5, u=u)
    o = O.Oracle(p)
    t = 30
    o.step(t)
    _, uu, C, _ = o.fields()
    assert np.allclose(uu, u, atol=1e-12)
    Cg = C.reshape(p.shape)
    m = Cg.sum()
    cen, var = [], []
    for axis_np in (2, 1, 0):   # x, y, z
        prof = Cg.sum(axis=tuple(a for a in range(3) if a != axis_np))
        x = np.arange(n, dtype=float)
        xb = (prof * x).sum() / m
        cen.append(xb)
        var.append((prof * (x - xb) ** 2).sum() / m)
    expect = (n - 1) / 2 + np.array(u) * t
    assert np.allclose(cen, expect, atol=2e-3)
    assert max(var) - min(var) < 2e-3 * np.mean(var)


def test_porosity_gradient_correction_keeps_uniform_concentration():
    """With V' = 0 Eq. diffusionporous keeps a uniform C stationary in a
    heterogeneous medium; this needs the D grad(eps)/eps part of V* in
    Eq. equild (P7). Smooth porosity 0.6 + 0.25 sin(2 pi x / L): the lattice
    keeps C uniform up to a second-order discretisation error (without the
    correction the stationary state would be eps*C uniform, i.e. C varying by
    a factor 2.4)."""
    dev = {}
    for nx in (32, 64):
        p = W.eps_bands(nx, 2, 2, C=0.5)
        o = O.Oracle(p)
        o.step(2000)
        _, u, C, _ = o.fields()
        dev[nx] = np.abs(C - 0.5).max()
        assert np.abs(u).max() < 1e-14
    assert dev[64] < 1e-3
    assert 3.0 < dev[32] / dev[64] < 5.0


@pytest.mark.parametrize("law", [1, 2])
def test_viscosity_field_follows_concentration(law):
    """The exported nu is (tau(C, t) - 1/2)/3 of the exported C, cell by cell
    (Section 5.5, Eq. nuall; linear hardening law)."""
    p = W.random_medium(6, 5, 4, seed=11, visc_law=law)
    o = O.Oracle(p)
    o.step(7)
    _, _, C, nu = o.fields()
    k = p.params
    live = p.solid == 0
    if law == 1:
        expect = (k["tau0"] + (k["tau1"] - k["tau0"]) * np.clip(C, 0, 1) - 0.5) / 3.0
    else:
        expect = k["nu_g"] * (1 + k["a"] * np.exp(k["alpha"] * 7)) * np.exp(k["beta"] * (1 - C))
    assert np.allclose(nu[live], expect[live], rtol=1e-13)


def _shear_wave_rate(L, tau, eps=1.0, K=None, A=1e-4):
    """Decay rate of a shear wave u_x = A sin(2 pi y / L) in a periodic
    column, measured from the amplitudes of the sine mode at two times one
    e-folding apart (after the initial transient), and the continuum rate
    nu k^2 + eps nu / K of the Brinkman momentum equation (Eq. momentum with
    nu_e = nu, no body force; the Darcy part absent without K)."""
    p = W.gaussian_pulse(nx=1, ny=L, nz=1)
    y = np.arange(L)
    u0 = np.zeros((L, 3), np.float32)
    u0[:, 0] = A * np.sin(2 * np.pi * y / L)
    K6 = None if K is None else np.tile(np.array([K, K, K, 0, 0, 0], np.float32), L)
    p = p.replace(u0=u0.ravel(), C0=None, params=dict(tau=tau), eps=np.full(L, eps, np.float32),
                  K6=K6)
    k = 2 * np.pi / L
    nu = (tau - 0.5) / 3.0
    lam = nu * k * k + (0.0 if K is None else eps * nu / K)
    t1, t2 = int(0.2 / lam) + 5, int(1.2 / lam) + 5
    s = np.sin(k * y)
    o = O.Oracle(p)
    o.step(t1)
    a1 = (o.fields()[1][:, 0] * s).sum()
    o.step(t2 - t1)
    a2 = (o.fields()[1][:, 0] * s).sum()
    assert np.abs(o.fields()[1][:, 1:]).max() <= 1e-9 * A   # the wave stays transverse
    return -np.log(a2 / a1) / (t2 - t1), lam


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.2])
def test_shear_wave_decays_at_the_viscous_rate(tau):
    """Free fluid (eps = 1): the measured rate tends to nu k^2 with
    nu = (tau - 1/2)/3 at second order in k (the error falls fourfold when L
    doubles) and is within 1e-3 of it at L = 64. A wrong viscosity, or a
    relaxation that is not BGK's 1/tau, fails by far more than that."""
    errs = []
    for L in (32, 64):
        r, lam = _shear_wave_rate(L, tau)
        errs.append(r / lam - 1.0)
    assert abs(errs[1]) < 1e-3
    assert 3.5 < errs[0] / errs[1] < 4.5


@pytest.mark.parametrize("tau", [0.6, 1.2])
def test_shear_wave_in_a_porous_medium_adds_the_darcy_rate(tau):
    """eps = 0.6 with isotropic K = 0.004 L^2 (a fixed Darcy number, the drag
    79 % of the rate): the rate tends to nu k^2 + eps nu / K at second order
    (the half-force velocity V' of Eqs. expandV / expandVsub turns the drag
    into an exact per-step factor (1 - a/2)/(1 + a/2), a = eps nu / K, whose
    rate differs from a by a^3/12 only). Without the drag, or with K in place
    of K/eps, the rate is off by tens of percent."""
    errs = []
    for L in (32, 64):
        r, lam = _shear_wave_rate(L, tau, eps=0.6, K=0.004 * L * L)
        errs.append(r / lam - 1.0)
    assert abs(errs[1]) < 1e-3
    assert 3.5 < errs[0] / errs[1] < 4.5


def _sound_wave_error(L, tau, eps=1.0, K=None, d=1e-5, periods=2):
    """Largest deviation, over two periods, of the density mode of a standing
    sound wave rho = 1 + d cos(k x) (fluid at rest, periodic row) from the
    damped oscillation of the linearised equations: with pressure rho/3 (the
    second moment of Eqs. equilc1 / equilc2), BGK's shear and bulk viscosity
    (nu and 2 nu / 3) and the Darcy drag a = eps nu / K, the mode obeys
    rho'' + (2 nu k^2 + a) rho' + (k^2 / 3) rho = 0, so with rho' = 0 at t = 0
    it is e^{-G t} (cos w t + (G / w) sin w t), G = nu k^2 + a / 2,
    w^2 = k^2 / 3 - G^2. Relative to the initial amplitude."""
    p = W.gaussian_pulse(nx=L, ny=1, nz=1)
    x = np.arange(L)
    k = 2 * np.pi / L
    K6 = None if K is None else np.tile(np.array([K, K, K, 0, 0, 0], np.float32), L)
    p = p.replace(rho0=(1.0 + d * np.cos(k * x)).astype(np.float32), C0=None,
                  params=dict(tau=tau), eps=np.full(L, eps, np.float32), K6=K6)
    nu = (tau - 0.5) / 3.0
    G = nu * k * k + (0.0 if K is None else 0.5 * eps * nu / K)
    w = np.sqrt(k * k / 3.0 - G * G)
    c = np.cos(k * x)
    o = O.Oracle(p)
    a0 = (o.fields()[0] - 1.0) @ c
    err = 0.0
    for t in range(1, int(periods * 2 * np.pi / w) + 1):
        o.step(1)
        model = a0 * np.exp(-G * t) * (np.cos(w * t) + G / w * np.sin(w * t))
        err = max(err, abs((o.fields()[0] - 1.0) @ c - model))
    return err / abs(a0)


@pytest.mark.parametrize("tau", [0.6, 0.8])
@pytest.mark.parametrize("porous", [False, True])
def test_sound_wave_speed_and_damping(tau, porous):
    """The density mode follows the damped oscillation at second order in k
    (the deviation falls at least threefold when L doubles, below 3e-3 of
    the amplitude at L = 64), free (eps = 1) and in a porous medium (eps =
    0.6, K = 0.004 L^2): pins the pressure rho/3, the bulk damping of BGK and
    the Darcy drag's share of the damping of a compressive mode."""
    kw = lambda L: dict(eps=0.6, K=0.004 * L * L) if porous else {}
    e32, e64 = (_sound_wave_error(L, tau, **kw(L)) for L in (32, 64))
    assert e64 < 3e-3
    assert e32 / e64 > 3.0
