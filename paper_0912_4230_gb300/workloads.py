"""Seeded synthetic inputs for the porous-media lattice-Boltzmann solver.

This module only builds input arrays (geometry, porosity, permeability,
initial fields, cell types, seeded perturbation factors) and parameter sets.
It contains none of the method's arithmetic, so the CUDA library and the CPU
oracle can both be fed from it without sharing any part of the computation.

Every array is float32 (uint8 for masks and cell types) in the cell order
n = x + nx*(y + ny*z); populations-shaped arrays are direction-major [19, N].
Random draws use numpy's PCG64 with an explicit seed.

The workloads follow the paper's experiments (Section 5) and the five
workload families of this library:
  plain_channel   16x16x64 Brinkman channel, FP64 (Section 5.1 analogue)
  miscible        layered anisotropic medium with solute inlet, 128^3
  drop            free-surface drop falling onto a solid wall (Section 5.3 analogue)
  precision       256^3, fully anisotropic SPD permeability per 32^3 block
  requests        stream of served solves of different sizes
plus the small validation problems used to pin the oracle.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

Q = 19
PERIODIC, WALL, INLET, OUTLET = 0, 1, 2, 3
LIQUID, INTERFACE, EMPTY = 0, 1, 2

PRESSURE, VELOCITY = 4, 5     # fluid faces only
ALL_PERIODIC = ((PERIODIC, PERIODIC),) * 3


@dataclass
class Problem:
    name: str
    nx: int
    ny: int
    nz: int
    bc: tuple
    sbc: tuple
    params: dict
    eps: np.ndarray
    K6: Optional[np.ndarray]
    solid: np.ndarray
    rho0: np.ndarray
    u0: np.ndarray
    C0: Optional[np.ndarray] = None
    cell_type: Optional[np.ndarray] = None
    lambda0: Optional[np.ndarray] = None
    f_scale: Optional[np.ndarray] = None
    steps: int = 0
    storage: str = "fp32"
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def shape(self):
        """(nz, ny, nx): numpy view order of a cell field."""
        return (self.nz, self.ny, self.nx)

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _grid(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.ravel(), y.ravel(), z.ravel()


def _uniform(N, v, dtype=np.float32):
    return np.full(N, v, dtype=dtype)


def _iso_K6(N, k):
    K6 = np.zeros((N, 6), np.float32)
    K6[:, 0:3] = k
    return K6.ravel()


def _base(name, nx, ny, nz, bc, sbc, params, eps, K6, solid=None, **kw):
    N = nx * ny * nz
    if solid is None:
        solid = np.zeros(N, np.uint8)
    return Problem(name=name, nx=nx, ny=ny, nz=nz, bc=bc, sbc=sbc, params=params,
                   eps=np.asarray(eps, np.float32), K6=K6, solid=solid,
                   rho0=kw.pop("rho0", _uniform(N, 1.0)),
                   u0=kw.pop("u0", np.zeros(3 * N, np.float32)), **kw)


# --------------------------------------------------------------------------
# Workload families
# --------------------------------------------------------------------------

def plain_channel(nx=16, ny=16, nz=64, steps=2000) -> Problem:
    """Single fluid, no solute: periodic in x and y, walls at both z ends,
    porosity 0.6, isotropic K = 1e-2, tau = 0.8, body force 1e-6 along x."""
    N = nx * ny * nz
    bc = ((PERIODIC, PERIODIC), (PERIODIC, PERIODIC), (WALL, WALL))
    params = dict(tau=0.8, G=(1e-6, 0.0, 0.0))
    return _base("plain_channel", nx, ny, nz, bc, bc, params, _uniform(N, 0.6),
                 _iso_K6(N, 1e-2), steps=steps, storage="fp64")


def miscible(nx=128, ny=128, nz=128, seed=0, steps=5000, storage="fp32") -> Problem:
    """Fluid plus solute in a layered, anisotropic porous medium.

    Porosity: bands of period 16 cells along x alternating 0.35 / 0.85, plus
    seeded U(-0.05, 0.05) per cell. Permeability: diagonal with
    K_xx = K_yy log-uniform in [1e-4, 1e-2] per cell and K_zz = 100 K_xx.
    Flow is driven by a body force 1e-5 along z (periodic fluid lattice); the
    solute enters at z = 0 with C = 1 and leaves at z = nz-1. Viscosity law:
    tau = 0.6 + 0.9 C. Solute relaxation time 0.8. Initial C = 0.
    """
    rng = _rng(seed)
    N = nx * ny * nz
    x, _, _ = _grid(nx, ny, nz)
    eps = np.where((x % 16) < 8, 0.35, 0.85) + rng.uniform(-0.05, 0.05, N)
    kxx = 10.0 ** rng.uniform(-4.0, -2.0, N)
    K6 = np.zeros((N, 6), np.float64)
    K6[:, 0] = kxx
    K6[:, 1] = kxx
    K6[:, 2] = 100.0 * kxx
    bc = ALL_PERIODIC
    sbc = ((PERIODIC, PERIODIC), (PERIODIC, PERIODIC), (INLET, OUTLET))
    params = dict(visc_law=1, tau0=0.6, tau1=1.5, G=(0.0, 0.0, 1e-5), solute=1,
                  tau_D=0.8, C_in=1.0)
    return _base("miscible", nx, ny, nz, bc, sbc, params, eps.astype(np.float32),
                 K6.astype(np.float32).ravel(), C0=np.zeros(N, np.float32),
                 steps=steps, storage=storage, meta=dict(seed=seed))


def forchheimer(nx=128, ny=128, nz=128, seed=0, steps=5000, storage="fp32", cF=1.0,
                G=1e-4) -> Problem:
    """The miscible medium made coarse enough for inertial drag: diagonal K with
    K_xx = K_yy = 10^U(-2, 0) per cell and K_zz = 10 K_xx, body force G along
    z, Forchheimer drag with the Ergun coefficient times cF. Porosity bands,
    solute inlet/outlet and viscosity law as in the miscible medium."""
    base = miscible(nx, ny, nz, seed=seed, steps=steps, storage=storage)
    rng = _rng(seed + 1000)
    N = nx * ny * nz
    kxx = 10.0 ** rng.uniform(-2.0, 0.0, N)
    K6 = np.zeros((N, 6), np.float32)
    K6[:, 0] = kxx
    K6[:, 1] = kxx
    K6[:, 2] = 10.0 * kxx
    params = dict(base.params, G=(0.0, 0.0, G), forchheimer=cF)
    return base.replace(name="forchheimer", K6=K6.ravel(), params=params)


def forchheimer_bulk(K=(1.0, 1.0, 1.0), eps=0.5, tau=0.8, G=(6e-3, 0.0, 0.0), cF=1.0,
                     n=4, steps=600) -> Problem:
    """Uniform periodic medium with diagonal K, body force G and Forchheimer
    drag: the steady velocity is uniform and solves the Darcy-Forchheimer
    balance."""
    N = n * n * n
    K6 = np.zeros((N, 6), np.float32)
    K6[:, 0], K6[:, 1], K6[:, 2] = K
    return _base("forchheimer_bulk", n, n, n, ALL_PERIODIC, ALL_PERIODIC,
                 dict(tau=tau, G=tuple(G), forchheimer=cF), _uniform(N, eps), K6.ravel(),
                 steps=steps, storage="fp64")


def _faces(P=None, u=None):
    fp = [[0.0, 0.0] for _ in range(3)]
    fu = [[[0.0] * 3, [0.0] * 3] for _ in range(3)]
    for (a, side), v in (P or {}).items():
        fp[a][side] = float(v)
    for (a, side), v in (u or {}).items():
        fu[a][side] = [float(c) for c in v]
    return tuple(tuple(x) for x in fp), tuple(tuple(tuple(y) for y in x) for x in fu)


def pressure_darcy(n=64, dP=4e-4, K=1.0, eps=0.5, tau=0.8, steps=4000) -> Problem:
    """Flow through a uniform medium between two PRESSURE faces along x
    (periodic y and z, one cell thick), face pressures 1/(3 eps) +- dP/2 (face
    densities near 1): the steady mass flux is uniform and the density falls
    linearly between the face densities 3 eps P."""
    N = n
    P0 = 1.0 / (3.0 * float(np.float32(eps)))
    P_in, P_out = P0 + 0.5 * dP, P0 - 0.5 * dP
    bc = ((PRESSURE, PRESSURE), (PERIODIC, PERIODIC), (PERIODIC, PERIODIC))
    fp, fu = _faces(P={(0, 0): P_in, (0, 1): P_out})
    K6 = np.zeros((N, 6), np.float32)
    K6[:, 0:3] = K
    return _base("pressure_darcy", n, 1, 1, bc, ((OUTLET, OUTLET),) + ALL_PERIODIC[1:],
                 dict(tau=tau, face_P=fp, face_u=fu), _uniform(N, eps), K6.ravel(),
                 rho0=_uniform(N, 3.0 * eps * 0.5 * (P_in + P_out)), steps=steps,
                 storage="fp64")


def velocity_couette(nz=32, u_b=1e-3, K=16.0, eps=0.6, tau=0.8, steps=6000) -> Problem:
    """Porous Couette flow: the z-low face moves with u_b along x (VELOCITY),
    the z-high face is a wall, x and y periodic; the steady profile solves
    Brinkman's equation nu V'' = eps nu V / K."""
    N = nz
    bc = ((PERIODIC, PERIODIC), (PERIODIC, PERIODIC), (VELOCITY, WALL))
    sbc = ((PERIODIC, PERIODIC), (PERIODIC, PERIODIC), (WALL, WALL))
    fp, fu = _faces(u={(2, 0): (u_b, 0.0, 0.0)})
    K6 = np.zeros((N, 6), np.float32)
    K6[:, 0:3] = K
    return _base("velocity_couette", 1, 1, nz, bc, sbc, dict(tau=tau, face_P=fp, face_u=fu),
                 _uniform(N, eps), K6.ravel(), steps=steps, storage="fp64")


def inflow_darcy(n=64, u_in=2e-4, K=1.0, eps=0.5, tau=0.8, steps=4000) -> Problem:
    """Flow rate imposed at the x-low face (VELOCITY, normal inflow u_in),
    pressure 1/(3 eps) at the x-high face (face density 1), uniform medium,
    periodic y and z."""
    N = n
    P_out = 1.0 / (3.0 * float(np.float32(eps)))
    bc = ((VELOCITY, PRESSURE), (PERIODIC, PERIODIC), (PERIODIC, PERIODIC))
    fp, fu = _faces(P={(0, 1): P_out}, u={(0, 0): (u_in, 0.0, 0.0)})
    K6 = np.zeros((N, 6), np.float32)
    K6[:, 0:3] = K
    return _base("inflow_darcy", n, 1, 1, bc, ((OUTLET, OUTLET),) + ALL_PERIODIC[1:],
                 dict(tau=tau, face_P=fp, face_u=fu), _uniform(N, eps), K6.ravel(),
                 rho0=_uniform(N, 3.0 * eps * P_out), steps=steps, storage="fp64")


def with_species(prob: Problem, tau_D=(), C_in=(), C0=()) -> Problem:
    """The same problem with solute species 1, 2, ... added to species 0:
    relaxation times tau_D[s-1], inlet concentrations C_in[s-1] and initial
    fields C0[s-1] (each N values, default species 0's)."""
    S = 1 + len(tau_D)
    N = prob.N
    fields = [np.asarray(prob.C0, np.float32).reshape(-1)[:N]]
    for s in range(1, S):
        c = C0[s - 1] if s - 1 < len(C0) and C0[s - 1] is not None else fields[0]
        fields.append(np.asarray(c, np.float32).reshape(N))
    params = dict(prob.params, species=S,
                  species_tau_D=(0.0,) + tuple(float(t) for t in tau_D),
                  species_C_in=(0.0,) + tuple(float(c) for c in
                                              (list(C_in) + [0.0] * S)[:S - 1]))
    return prob.replace(params=params, C0=np.concatenate(fields))


def miscible_species(nx=128, ny=128, nz=128, seed=0, steps=5000, storage="fp32") -> Problem:
    """The miscible medium with three solute species sharing the flow:
    species 0 as there (tau_D 0.8, inlet C 1, it sets the viscosity), species
    1 faster (tau_D 1.2, inlet C 0.5), species 2 slower (tau_D 0.6, inlet C 0,
    initially 0.3 everywhere)."""
    base = miscible(nx, ny, nz, seed=seed, steps=steps, storage=storage)
    N = base.N
    return with_species(base, tau_D=(1.2, 0.6), C_in=(0.5, 0.0),
                        C0=(None, np.full(N, 0.3, np.float32))).replace(name="miscible_species")


def wood_density(xi, rho0=310.0, a=0.62, b=0.2, c=-0.2):
    """Eq. wooddensityfunc with the ring coordinate xi in [0, 1) of one year
    ring: rho = rho0 [1 + 2 a xi^b exp(-c xi)] (kg/m^3)."""
    xi = np.asarray(xi, dtype=np.float64)
    return rho0 * (1.0 + 2.0 * a * np.power(xi, b) * np.exp(-c * xi))


def wood_tensor(rho, rho_max=1500.0, scale=1.0):
    """Eq. Ktensor's principal permeabilities (radial, longitudinal,
    tangential) for the density rho: (rho_max/rho)^2 eps^(11/3) (8.2, 51470,
    0.82) times `scale` (the lattice unit), eps = 1 - rho/rho_max (Eq.
    epsilonfunction)."""
    rho = np.asarray(rho, dtype=np.float64)
    eps = 1.0 - rho / rho_max
    f = (rho_max / rho) ** 2 * eps ** (11.0 / 3.0) * scale
    return eps, np.stack([8.2 * f, 51470.0 * f, 0.82 * f], axis=-1)


def wood(nx=90, ny=90, nz=1, wood_depth=60, delta=30.0, angle=45.0, rho0=310.0, a=0.62,
         b=0.2, c=-0.2, rho_max=1500.0, K_scale=1e-3, P_ext=0.0441, nu_g=0.15,
         a_h=2.05e-9, alpha=2e-3, beta=1e-3, tau_D=0.8, steps=2000) -> Problem:
    """Penetration of an adhesive into wood (Section 5.5), read as miscible
    displacement: the adhesive (solute concentration C = 1) fills a reservoir
    above the wood (y >= wood_depth: eps = 1, negligible drag) and is pressed
    by P_ext into the wood sample (y < wood_depth), initially filled with
    solvent (C = 0). Year rings of width delta cells inclined by `angle` in
    the x-y plane: density from Eq. wooddensityfunc along the ring
    coordinate, porosity from Eq. epsilonfunction, permeability tensor of Eq.
    Ktensor in the ring frame (radial across the rings, longitudinal along
    z, tangential along the rings), rotated into the lattice (a full SPD K),
    scaled by K_scale to lattice units. Faces: top PRESSURE 1/3 + P_ext with
    solute INLET C = 1, bottom PRESSURE 1/(3 mean eps) with solute OUTLET, x and
    z periodic. Viscosity Eq. nuall (hardening)."""
    N = nx * ny * nz
    x, y, z = _grid(nx, ny, nz)
    th = np.deg2rad(angle)
    r_dir = np.array([np.cos(th), np.sin(th), 0.0])      # radial: across the rings
    t_dir = np.array([-np.sin(th), np.cos(th), 0.0])     # tangential: along the rings
    l_dir = np.array([0.0, 0.0, 1.0])                    # longitudinal: the fibres
    xi = np.mod((x * r_dir[0] + y * r_dir[1]) / delta, 1.0)
    rho_w = wood_density(xi, rho0, a, b, c)
    eps_w, kp = wood_tensor(rho_w, rho_max, K_scale)
    R = np.stack([r_dir, l_dir, t_dir], axis=1)           # columns: principal axes
    Kw = np.einsum("ij,nj,kj->nik", R, kp, R)
    in_wood = y < wood_depth
    eps = np.where(in_wood, eps_w, 1.0)
    K = np.where(in_wood[:, None, None], Kw, 1e6 * np.eye(3)[None])
    K6 = np.stack([K[:, 0, 0], K[:, 1, 1], K[:, 2, 2], K[:, 0, 1], K[:, 1, 2], K[:, 2, 0]], axis=1)
    C0 = np.where(in_wood, 0.0, 1.0)
    P_top = 1.0 / 3.0 + P_ext
    eps_bottom = float(np.mean(eps[y == 0]))
    P_bot = 1.0 / (3.0 * eps_bottom)
    rho0_field = np.where(in_wood, 3.0 * eps * P_bot, 3.0 * P_top).astype(np.float32)
    bc = ((PERIODIC, PERIODIC), (PRESSURE, PRESSURE), (PERIODIC, PERIODIC))
    sbc = ((PERIODIC, PERIODIC), (OUTLET, INLET), (PERIODIC, PERIODIC))
    fp, fu = _faces(P={(1, 0): P_bot, (1, 1): P_top})
    params = dict(visc_law=2, nu_g=nu_g, a=a_h, alpha=alpha, beta=beta, solute=1,
                  tau_D=tau_D, C_in=1.0, face_P=fp, face_u=fu)
    return _base("wood", nx, ny, nz, bc, sbc, params, eps.astype(np.float32),
                 K6.astype(np.float32).ravel(), rho0=rho0_field, C0=C0.astype(np.float32),
                 steps=steps, storage="fp64",
                 meta=dict(wood_depth=wood_depth, delta=delta, angle=angle, rho_max=rho_max))


def _random_rotations(nblocks, seed):
    """Haar-random rotation matrices from unit quaternions of 4 normals."""
    rng = _rng(seed)
    qv = rng.standard_normal((nblocks, 4))
    qv /= np.linalg.norm(qv, axis=1, keepdims=True)
    w, x, y, z = qv.T
    R = np.empty((nblocks, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def precision(nx=256, ny=256, nz=256, seed=0, rot_seed=4, block=32, steps=10000,
              storage="fp16") -> Problem:
    """The miscible medium with a full SPD permeability per cell:
    K = R_b diag(K_xx, K_xx, 100 K_xx) R_b^T with one Haar-random rotation
    R_b per block^3 block of cells (seeded by rot_seed)."""
    base = miscible(nx, ny, nz, seed=seed, steps=steps, storage=storage)
    N = base.N
    kxx = base.K6.reshape(N, 6)[:, 0].astype(np.float64)
    x, y, z = _grid(nx, ny, nz)
    bx, by, bz = -(-nx // block), -(-ny // block), -(-nz // block)
    R = _random_rotations(bx * by * bz, rot_seed)
    b = (x // block) + bx * ((y // block) + by * (z // block))
    Rb = R[b]                                           # [N, 3, 3]
    d = np.stack([kxx, kxx, 100.0 * kxx], axis=1)       # [N, 3]
    K = np.einsum("nij,nj,nkj->nik", Rb, d, Rb)
    K6 = np.stack([K[:, 0, 0], K[:, 1, 1], K[:, 2, 2], K[:, 0, 1], K[:, 1, 2], K[:, 2, 0]],
                  axis=1)
    return base.replace(name="precision", K6=K6.astype(np.float32).ravel(),
                        meta=dict(seed=seed, rot_seed=rot_seed, block=block))


def drop(nx=192, ny=192, nz=128, R=24.0, gap=40.0, seed=0, steps=8000, A=1e-3,
         wall_rho=0.6, tau=0.7, u_drop=0.02, perturb=0.01) -> Problem:
    """Free-surface liquid drop (density 1) above a solid bottom layer.

    wall_rho 0.6: a hydrophobic wall of about 120 degrees (a 2D drop relaxed
    from a half disc settles at 119 degrees in the oracle; from flatter or
    rounder starting caps at 98 or 132 degrees: the wetting reading has
    contact-angle hysteresis; tests/golden/contact_angle.py).

    The solid layer is z = 0 (its face towards the liquid lies at z = 0.5 in
    cell-centre coordinates); the drop's lowest point is `gap` cells above that
    face, so its centre is at z = 0.5 + gap + R. The top face is a bounce-back
    wall; x and y are periodic. Liquid cells: centre within R of the drop
    centre; interface cells: every other cell with a liquid D3Q19 neighbour
    (fill 0.5); all others empty. Initial velocity (0, 0, -u_drop) in the drop.
    Populations are scaled by seeded factors 1 + perturb*U(-1, 1).
    """
    rng = _rng(seed)
    N = nx * ny * nz
    x, y, z = _grid(nx, ny, nz)
    cx, cy, cz = (nx - 1) / 2.0, (ny - 1) / 2.0, 0.5 + gap + R
    inside = (x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2 <= R * R
    solid = (z == 0).astype(np.uint8)
    liquid = inside & (solid == 0)
    lq = liquid.reshape(nz, ny, nx)
    near = np.zeros_like(lq)
    for dx, dy, dz in [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)
                       if 0 < a * a + b * b + c * c <= 2]:
        sh = np.roll(lq, shift=(dz, dy, dx), axis=(0, 1, 2))
        if dz == 1:
            sh[0] = False
        if dz == -1:
            sh[-1] = False
        near |= sh
    near = near.ravel()
    ctype = np.full(N, EMPTY, np.uint8)
    ctype[near] = INTERFACE
    ctype[liquid] = LIQUID
    ctype[solid == 1] = EMPTY
    lam = np.where(ctype == LIQUID, 1.0, np.where(ctype == INTERFACE, 0.5, 0.0))
    u0 = np.zeros((N, 3), np.float32)
    u0[ctype != EMPTY, 2] = -u_drop
    bc = ((PERIODIC, PERIODIC), (PERIODIC, PERIODIC), (WALL, WALL))
    params = dict(tau=tau, A=A, wall_rho=wall_rho, free_surface=1)
    f_scale = (1.0 + perturb * rng.uniform(-1.0, 1.0, Q * N)).astype(np.float32) \
        if perturb else None
    return _base("drop", nx, ny, nz, bc, bc, params, _uniform(N, 1.0), None, solid=solid,
                 u0=u0.ravel(), cell_type=ctype, lambda0=lam.astype(np.float32),
                 f_scale=f_scale, steps=steps, meta=dict(seed=seed, R=R, gap=gap))


def requests(n=256, rate=50.0, seed=5, sides=(32, 48, 64, 96, 128, 160),
             steps_range=(2000, 20000)):
    """Serving stream: Poisson arrivals (exponential gaps), cubic-ish domains
    with side from `sides` and z-aspect U(1, 2), per-request seed = id."""
    rng = _rng(seed)
    gaps = rng.exponential(1.0 / rate, n)
    t = np.cumsum(gaps)
    out = []
    for i in range(n):
        s = int(rng.choice(sides))
        nz = int(round(s * rng.uniform(1.0, 2.0)))
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        out.append(dict(id=i, arrival=float(t[i]), nx=s, ny=s, nz=nz, steps=steps, seed=i))
    return out


def request_problem(req, storage="fp32") -> Problem:
    """The medium of one served request: the miscible family at its size."""
    p = miscible(req["nx"], req["ny"], req["nz"], seed=req["seed"], steps=req["steps"],
                 storage=storage)
    return p.replace(name=f"request{req['id']}")


# --------------------------------------------------------------------------
# Validation problems for the oracle pins
# --------------------------------------------------------------------------

def brinkman(nz=64, K=16.0, eps=0.6, tau=0.8, G=1e-6, nxy=1, steps=0) -> Problem:
    """Generalised Poiseuille (Brinkman) channel: walls at both z ends,
    periodic in x, y, body force G along x, isotropic K (Section 5.1)."""
    N = nxy * nxy * nz
    bc = ((PERIODIC, PERIODIC), (PERIODIC, PERIODIC), (WALL, WALL))
    return _base("brinkman", nxy, nxy, nz, bc, bc, dict(tau=tau, G=(G, 0.0, 0.0)),
                 _uniform(N, eps), _iso_K6(N, K), steps=steps, storage="fp64")


def aniso_channel(direction=0, n=70, eps=0.3, tau=0.6, G=0.1, Kxx=1e-3, Kyy=1e-5,
                  Kzz=1e-3, steps=300) -> Problem:
    """Section 5.2: diagonal K = diag(Kxx, Kyy, Kzz), flow along x with walls
    at the y ends (direction 0) or along y with walls at the x ends (1)."""
    N = n * n
    K6 = np.zeros((N, 6), np.float32)
    K6[:, 0], K6[:, 1], K6[:, 2] = Kxx, Kyy, Kzz
    if direction == 0:
        bc = ((PERIODIC, PERIODIC), (WALL, WALL), (PERIODIC, PERIODIC))
        g = (G, 0.0, 0.0)
    else:
        bc = ((WALL, WALL), (PERIODIC, PERIODIC), (PERIODIC, PERIODIC))
        g = (0.0, G, 0.0)
    return _base("aniso_channel", n, n, 1, bc, bc, dict(tau=tau, G=g), _uniform(N, eps),
                 K6.ravel(), steps=steps, storage="fp64")


def gaussian_pulse(nx=64, ny=1, nz=1, sigma0=4.0, tau_D=0.8, u=(0.0, 0.0, 0.0),
                   amplitude=1.0, base=0.0) -> Problem:
    """Solute pulse C0 = base + amplitude*exp(-r^2/(2 sigma0^2)) about the
    domain centre, eps = 1, no permeability, periodic, uniform velocity u."""
    N = nx * ny * nz
    x, y, z = _grid(nx, ny, nz)
    r2 = np.zeros(N)
    for c, n in ((x, nx), (y, ny), (z, nz)):
        if n > 1:
            r2 = r2 + (c - (n - 1) / 2.0) ** 2
    C0 = base + amplitude * np.exp(-r2 / (2 * sigma0 ** 2))
    u0 = np.tile(np.asarray(u, np.float32), N)
    params = dict(tau=0.8, solute=1, tau_D=tau_D)
    return _base("gaussian_pulse", nx, ny, nz, ALL_PERIODIC, ALL_PERIODIC, params,
                 _uniform(N, 1.0), None, u0=u0, C0=C0.astype(np.float32), storage="fp64")


def eps_bands(nx=32, ny=4, nz=4, C=0.5, tau_D=0.8, smooth=True) -> Problem:
    """Porosity varying along x, fluid at rest, uniform solute concentration,
    periodic. smooth: eps = 0.6 + 0.25 sin(2 pi x / nx); otherwise bands
    0.35 / 0.85 of period 16."""
    N = nx * ny * nz
    x, _, _ = _grid(nx, ny, nz)
    if smooth:
        eps = 0.6 + 0.25 * np.sin(2 * np.pi * x / nx)
    else:
        eps = np.where((x % 16) < 8, 0.35, 0.85)
    params = dict(tau=0.8, solute=1, tau_D=tau_D)
    return _base("eps_bands", nx, ny, nz, ALL_PERIODIC, ALL_PERIODIC, params,
                 eps.astype(np.float32), None, C0=_uniform(N, C), storage="fp64")


def random_medium(nx=8, ny=6, nz=5, seed=1, solid_frac=0.1, walls=True, solute=True,
                  inlet=True, spd=True, visc_law=1, A=0.0, u_amp=0.02,
                  open_faces=False) -> Problem:
    """Small heterogeneous problem exercising every feature at once (random
    porosity, SPD K, solids, walls, inlet/outlet, random initial velocity).
    open_faces: fluid faces VELOCITY / PRESSURE along x and PRESSURE along z
    (solute INLET / OUTLET on both), walls along y."""
    rng = _rng(seed)
    N = nx * ny * nz
    eps = rng.uniform(0.3, 1.0, N)
    if open_faces:   # pressure faces hold 3 eps P: keep the porosity near one value
        eps = rng.uniform(0.85, 0.95, N)
    k = 10.0 ** rng.uniform(-3, 0, N)
    K6 = np.zeros((N, 6))
    K6[:, 0] = k * rng.uniform(0.5, 2, N)
    K6[:, 1] = k * rng.uniform(0.5, 2, N)
    K6[:, 2] = k * rng.uniform(0.5, 2, N)
    if spd:
        K6[:, 3] = 0.3 * k * rng.uniform(-1, 1, N)
        K6[:, 4] = 0.3 * k * rng.uniform(-1, 1, N)
        K6[:, 5] = 0.3 * k * rng.uniform(-1, 1, N)
    solid = (rng.uniform(0, 1, N) < solid_frac).astype(np.uint8)
    bc = [[PERIODIC, PERIODIC], [PERIODIC, PERIODIC], [PERIODIC, PERIODIC]]
    sbc = [[PERIODIC, PERIODIC], [PERIODIC, PERIODIC], [PERIODIC, PERIODIC]]
    if walls:
        bc[1] = [WALL, WALL]
        sbc[1] = [WALL, WALL]
    if inlet and solute:
        sbc[2] = [INLET, OUTLET]
    extra = {}
    if open_faces:
        bc[0] = [VELOCITY, PRESSURE]
        bc[2] = [PRESSURE, PRESSURE]
        sbc[0] = [INLET, OUTLET]
        sbc[2] = [INLET, OUTLET]
        P0 = 1.0 / (3.0 * 0.9)
        fp, fu = _faces(P={(0, 1): P0 * 0.998, (2, 0): P0 * 1.002, (2, 1): P0 * 0.999},
                        u={(0, 0): (2e-4, 0.004, -0.003)})
        extra = dict(face_P=fp, face_u=fu)
    params = dict(tau=0.9, visc_law=visc_law if solute else 0, tau0=0.7, tau1=1.3,
                  nu_g=0.1, a=0.05, alpha=0.01, beta=0.5,
                  G=(2e-4, -1e-4, 3e-4), solute=int(solute), tau_D=0.75, C_in=1.0,
                  A=A, wall_rho=0.3, **extra)
    rho0 = (1.0 + 0.01 * rng.uniform(-1, 1, N)).astype(np.float32)
    u0 = (u_amp * rng.uniform(-1, 1, 3 * N)).astype(np.float32)
    C0 = rng.uniform(0, 1, N).astype(np.float32) if solute else None
    return _base("random_medium", nx, ny, nz, tuple(map(tuple, bc)), tuple(map(tuple, sbc)),
                 params, eps.astype(np.float32), K6.astype(np.float32).ravel(), solid=solid,
                 rho0=rho0, u0=u0, C0=C0, storage="fp64", meta=dict(seed=seed))


def thin_drop(n=64, R=10.0, A=1e-3, tau=0.7, wall_rho=0.0, shape="disc") -> Problem:
    """2D-thin (nz = 1, periodic) free-surface liquid patch in gas: a disc of
    radius R, or a square of side 2R, centred; no walls, no body force."""
    N = n * n
    x, y, _ = _grid(n, n, 1)
    c = (n - 1) / 2.0
    if shape == "disc":
        liquid = (x - c) ** 2 + (y - c) ** 2 <= R * R
    else:
        liquid = (np.abs(x - c) <= R) & (np.abs(y - c) <= R)
    lq = liquid.reshape(n, n)
    near = np.zeros_like(lq)
    for dx, dy in [(a, b) for a in (-1, 0, 1) for b in (-1, 0, 1) if (a, b) != (0, 0)]:
        near |= np.roll(lq, shift=(dy, dx), axis=(0, 1))
    ctype = np.full(N, EMPTY, np.uint8)
    ctype[near.ravel()] = INTERFACE
    ctype[liquid] = LIQUID
    lam = np.where(ctype == LIQUID, 1.0, np.where(ctype == INTERFACE, 0.5, 0.0))
    params = dict(tau=tau, A=A, wall_rho=wall_rho, free_surface=1)
    return _base("thin_drop", n, n, 1, ALL_PERIODIC, ALL_PERIODIC, params, _uniform(N, 1.0),
                 None, cell_type=ctype, lambda0=lam.astype(np.float32), storage="fp64",
                 meta=dict(R=R, shape=shape))


def crop(p: Problem, x0, y0, z0, nx, ny, nz) -> Problem:
    """A box cut out of a problem, run as its own problem with the same face
    kinds (static and initial fields sliced; perturbation factors dropped)."""
    sl = (slice(z0, z0 + nz), slice(y0, y0 + ny), slice(x0, x0 + nx))

    def cut(a, k=1):
        if a is None:
            return None
        if k == 1:
            return np.ascontiguousarray(a.reshape(p.shape)[sl]).ravel()
        return np.ascontiguousarray(a.reshape(p.shape + (k,))[sl]).ravel()

    return p.replace(name=p.name + "_crop", nx=nx, ny=ny, nz=nz, eps=cut(p.eps),
                     K6=cut(p.K6, 6), solid=cut(p.solid), rho0=cut(p.rho0), u0=cut(p.u0, 3),
                     C0=cut(p.C0), cell_type=cut(p.cell_type), lambda0=cut(p.lambda0),
                     f_scale=None)
