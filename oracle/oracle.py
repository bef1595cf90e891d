"""ctypes wrapper of the FP64 CPU oracle (``lb_oracle.c``).

TEST INFRASTRUCTURE ONLY. The oracle is the plain, slow, cell-by-cell FP64
restatement of the lattice-Boltzmann scheme of Mendoza, Wittel and Herrmann
(arXiv:0912.4230, Sections 2-4). Only the tests, ``__graft_entry__.smoke()`` and
the benchmark's CPU-baseline leg may import this module. It shares no code with
the CUDA library and never calls it.

Parity status per function (pins live in ``tests/test_oracle_*.py``):
  velocity set, f^eq, forcing T_q, velocity solve, h^eq, viscosity laws,
  streaming/bounce-back (the exact discrete Poiseuille solution), the viscous
  and Darcy decay of a shear wave, inlet/outlet
  fluxes, colour gradient: pinned.
  free surface: pinned by exact mass conservation, free fall of a drop, and
  the closed interface layer (no liquid cell next to an empty one, no mass in
  empty cells, m - rho kept in cells that stay liquid); the conversion
  thresholds and the equal sharing of excess mass are readings the paper
  gives no value for. Wetting (wall_rho): parity unpinned (no printed angle).
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import sys
from ctypes import c_double, c_int32, c_int64, c_void_p, POINTER

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lb_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liblb_oracle.so")

Q = 19
PERIODIC, WALL, INLET, OUTLET = 0, 1, 2, 3
LIQUID, INTERFACE, EMPTY = 0, 1, 2


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("nx", c_int32), ("ny", c_int32), ("nz", c_int32),
        ("bc", (c_int32 * 2) * 3), ("sbc", (c_int32 * 2) * 3),
        ("tau", c_double), ("visc_law", c_int32),
        ("tau0", c_double), ("tau1", c_double),
        ("nu_g", c_double), ("a", c_double), ("alpha", c_double), ("beta", c_double),
        ("G", c_double * 3), ("A", c_double), ("wall_rho", c_double),
        ("solute", c_int32), ("tau_D", c_double), ("C_in", c_double),
        ("free_surface", c_int32), ("threads", c_int32),
        ("forchheimer", c_double),
        ("face_P", (c_double * 2) * 3), ("face_u", ((c_double * 3) * 2) * 3),
        ("species", c_int32), ("species_tau_D", c_double * 8), ("species_C_in", c_double * 8),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no intrinsics)."""
    os.makedirs(_BUILD, exist_ok=True)
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", "{out}", "-lm"]
    # rebuilt unless the hash of the sources and the command recorded beside
    # the library matches (file times are not trusted)
    h = hashlib.sha256(" ".join(cmd).encode())
    for p in (_SRC, os.path.join(_HERE, "lb_oracle.h")):
        with open(p, "rb") as fh:
            h.update(fh.read())
    digest, stamp = h.hexdigest(), _SO + ".sha256"
    if not force and os.path.exists(_SO) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read().strip() == digest:
                return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.run([tmp if a == "{out}" else a for a in cmd], check=True)
    os.replace(tmp, _SO)
    with open(stamp + f".{os.getpid()}.tmp", "w") as fh:
        fh.write(digest + "\n")
    os.replace(stamp + f".{os.getpid()}.tmp", stamp)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.orc_create.restype = c_void_p
        L.orc_create.argtypes = [POINTER(OrcParams), c_void_p, c_void_p, c_void_p]
        L.orc_init.argtypes = [c_void_p] + [c_void_p] * 6
        L.orc_set_populations.argtypes = [c_void_p, c_void_p, c_void_p]
        L.orc_get_populations.argtypes = [c_void_p, c_void_p, c_void_p]
        L.orc_step.argtypes = [c_void_p, c_int64]
        L.orc_fields.argtypes = [c_void_p] + [c_void_p] * 4
        L.orc_reduce.argtypes = [c_void_p, c_void_p]
        L.orc_species_state.argtypes = [c_void_p, c_int32, c_void_p, c_void_p, c_void_p]
        L.orc_neighbors.argtypes = [c_void_p, c_int32, c_void_p]
        L.orc_free_surface_state.argtypes = [c_void_p, c_void_p, c_void_p]
        L.orc_time.restype = c_int64
        L.orc_time.argtypes = [c_void_p]
        L.orc_destroy.argtypes = [c_void_p]
        L.orc_velocity_set.argtypes = [c_void_p, c_void_p, c_void_p]
        L.orc_feq.argtypes = [c_double, c_void_p, c_double, c_double, c_double, c_void_p, c_void_p]
        L.orc_forcing.argtypes = [c_double, c_double, c_double, c_void_p, c_void_p, c_void_p]
        L.orc_velocity_solve.argtypes = [c_void_p, c_double, c_double, c_void_p, c_void_p,
                                         c_double, c_void_p, c_void_p]
        L.orc_heq.argtypes = [c_double, c_double, c_void_p, c_void_p]
        L.orc_tau_of.restype = c_double
        L.orc_tau_of.argtypes = [POINTER(OrcParams), c_double, c_int64]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def make_params(prob, threads: int = 0) -> OrcParams:
    """Oracle parameter block from a workload description (``workloads.Problem``)."""
    p = OrcParams()
    p.nx, p.ny, p.nz = prob.nx, prob.ny, prob.nz
    for a in range(3):
        for s in range(2):
            p.bc[a][s] = prob.bc[a][s]
            p.sbc[a][s] = prob.sbc[a][s]
    k = prob.params
    p.tau = k.get("tau", 1.0)
    p.visc_law = k.get("visc_law", 0)
    p.tau0 = k.get("tau0", 1.0)
    p.tau1 = k.get("tau1", 1.0)
    p.nu_g = k.get("nu_g", 0.0)
    p.a = k.get("a", 0.0)
    p.alpha = k.get("alpha", 0.0)
    p.beta = k.get("beta", 0.0)
    for a in range(3):
        p.G[a] = k.get("G", (0.0, 0.0, 0.0))[a]
    p.A = k.get("A", 0.0)
    p.wall_rho = k.get("wall_rho", 0.0)
    p.solute = int(k.get("solute", 0))
    p.tau_D = k.get("tau_D", 1.0)
    p.C_in = k.get("C_in", 0.0)
    p.free_surface = int(k.get("free_surface", 0))
    p.threads = threads
    p.forchheimer = k.get("forchheimer", 0.0)
    p.species = int(k.get("species", 1 if k.get("solute") else 0))
    for s_, v in enumerate(k.get("species_tau_D", ())):
        p.species_tau_D[s_] = v
    for s_, v in enumerate(k.get("species_C_in", ())):
        p.species_C_in[s_] = v
    fp = k.get("face_P", ((0.0, 0.0),) * 3)
    fu = k.get("face_u", (((0.0,) * 3,) * 2,) * 3)
    for a in range(3):
        for s in range(2):
            p.face_P[a][s] = fp[a][s]
            for i in range(3):
                p.face_u[a][s][i] = fu[a][s][i]
    return p


# ---------------------------------------------------------------- single cell

def velocity_set():
    c = np.zeros(3 * Q, np.int32)
    w = np.zeros(Q, np.float64)
    opp = np.zeros(Q, np.int32)
    lib().orc_velocity_set(_ptr(c), _ptr(w), _ptr(opp))
    return c.reshape(Q, 3), w, opp


def feq(rho, u, eps, tau, A=0.0, F=(0.0, 0.0, 0.0)):
    out = np.zeros(Q)
    lib().orc_feq(rho, _ptr(_f64(u)), eps, tau, A, _ptr(_f64(F)), _ptr(out))
    return out


def forcing(rho, tau, eps, u, Fext):
    out = np.zeros(Q)
    lib().orc_forcing(rho, tau, eps, _ptr(_f64(u)), _ptr(_f64(Fext)), _ptr(out))
    return out


def velocity_solve(V, eps, nu, Kinv9, G, cF=0.0):
    Vp = np.zeros(3)
    Fe = np.zeros(3)
    kin = None if Kinv9 is None else _f64(np.asarray(Kinv9).reshape(9))
    lib().orc_velocity_solve(_ptr(_f64(V)), eps, nu, _ptr(kin), _ptr(_f64(G)), float(cF),
                             _ptr(Vp), _ptr(Fe))
    return Vp, Fe


def heq(eps, C, Vstar):
    out = np.zeros(Q)
    lib().orc_heq(eps, C, _ptr(_f64(Vstar)), _ptr(out))
    return out


def tau_of(prob, C, t):
    p = make_params(prob)
    return lib().orc_tau_of(ctypes.byref(p), C, t)


# ---------------------------------------------------------------- lattices

class Oracle:
    """An FP64 lattice built from a ``workloads.Problem``; runs on the host."""

    def __init__(self, prob, threads: int = 0):
        self.prob = prob
        self.N = prob.nx * prob.ny * prob.nz
        self._params = make_params(prob, threads)
        self._keep = [_f64(prob.eps), _f64(prob.K6),
                      np.ascontiguousarray(prob.solid, dtype=np.uint8)]
        h = lib().orc_create(ctypes.byref(self._params), _ptr(self._keep[0]),
                             _ptr(self._keep[1]), _ptr(self._keep[2]))
        if not h:
            raise ValueError("oracle rejected the problem description")
        self._h = h
        args = [_f64(prob.rho0), _f64(prob.u0), _f64(prob.C0),
                None if prob.cell_type is None else np.ascontiguousarray(prob.cell_type, np.uint8),
                _f64(prob.lambda0), _f64(prob.f_scale)]
        rc = lib().orc_init(self._h, *[_ptr(a) for a in args])
        if rc != 0:
            raise ValueError("oracle init rejected its inputs")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def step(self, n: int = 1):
        lib().orc_step(self._h, int(n))

    @property
    def t(self) -> int:
        return lib().orc_time(self._h)

    def fields(self):
        N = self.N
        rho, u, C, nu = np.zeros(N), np.zeros(3 * N), np.zeros(N), np.zeros(N)
        lib().orc_fields(self._h, _ptr(rho), _ptr(u), _ptr(C), _ptr(nu))
        return rho, u.reshape(N, 3), C, nu

    def reduce(self):
        out = np.zeros(4)
        lib().orc_reduce(self._h, _ptr(out))
        return out

    def species_state(self, s: int):
        """Species s: (C field, [solute total, inlet flux, outlet flux], h[19, N])."""
        N = self.N
        C, out, h = np.zeros(N), np.zeros(3), np.zeros(Q * N)
        if lib().orc_species_state(self._h, int(s), _ptr(C), _ptr(out), _ptr(h)) != 0:
            raise ValueError(f"no solute species {s}")
        return C, out, h.reshape(Q, N)

    def populations(self):
        f = np.zeros(Q * self.N)
        h = np.zeros(Q * self.N) if self.prob.params.get("solute") else None
        lib().orc_get_populations(self._h, _ptr(f), _ptr(h))
        return f.reshape(Q, self.N), (None if h is None else h.reshape(Q, self.N))

    def set_populations(self, f=None, h=None):
        lib().orc_set_populations(self._h, _ptr(_f64(f)), _ptr(_f64(h)))

    def neighbors(self, lattice: int = 0):
        src = np.zeros(Q * self.N, np.int32)
        lib().orc_neighbors(self._h, lattice, _ptr(src))
        return src.reshape(Q, self.N)

    def free_surface_state(self):
        t = np.zeros(self.N, np.uint8)
        m = np.zeros(self.N)
        lib().orc_free_surface_state(self._h, _ptr(t), _ptr(m))
        return t, m


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
