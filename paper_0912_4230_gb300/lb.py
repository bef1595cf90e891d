"""ctypes binding of the CUDA library (C ABI in ``include/lb.h``).

Argument marshalling only: every step of the lattice-Boltzmann update runs in
the library's CUDA kernels. The functions keep the C names (``lb_create``,
``lb_step``, ``lb_fields`` ...); :class:`Lattice` wraps one context for a
:class:`~paper_0912_4230_gb300.workloads.Problem`.

Array arguments may be numpy arrays (host memory) or torch CUDA tensors
(device memory); both are passed as raw pointers. There is no CPU fallback:
if the shared library is missing or cannot be loaded this module raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_int32, c_int64, c_size_t, c_void_p

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "liblbgb.so")

Q = 19
LB_OK, LB_EINVAL, LB_ENOMEM, LB_ECUDA, LB_ENONFINITE, LB_ETIMEOUT, LB_EUNSUPPORTED = \
    0, -1, -2, -3, -4, -5, -6
PERIODIC, WALL, INLET, OUTLET, PRESSURE, VELOCITY = 0, 1, 2, 3, 4, 5
STORE = {"fp32": 0, "fp64": 1, "fp16": 2, "bf16": 3}

EXPORTS = ["lb_create", "lb_set_stream", "lb_init", "lb_set_populations", "lb_get_populations",
           "lb_step", "lb_fields", "lb_reduce", "lb_debug_neighbors", "lb_free_surface_state",
           "lb_sync", "lb_time", "lb_last_error", "lb_destroy", "lb_set_allocator",
           "lb_totals_noalloc", "lb_step_batch", "lb_autotune", "lb_debug_wait_timeout",
           "lb_species_state", "lb_set_graphs", "lb_debug_graphs", "lb_arena_create",
           "lb_arena_destroy", "lb_arena_use", "lb_arena_alloc", "lb_arena_free", "lb_arena_stats",
           "lb_bytes_required"]


class LbError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"lb error {code}: {msg}")
        self.code = code


class lb_domain(ctypes.Structure):
    _fields_ = [("nx", c_int32), ("ny", c_int32), ("nz", c_int32),
                ("bc", (c_int32 * 2) * 3), ("sbc", (c_int32 * 2) * 3)]


class lb_params(ctypes.Structure):
    _fields_ = [("tau", c_double), ("visc_law", c_int32), ("tau0", c_double), ("tau1", c_double),
                ("nu_g", c_double), ("a", c_double), ("alpha", c_double), ("beta", c_double),
                ("G", c_double * 3), ("A", c_double), ("wall_rho", c_double),
                ("forchheimer", c_double), ("solute", c_int32), ("tau_D", c_double),
                ("C_in", c_double), ("free_surface", c_int32), ("storage", c_int32),
                ("check_every", c_int32), ("kernel", c_int32),
                ("face_P", (c_double * 2) * 3), ("face_u", ((c_double * 3) * 2) * 3),
                ("species", c_int32), ("species_tau_D", c_double * 8),
                ("species_C_in", c_double * 8)]


_lib = None


def load() -> ctypes.CDLL:
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
    L = ctypes.CDLL(LIB_PATH)
    vp = c_void_p
    L.lb_create.argtypes = [POINTER(lb_domain), vp, vp, vp, POINTER(lb_params), POINTER(vp)]
    L.lb_set_stream.argtypes = [vp, vp]
    L.lb_init.argtypes = [vp] * 7
    L.lb_set_populations.argtypes = [vp, vp, vp]
    L.lb_get_populations.argtypes = [vp, vp, vp]
    L.lb_step.argtypes = [vp, c_int64]
    L.lb_fields.argtypes = [vp] * 5
    L.lb_reduce.argtypes = [vp] * 5
    L.lb_debug_neighbors.argtypes = [vp, c_int32, vp]
    L.lb_debug_wait_timeout.argtypes = [vp, c_int64]
    L.lb_set_graphs.argtypes = [vp, c_int32]
    L.lb_debug_graphs.argtypes = [vp]
    L.lb_species_state.argtypes = [vp, c_int32, vp, vp, vp]
    L.lb_free_surface_state.argtypes = [vp, vp, vp]
    L.lb_sync.argtypes = [vp]
    L.lb_time.argtypes = [vp]
    L.lb_time.restype = c_int64
    L.lb_last_error.argtypes = [vp]
    L.lb_last_error.restype = ctypes.c_char_p
    L.lb_destroy.argtypes = [vp]
    L.lb_destroy.restype = None
    ALLOC = ctypes.CFUNCTYPE(vp, c_size_t, vp)
    FREE = ctypes.CFUNCTYPE(None, vp, vp)
    L.lb_set_allocator.argtypes = [ALLOC, FREE, vp]
    L._ALLOC, L._FREE = ALLOC, FREE
    L.lb_totals_noalloc.argtypes = [vp, vp, vp, c_int64, vp, vp]
    L.lb_step_batch.argtypes = [vp, c_int32, c_int64]
    L.lb_autotune.argtypes = [vp, c_int32, vp]
    L.lb_arena_create.argtypes = [vp, c_size_t, POINTER(vp)]
    L.lb_arena_destroy.argtypes = [vp]
    L.lb_arena_destroy.restype = None
    L.lb_arena_use.argtypes = [vp]
    L.lb_arena_alloc.argtypes = [vp, c_size_t]
    L.lb_arena_alloc.restype = vp
    L.lb_arena_free.argtypes = [vp, vp]
    L.lb_arena_free.restype = None
    L.lb_arena_stats.argtypes = [vp] * 5
    L.lb_bytes_required.argtypes = [POINTER(lb_domain), POINTER(lb_params), c_int32, c_int32,
                                    POINTER(c_size_t)]
    _lib = L
    return L


_F32, _F64, _U8, _I32 = np.float32, np.float64, np.uint8, np.int32


def _ptr(a, dtype=None):
    """Raw pointer of a numpy array or torch tensor (None passes NULL).

    The library reads and writes each array as one dense run of its element
    type, so a strided view, or an element type other than the one the C
    declaration names (``dtype``), is refused here instead of being read as
    something else; a bool array stands for uint8 (0/1 bytes)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("lb: tensor arguments must be contiguous")
        if dtype is not None:
            name = str(a.dtype).replace("torch.", "")
            if name != np.dtype(dtype).name and not (dtype is _U8 and name == "bool"):
                raise TypeError(f"lb: tensor of {name} where the library takes {np.dtype(dtype).name}")
        return c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray):
        raise TypeError(f"lb: array argument expected, got {type(a).__name__}")
    if not a.flags.c_contiguous:
        raise ValueError("lb: array arguments must be C-contiguous")
    if dtype is not None and a.dtype != dtype and not (dtype is _U8 and a.dtype == np.bool_):
        raise TypeError(f"lb: array of {a.dtype} where the library takes {np.dtype(dtype).name}")
    return a.ctypes.data_as(c_void_p)


def _check(rc: int, ctx=None):
    if rc != LB_OK:
        msg = load().lb_last_error(ctx).decode(errors="replace")
        raise LbError(rc, msg)


# ---------------------------------------------------------------- C names

def lb_create(domain: lb_domain, porosity, K6, solid, params: lb_params):
    ctx = c_void_p()
    rc = load().lb_create(ctypes.byref(domain), _ptr(porosity, _F32), _ptr(K6, _F32), _ptr(solid, _U8),
                          ctypes.byref(params), ctypes.byref(ctx))
    _check(rc, None)
    return ctx


def lb_set_stream(ctx, stream_handle: int):
    """ctx None: stream of later lb_create calls on this thread."""
    _check(load().lb_set_stream(ctx, c_void_p(stream_handle)), ctx)


def lb_init(ctx, rho0, u0, C0=None, cell_type=None, lambda0=None, f_scale=None):
    _check(load().lb_init(ctx, _ptr(rho0, _F32), _ptr(u0, _F32), _ptr(C0, _F32),
                          _ptr(cell_type, _U8), _ptr(lambda0, _F32), _ptr(f_scale, _F32)), ctx)


def lb_set_populations(ctx, f=None, h=None):
    _check(load().lb_set_populations(ctx, _ptr(f, _F64), _ptr(h, _F64)), ctx)


def lb_get_populations(ctx, f=None, h=None):
    _check(load().lb_get_populations(ctx, _ptr(f, _F64), _ptr(h, _F64)), ctx)


def lb_step(ctx, n: int):
    _check(load().lb_step(ctx, int(n)), ctx)


def lb_autotune(ctx, reps: int = 5) -> int:
    """Time the candidate kernels and launch shapes and keep the fastest;
    returns the choice (per-cell kernel: the row width; row-staged kernel:
    1000 + the row width; 256 = row-pipelined; 0 = not tuned)."""
    ch = c_int32()
    _check(load().lb_autotune(ctx, int(reps), ctypes.byref(ch)), ctx)
    return ch.value


def lb_step_batch(ctxs, n_steps: int):
    """Advance several contexts by n_steps in one batched launch per step."""
    arr = (c_void_p * len(ctxs))(*[c.value if isinstance(c, c_void_p) else c for c in ctxs])
    _check(load().lb_step_batch(arr, len(ctxs), int(n_steps)), ctxs[0] if len(ctxs) else None)


def lb_fields(ctx, rho=None, u=None, C=None, nu=None):
    _check(load().lb_fields(ctx, _ptr(rho, _F32), _ptr(u, _F32), _ptr(C, _F32), _ptr(nu, _F32)), ctx)


def lb_reduce(ctx):
    out = [c_double() for _ in range(4)]
    _check(load().lb_reduce(ctx, *[ctypes.byref(o) for o in out]), ctx)
    return np.array([o.value for o in out])


def lb_debug_neighbors(ctx, lattice: int, src):
    _check(load().lb_debug_neighbors(ctx, int(lattice), _ptr(src, _I32)), ctx)


def lb_debug_wait_timeout(ctx, limit_ns: int):
    _check(load().lb_debug_wait_timeout(ctx, int(limit_ns)), ctx)


def lb_set_graphs(ctx, enable: bool):
    _check(load().lb_set_graphs(ctx, 1 if enable else 0), ctx)


def lb_debug_graphs(ctx) -> int:
    rc = load().lb_debug_graphs(ctx)
    if rc < 0:
        _check(rc, ctx)
    return rc


def lb_species_state(ctx, s: int, C=None, totals=None, h=None):
    _check(load().lb_species_state(ctx, int(s), _ptr(C, _F32), _ptr(totals, _F64), _ptr(h, _F64)), ctx)


def lb_free_surface_state(ctx, cell_type=None, mass=None):
    _check(load().lb_free_surface_state(ctx, _ptr(cell_type, _U8), _ptr(mass, _F64)), ctx)


def lb_sync(ctx):
    _check(load().lb_sync(ctx), ctx)


def lb_time(ctx) -> int:
    return load().lb_time(ctx)


def lb_last_error(ctx=None) -> str:
    return load().lb_last_error(ctx).decode(errors="replace")


def lb_destroy(ctx):
    load().lb_destroy(ctx)


def lb_bytes_required(domain: lb_domain, params: lb_params, k_rows: int, f_scale: bool = False) -> int:
    """Device bytes one lattice takes, from the library's own allocation
    layout (k_rows: 0 without K, 3 diagonal, 6 full tensor or unknown)."""
    out = c_size_t()
    _check(load().lb_bytes_required(ctypes.byref(domain), ctypes.byref(params), int(k_rows),
                                    1 if f_scale else 0, ctypes.byref(out)), None)
    return out.value


def lb_totals_noalloc(f, h, solid, n_cells: int, out, stream_handle: int = 0):
    """FP64 (mass, solute) of caller-owned device arrays without any device
    allocation (see include/lb.h); out receives 2 doubles."""
    rc = load().lb_totals_noalloc(_ptr(f, _F32), _ptr(h, _F32), _ptr(solid, _U8), int(n_cells),
                                  _ptr(out, _F64), c_void_p(stream_handle))
    _check(rc, None)


# every callback pair ever installed stays referenced: a context keeps the
# hooks it was created with and calls release from lb_destroy, possibly after
# another allocator (or none) has been installed
_allocator_refs = []


def lb_set_allocator(alloc=None, release=None):
    """Route device allocations through Python callables alloc(nbytes) -> int
    pointer and release(ptr); ``use_torch_allocator()`` installs torch's."""
    L = load()
    if alloc is None:
        _check(L.lb_set_allocator(L._ALLOC(0), L._FREE(0), None))
        return

    def _a(nbytes, _user):
        try:
            return alloc(int(nbytes)) or None
        except Exception:
            return None

    def _r(ptr, _user):
        release(ptr)

    refs = (L._ALLOC(_a), L._FREE(_r))
    _allocator_refs.append(refs)
    _check(L.lb_set_allocator(refs[0], refs[1], None))


def use_torch_allocator():
    """Allocate the library's device memory from torch's caching allocator."""
    import torch
    lb_set_allocator(lambda n: torch.cuda.caching_allocator_alloc(n),
                     lambda p: torch.cuda.caching_allocator_delete(p))


class Arena:
    """Packed lattice arena (lb_arena_*): one region of device memory
    (``base``, ``nbytes``; base None: the library allocates it) from which
    the lattices created while it is in use are sub-allocated."""

    def __init__(self, nbytes: int, base=None):
        out = c_void_p()
        rc = load().lb_arena_create(None if base is None else c_void_p(int(base)),
                                    c_size_t(int(nbytes)), ctypes.byref(out))
        if rc != LB_OK:
            raise LbError(rc, "lb_arena_create failed")
        self.ptr = out
        self.nbytes = int(nbytes)

    def use(self):
        _check(load().lb_arena_use(self.ptr))

    @staticmethod
    def use_none():
        _check(load().lb_arena_use(None))

    def alloc(self, nbytes: int):
        return load().lb_arena_alloc(self.ptr, c_size_t(int(nbytes)))

    def free(self, ptr):
        load().lb_arena_free(self.ptr, c_void_p(ptr))

    def stats(self) -> dict:
        v = [c_size_t() for _ in range(4)]
        _check(load().lb_arena_stats(self.ptr, *[ctypes.byref(x) for x in v]))
        return dict(used=v[0].value, largest_free=v[1].value, peak=v[2].value, blocks=v[3].value)

    def close(self):
        if self.ptr:
            load().lb_arena_destroy(self.ptr)
            self.ptr = None


# ---------------------------------------------------------------- convenience

def make_domain(prob) -> lb_domain:
    d = lb_domain()
    d.nx, d.ny, d.nz = prob.nx, prob.ny, prob.nz
    for a in range(3):
        for s in range(2):
            d.bc[a][s] = prob.bc[a][s]
            d.sbc[a][s] = prob.sbc[a][s]
    return d


KERNEL = {"auto": 0, "cell": 1, "rows": 2, "staged": 3}


def make_params(prob, storage=None, check_every=0, kernel="auto") -> lb_params:
    k = prob.params
    p = lb_params()
    p.tau = k.get("tau", 1.0)
    p.visc_law = k.get("visc_law", 0)
    p.tau0, p.tau1 = k.get("tau0", 1.0), k.get("tau1", 1.0)
    p.nu_g, p.a, p.alpha, p.beta = (k.get("nu_g", 0.0), k.get("a", 0.0), k.get("alpha", 0.0),
                                    k.get("beta", 0.0))
    for i in range(3):
        p.G[i] = k.get("G", (0.0, 0.0, 0.0))[i]
    p.A = k.get("A", 0.0)
    p.wall_rho = k.get("wall_rho", 0.0)
    fp = k.get("face_P", ((0.0, 0.0),) * 3)
    fu = k.get("face_u", (((0.0,) * 3,) * 2,) * 3)
    for ax in range(3):
        for side in range(2):
            p.face_P[ax][side] = fp[ax][side]
            for i in range(3):
                p.face_u[ax][side][i] = fu[ax][side][i]
    p.forchheimer = k.get("forchheimer", 0.0)
    p.species = int(k.get("species", 1 if k.get("solute") else 0))
    for s_, v in enumerate(k.get("species_tau_D", ())):
        p.species_tau_D[s_] = v
    for s_, v in enumerate(k.get("species_C_in", ())):
        p.species_C_in[s_] = v
    p.solute = int(k.get("solute", 0))
    p.tau_D = k.get("tau_D", 1.0)
    p.C_in = k.get("C_in", 0.0)
    p.free_surface = int(k.get("free_surface", 0))
    p.storage = STORE[storage or prob.storage]
    p.check_every = check_every
    p.kernel = KERNEL[kernel]
    return p


def _f32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float32)


class Lattice:
    """One library context built from a workload description."""

    def __init__(self, prob, storage=None, check_every=0, stream=None, init=True,
                 kernel="auto"):
        self.prob = prob
        self.N = prob.N
        self.solute = bool(prob.params.get("solute"))
        self.fs = bool(prob.params.get("free_surface"))
        self._dom = make_domain(prob)
        self._prm = make_params(prob, storage, check_every, kernel)
        self.ctx = lb_create(self._dom, _f32(prob.eps), _f32(prob.K6),
                             np.ascontiguousarray(prob.solid, np.uint8), self._prm)
        if stream is not None:
            lb_set_stream(self.ctx, stream)
        if init:
            self.init()

    def init(self, rho0=None, u0=None, C0=None):
        p = self.prob
        lb_init(self.ctx, _f32(p.rho0 if rho0 is None else rho0),
                _f32(p.u0 if u0 is None else u0),
                _f32(p.C0 if C0 is None else C0) if self.solute else None,
                None if p.cell_type is None else np.ascontiguousarray(p.cell_type, np.uint8),
                _f32(p.lambda0), _f32(p.f_scale))

    def step(self, n=1):
        lb_step(self.ctx, n)

    def set_graphs(self, enable: bool):
        lb_set_graphs(self.ctx, enable)

    @property
    def t(self):
        return lb_time(self.ctx)

    def fields(self):
        N = self.N
        rho, u = np.zeros(N, np.float32), np.zeros(3 * N, np.float32)
        C, nu = np.zeros(N, np.float32), np.zeros(N, np.float32)
        lb_fields(self.ctx, rho, u, C, nu)
        return rho, u.reshape(N, 3), C, nu

    def reduce(self):
        return lb_reduce(self.ctx)

    def species_state(self, s: int):
        """Species s: (C field, [solute total, inlet flux, outlet flux], h[19, N])."""
        N = self.N
        C, tot, h = np.zeros(N, np.float32), np.zeros(3), np.zeros(Q * N)
        lb_species_state(self.ctx, s, C, tot, h)
        return C, tot, h.reshape(Q, N)

    def populations(self):
        f = np.zeros(Q * self.N)
        h = np.zeros(Q * self.N) if self.solute else None
        lb_get_populations(self.ctx, f, h)
        return f.reshape(Q, self.N), (None if h is None else h.reshape(Q, self.N))

    def set_populations(self, f=None, h=None):
        lb_set_populations(self.ctx, None if f is None else np.ascontiguousarray(f, np.float64),
                           None if h is None else np.ascontiguousarray(h, np.float64))

    def neighbors(self, lattice=0):
        src = np.zeros(Q * self.N, np.int32)
        lb_debug_neighbors(self.ctx, lattice, src)
        return src.reshape(Q, self.N)

    def free_surface_state(self):
        t = np.zeros(self.N, np.uint8)
        m = np.zeros(self.N, np.float64)
        lb_free_surface_state(self.ctx, t, m)
        return t, m

    def sync(self):
        lb_sync(self.ctx)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            lb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
