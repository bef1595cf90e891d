"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function include/lb.h declares, and rejects invalid requests before
touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_0912_4230_gb300 import build as lib_build
from paper_0912_4230_gb300 import lb, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    lib_build.build()
    return lb.load()


def declared():
    src = open(os.path.join(ROOT, "include", "lb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lb_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = declared()
    assert len(names) >= 14
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(lb.EXPORTS)


def test_struct_layouts_match_header():
    # lb_domain: 3 + 6 + 6 int32; lb_params: doubles and int32 in header order
    assert lb.lb_domain.bc.offset == 12 and lb.lb_domain.sbc.offset == 36
    src = open(os.path.join(ROOT, "include", "lb.h")).read()
    body = src[src.index("typedef struct {\n  double tau;") + len("typedef struct {"):src.index("} lb_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        names += [v.strip().split("[")[0] for v in decl.split(None, 1)[1].split(",")]
    assert names == [f[0] for f in lb.lb_params._fields_]


def _create(prob, **over):
    dom = lb.make_domain(prob)
    prm = lb.make_params(prob)
    for k, v in over.items():
        if k.startswith("dom_"):
            setattr(dom, k[4:], v)
        else:
            setattr(prm, k, v)
    return lb.lb_create(dom, prob.eps, prob.K6, prob.solid, prm)


def test_open_faces_refuse_free_surface_and_surface_tension(L):
    for extra in (dict(A=1e-3), dict(free_surface=1)):
        prob = W.random_medium(4, 4, 4, seed=0, open_faces=True, solute=False)
        prob = prob.replace(K6=None)
        with pytest.raises(lb.LbError) as e:
            _create(prob, **extra)
        assert e.value.code == lb.LB_EUNSUPPORTED


@pytest.mark.parametrize("over,code", [
    (dict(forchheimer=-0.5), lb.LB_EINVAL),
    (dict(visc_law=0, tau=0.5), lb.LB_EINVAL),
    (dict(tau0=0.5), lb.LB_EINVAL),
    (dict(solute=0), lb.LB_EINVAL),
    (dict(visc_law=3), lb.LB_EINVAL),
    (dict(tau_D=0.4), lb.LB_EINVAL),
    (dict(storage=9), lb.LB_EINVAL),
    (dict(check_every=-1), lb.LB_EINVAL),
    (dict(free_surface=1), lb.LB_EUNSUPPORTED),
    (dict(dom_nx=0), lb.LB_EINVAL),
])
def test_invalid_requests_are_rejected_on_the_host(L, over, code):
    prob = W.random_medium(4, 4, 4, seed=0)
    with pytest.raises(lb.LbError) as e:
        _create(prob, **over)
    assert e.value.code == code
    assert lb.lb_last_error(None)


def test_invalid_face_kinds_rejected(L):
    prob = W.random_medium(4, 4, 4, seed=0)
    dom = lb.make_domain(prob)
    dom.bc[0][0] = W.WALL       # one side periodic, the other a wall
    dom.bc[0][1] = W.PERIODIC
    with pytest.raises(lb.LbError) as e:
        lb.lb_create(dom, prob.eps, prob.K6, prob.solid, lb.make_params(prob))
    assert e.value.code == lb.LB_EINVAL
    dom = lb.make_domain(prob)
    dom.bc[2][0] = dom.bc[2][1] = W.INLET  # fluid faces cannot be inlets
    with pytest.raises(lb.LbError):
        lb.lb_create(dom, prob.eps, prob.K6, prob.solid, lb.make_params(prob))


def test_null_contexts_and_batches_are_refused(L):
    """Calls on a NULL context return LB_EINVAL without touching a GPU."""
    vp = ctypes.c_void_p
    assert L.lb_set_graphs(None, 1) == lb.LB_EINVAL
    assert L.lb_debug_graphs(None) == lb.LB_EINVAL
    assert L.lb_step(None, 1) == lb.LB_EINVAL
    assert L.lb_step_batch(None, 1, 1) == lb.LB_EINVAL
    arr = (vp * 1)(None)
    assert L.lb_step_batch(arr, 0, 1) == lb.LB_EINVAL      # no lattices
    with pytest.raises(lb.LbError) as e:                     # the same through the binding
        lb.lb_step_batch([], 1)
    assert e.value.code == lb.LB_EINVAL
    assert L.lb_arena_stats(None, None, None, None, None) == lb.LB_EINVAL
    assert L.lb_arena_alloc(None, 256) is None
    out = vp(1)
    assert L.lb_arena_create(None, 16, ctypes.byref(out)) == lb.LB_EINVAL   # below one block
    assert out.value is None


def test_array_arguments_must_match_the_declared_element_type():
    """The binding passes raw pointers, so it refuses strided views and
    element types other than the declared one before the library sees them."""
    torch = pytest.importorskip("torch")
    a = np.zeros((4, 3), np.float32)
    assert lb._ptr(None, np.float32) is None
    assert lb._ptr(a, np.float32).value == a.ctypes.data
    assert lb._ptr(np.zeros(3, bool), np.uint8) is not None        # 0/1 bytes
    with pytest.raises(ValueError):
        lb._ptr(a.T, np.float32)
    with pytest.raises(ValueError):
        lb._ptr(a[:, 0], np.float32)
    with pytest.raises(TypeError):
        lb._ptr(a.astype(np.float64), np.float32)
    with pytest.raises(TypeError):
        lb._ptr([0.0, 1.0], np.float32)
    t = torch.zeros(4, 3, dtype=torch.float32)
    assert lb._ptr(t, np.float32).value == t.data_ptr()
    assert lb._ptr(torch.zeros(3, dtype=torch.bool), np.uint8) is not None
    with pytest.raises(ValueError):
        lb._ptr(t.t(), np.float32)
    with pytest.raises(TypeError):
        lb._ptr(t.double(), np.float32)
    # the wrappers check before any library call: a wrong type never reaches it
    with pytest.raises(TypeError):
        lb.lb_fields(None, np.zeros(4, np.float64))
    with pytest.raises(TypeError):
        lb.lb_set_populations(None, np.zeros(19, np.float32))


def test_allocator_hooks_install_reset_and_stay_referenced(L):
    """Hooks are installed and reset without a GPU; a half-set pair is
    refused; the binding keeps every installed pair alive, since a context
    created under it calls its release from lb_destroy later."""
    n0 = len(lb._allocator_refs)
    lb.lb_set_allocator(lambda n: 0, lambda p: None)
    keep = lb._allocator_refs[-1]
    assert L.lb_set_allocator(L._ALLOC(0), keep[1], None) == lb.LB_EINVAL
    lb.lb_set_allocator(None)
    assert len(lb._allocator_refs) == n0 + 1 and lb._allocator_refs[-1] is keep
