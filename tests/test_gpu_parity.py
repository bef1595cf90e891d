"""GPU (CUDA library through the C ABI) against the FP64 CPU oracle.

Tolerances: FP32 storage max|du| <= 1e-5 max|u|, max|drho| <= 1e-6,
max|dC| <= 1e-5, max|dnu| <= 3.4e-6 (nu = (tau0 + (tau1 - tau0) C - 1/2)/3
turns the C tolerance into 0.3e-5). FP64 storage: the populations agree to
1e-13 (absolute, values ~0.05); the exported fields are float32, so they
agree to float32 rounding (2^-24 relative, 1.2e-7 with margin). Index work
(pull sources, boundary classes) is bit-exact.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_0912_4230_gb300 import lb, workloads as W

pytestmark = pytest.mark.gpu

TOL = {
    "fp32": dict(u=1e-5, rho=1e-6, C=1e-5, nu=3.4e-6),
    "fp64": dict(u=1.2e-7, rho=1.2e-7, C=1.2e-7, nu=1.2e-7),
}


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def run_both(prob, steps, storage, threads=0, check_every=0):
    g = lb.Lattice(prob, storage=storage, check_every=check_every)
    g.step(steps)
    o = O.Oracle(prob, threads=threads)
    o.step(steps)
    return g, o


def compare(g, o, prob, storage, tol=None):
    tol = tol or TOL[storage]
    rho, u, C, nu = g.fields()
    r_rho, r_u, r_C, r_nu = o.fields()
    live = prob.solid == 0
    if prob.cell_type is not None:
        t, _ = o.free_surface_state()
        live = live & (t != W.EMPTY)
    umax = np.abs(r_u[live]).max()
    err = dict(
        u=np.abs(u[live] - r_u[live]).max() / umax if umax > 0 else np.abs(u[live]).max(),
        rho=np.abs(rho[live] - r_rho[live]).max(),
        C=np.abs(C[live] - r_C[live]).max(),
        nu=np.abs(nu[live] - r_nu[live]).max(),
    )
    for k in ("u", "rho", "C", "nu"):
        assert err[k] <= tol[k], (k, err)
    return err


@pytest.mark.parametrize("dims", [(3, 4, 5), (4, 3, 5), (1, 2, 3), (37, 5, 3)])
@pytest.mark.parametrize("seed", [0, 1])
def test_neighbor_table_bit_exact(dims, seed):
    prob = W.random_medium(*dims, seed=seed, solid_frac=0.2)
    g = lb.Lattice(prob, storage="fp32")
    o = O.Oracle(prob)
    for lattice in (0, 1):
        assert np.array_equal(g.neighbors(lattice), o.neighbors(lattice))


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
@pytest.mark.parametrize("law", [1, 2])
@pytest.mark.parametrize("A", [0.0, 1e-3])
def test_random_medium_all_features(storage, law, A):
    """Every feature at once: random porosity, full SPD K, solid cells, walls,
    solute inlet/outlet, hardening law, surface tension, body force; sizes
    spanning several blocks with a ragged tail."""
    prob = W.random_medium(19, 13, 11, seed=21, visc_law=law, A=A)
    g, o = run_both(prob, 25, storage)
    compare(g, o, prob, storage)
    f, h = g.populations()
    rf, rh = o.populations()
    live = prob.solid == 0
    tolp = 1e-13 if storage == "fp64" else 2e-7
    assert np.abs(f[:, live] - rf[:, live]).max() < tolp
    assert np.abs(h[:, live] - rh[:, live]).max() < tolp


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_diagonal_and_no_permeability(storage):
    p = W.random_medium(17, 9, 8, seed=5, spd=False)
    g, o = run_both(p, 20, storage)
    compare(g, o, p, storage)
    p2 = p.replace(K6=None)
    g, o = run_both(p2, 20, storage)
    compare(g, o, p2, storage)


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_plain_channel_full(storage):
    """16x16x64 plain channel, 2000 steps, against the oracle and against the
    Darcy velocity in the bulk."""
    p = W.plain_channel()
    g, o = run_both(p, p.steps, storage)
    compare(g, o, p, storage)
    if storage == "fp64":
        f, _ = g.populations()
        rf, _ = o.populations()
        assert np.abs(f - rf).max() < 1e-13
    _, u, _, _ = g.fields()
    darcy = 1e-6 * float(np.float32(1e-2)) / 0.1
    bulk = u[:, 0].reshape(p.shape)[20:-20]
    assert np.abs(bulk / darcy - 1).max() < (2e-7 if storage == "fp64" else 1e-4)


def test_miscible_small_parity_and_balances():
    """Layered anisotropic medium with solute inlet (40x36x30, 300 steps):
    fields against the oracle, and the GPU's own solute and mass balance."""
    p = W.miscible(40, 36, 30, seed=3)
    g = lb.Lattice(p, storage="fp32", check_every=1)
    m0 = g.reduce()
    g.step(300)
    o = O.Oracle(p)
    o.step(300)
    err = compare(g, o, p, "fp32")
    r = g.reduce()
    ro = o.reduce()
    assert r[0] == pytest.approx(m0[0], rel=1e-9)          # mass
    assert r[2] == pytest.approx(ro[2], rel=1e-5)          # flux in
    assert r[3] == pytest.approx(ro[3], rel=1e-4, abs=1e-9)  # flux out
    assert (r[1] - m0[1]) == pytest.approx(r[2] - r[3], rel=1e-4)
    assert err["u"] < 1e-5


@pytest.mark.parametrize("kernel", ["tuned", "cell", "staged"])
def test_miscible_full_size_first_steps(kernel):
    """128^3, three steps from the seeded initial state, every cell against
    the oracle: with the kernel and launch shape the timing autotuner picks
    (what the benchmark runs), and with each kernel forced."""
    p = W.miscible(128, 128, 128, seed=0)
    g = lb.Lattice(p, storage="fp32", kernel="auto" if kernel == "tuned" else kernel)
    if kernel == "tuned":
        lb.lb_autotune(g.ctx, 3)
    g.step(3)
    o = O.Oracle(p)
    o.step(3)
    compare(g, o, p, "fp32")


def test_precision_crop_spd_fp32():
    """32^3 crop of the rotated-tensor medium, FP32 storage."""
    big = W.precision(64, 64, 64, storage="fp32")
    p = W.crop(big, 16, 0, 8, 32, 32, 32)
    g, o = run_both(p, 200, "fp32")
    compare(g, o, p, "fp32")


@pytest.fixture(scope="module")
def precision_full():
    """256^3 rotated-tensor medium and the oracle's fields after 3 steps."""
    p = W.precision(256, 256, 256, storage="fp32")
    o = O.Oracle(p)
    o.step(3)
    out = (p, o.fields())
    del o  # releases the oracle's ~10 GB of FP64 state
    return out


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
def test_precision_full_size_first_steps(precision_full, storage):
    """256^3 with a full SPD K per cell, in the benchmark's configuration
    (autotuned launch), three steps, every cell against the oracle: FP32 to
    the FP32 tolerances, FP16/BF16 to their long-run bounds."""
    p, (r_rho, r_u, r_C, r_nu) = precision_full
    g = lb.Lattice(p, storage=storage, check_every=1)
    lb.lb_autotune(g.ctx, 2)
    g.step(3)
    rho, u, C, nu = g.fields()
    rel = np.abs(u - r_u).max() / np.abs(r_u).max()
    if storage == "fp32":
        tol = TOL["fp32"]
        assert rel <= tol["u"]
        assert np.abs(rho - r_rho).max() <= tol["rho"]
        assert np.abs(C - r_C).max() <= tol["C"]
        assert np.abs(nu - r_nu).max() <= tol["nu"]
    else:
        assert rel <= (1e-3 if storage == "fp16" else 5e-3)
        assert np.abs(C - r_C).max() <= 1e-3
    g.close()


@pytest.mark.parametrize("storage,bound", [("fp16", 1e-3), ("bf16", 5e-3)])
def test_reduced_precision_storage_error(storage, bound):
    """FP16 / BF16 deviation storage on the rotated-tensor crop: error of u
    against the FP64 oracle, relative to max|u|, and mass drift."""
    big = W.precision(64, 64, 64, storage=storage)
    p = W.crop(big, 16, 0, 8, 32, 32, 32)
    g = lb.Lattice(p, storage=storage)
    m0 = g.reduce()[0]
    g.step(200)
    o = O.Oracle(p)
    o.step(200)
    _, u, _, _ = g.fields()
    _, ru, _, _ = o.fields()
    rel = np.abs(u - ru).max() / np.abs(ru).max()
    print(f"{storage}: max|du|/max|u| = {rel:.3e}")
    assert rel <= bound
    assert abs(g.reduce()[0] / m0 - 1) <= 1e-6


def test_nonfinite_state_is_reported():
    """A NaN population makes the step's FP64 reduction report LB_ENONFINITE."""
    p = W.random_medium(8, 8, 8, seed=2)
    g = lb.Lattice(p, storage="fp32", check_every=1)
    f, h = g.populations()
    f[3, 17] = np.nan
    g.set_populations(f, h)
    g.step(2)
    with pytest.raises(lb.LbError) as e:
        g.sync()
    assert e.value.code == lb.LB_ENONFINITE


def test_single_cell_and_thin_lattices():
    for dims in [(1, 1, 1), (1, 1, 7), (5, 1, 1)]:
        p = W.random_medium(*dims, seed=9, solid_frac=0.0, walls=False, inlet=False)
        g, o = run_both(p, 10, "fp64")
        compare(g, o, p, "fp64")
        f, h = g.populations()
        rf, rh = o.populations()
        assert np.abs(f - rf).max() < 1e-13 and np.abs(h - rh).max() < 1e-13


def test_torch_allocator_and_stream():
    torch = pytest.importorskip("torch")
    lb.use_torch_allocator()
    try:
        s = torch.cuda.Stream()
        p = W.random_medium(12, 10, 8, seed=6)
        g = lb.Lattice(p, storage="fp32", stream=s.cuda_stream)
        g.step(5)
        o = O.Oracle(p)
        o.step(5)
        compare(g, o, p, "fp32")
        g.close()
    finally:
        lb.lb_set_allocator(None)


@pytest.mark.parametrize("dims,factory", [((128, 12, 10), "miscible"), ((128, 10, 8), "precision"),
                                          ((256, 5, 6), "miscible")])
def test_row_pipelined_kernel(dims, factory):
    """The row-pipelined kernel (shared-memory staging by bulk copies) against
    the oracle and against the one-thread-per-cell kernel; the rows on the
    inlet and outlet faces take the per-cell path inside the same launch."""
    if factory == "miscible":
        p = W.miscible(*dims, seed=3)
    else:
        p = W.precision(*dims, storage="fp32", block=8)
    rows = lb.Lattice(p, storage="fp32", kernel="rows", check_every=1)
    cell = lb.Lattice(p, storage="fp32", kernel="cell", check_every=1)
    rows.step(60)
    cell.step(60)
    o = O.Oracle(p)
    o.step(60)
    compare(rows, o, p, "fp32")
    fr, hr = rows.populations()
    fc, hc = cell.populations()
    # same arithmetic; FMA contraction may differ between the two kernels
    assert np.abs(fr - fc).max() < 5e-7 and np.abs(hr - hc).max() < 5e-7
    rr, rc = rows.reduce(), cell.reduce()
    assert rr[2] == pytest.approx(rc[2], rel=1e-6) and rr[3] == pytest.approx(rc[3], rel=1e-5, abs=1e-12)


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_row_pipelined_kernel_is_fp32_only(storage):
    p = W.precision(128, 8, 8, storage=storage, block=8)
    with pytest.raises(lb.LbError) as e:
        lb.Lattice(p, storage=storage, kernel="rows")
    assert e.value.code == lb.LB_EUNSUPPORTED


def test_row_pipelined_kernel_rejects_other_shapes():
    p = W.random_medium(40, 6, 5, seed=1)
    with pytest.raises(lb.LbError) as e:
        lb.Lattice(p, storage="fp32", kernel="rows")
    assert e.value.code == lb.LB_EUNSUPPORTED


STAGED_CASES = {
    # every feature (solids, walls, solute inlet/outlet, full K, surface
    # tension, hardening law); 19-cell rows: 32-thread blocks with a ragged
    # tail; 2400 rows, more than one resident wave, so blocks walk several rows
    "random": lambda: W.random_medium(19, 60, 40, seed=21, visc_law=2, A=1e-3),
    # diagonal K, solute inlet/outlet on the z faces; 40-cell rows: 64-thread blocks
    "miscible40": lambda: W.miscible(40, 36, 30, seed=3),
    # 128-thread blocks, 5120 rows
    "miscible128": lambda: W.miscible(128, 128, 40, seed=2),
    # no permeability, no solute (solids and walls kept)
    "plain": lambda: W.random_medium(33, 20, 30, seed=5, spd=False, solute=False).replace(K6=None),
}


@pytest.mark.parametrize("case", list(STAGED_CASES))
@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_row_staged_kernel(case, storage):
    """The row-staged kernel (persistent blocks, cp.async staging of the next
    row) against the oracle and against the one-thread-per-cell kernel; the
    two share the per-cell arithmetic, boundary cells take the per-cell path."""
    p = STAGED_CASES[case]()
    steps = 25
    st = lb.Lattice(p, storage=storage, kernel="staged", check_every=1)
    cell = lb.Lattice(p, storage=storage, kernel="cell", check_every=1)
    st.step(steps)
    cell.step(steps)
    o = O.Oracle(p)
    o.step(steps)
    compare(st, o, p, storage)
    fs, hs = st.populations()
    fc, hc = cell.populations()
    live = p.solid == 0
    tol = 1e-14 if storage == "fp64" else 5e-7
    assert np.abs(fs[:, live] - fc[:, live]).max() <= tol
    if hs is not None:
        assert np.abs(hs[:, live] - hc[:, live]).max() <= tol
    rs, rc = st.reduce(), cell.reduce()
    assert rs[0] == pytest.approx(rc[0], rel=1e-9)
    assert rs[2] == pytest.approx(rc[2], rel=1e-6, abs=1e-12)
    assert rs[3] == pytest.approx(rc[3], rel=1e-5, abs=1e-12)


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_row_staged_kernel_needs_fp32_or_fp64(storage):
    p = W.miscible(64, 8, 8, seed=1, storage=storage)
    with pytest.raises(lb.LbError) as e:
        lb.Lattice(p, storage=storage, kernel="staged")
    assert e.value.code == lb.LB_EUNSUPPORTED


def test_miscible_full_size_after_5000_steps():
    """128^3 in the benchmark's configuration (autotuned launch, FP32) after
    the workload's 5000 steps: the solute balance of the whole run, and one
    more step from the state reached, every cell against the oracle started
    from the same populations. By then the solute has spread some 30 cells
    in from the inlet (D = 1/10, sqrt(2 D t) = 32), so the step is checked
    where C, tau(C) and the inlet flux all vary."""
    p = W.miscible(128, 128, 128, seed=0)
    g = lb.Lattice(p, storage="fp32", check_every=1)
    lb.lb_autotune(g.ctx, 3)
    r0 = g.reduce()
    g.step(5000)
    r = g.reduce()
    # Solute conservation, Eqs. boltzeqD/equild: the change of the total is
    # what entered minus what left. FP32 storage rounds every stored
    # population to 2^-24 relative each step; rounding errors of independent
    # sign grow like sqrt(5000) * 2^-24 = 4e-6 of the total over the run, and
    # 1e-4 (the bound of the 300-step balance test) leaves room for
    # correlation between them.
    assert r[2] > 0 and r[1] > 0
    assert (r[1] - r0[1]) == pytest.approx(r[2] - r[3], rel=1e-4)
    f, h = g.populations()
    o = O.Oracle(p)
    o.set_populations(f, h)
    g.step(1)
    o.step(1)
    err = compare(g, o, p, "fp32")
    _, _, C, _ = g.fields()
    plane = slice(16 * p.nx * p.ny, 17 * p.nx * p.ny)   # z = 16
    assert C[plane][p.solid[plane] == 0].mean() > 0.1
    print("after 5000 steps, one step vs oracle:", err, "balance",
          (r[1] - r0[1]) / (r[2] - r[3]) - 1)


def test_fp32_long_run_parity():
    """3000 steps of the miscible medium (32x32x48 crop): the FP32 path stays
    inside the tolerances over a long run (no systematic drift of C)."""
    p = W.crop(W.miscible(64, 64, 64, seed=0), 16, 0, 0, 32, 32, 48)
    g, o = run_both(p, 3000, "fp32", threads=0)
    err = compare(g, o, p, "fp32")
    assert err["C"] < 2e-6


def test_fp16_long_run_error():
    """FP16 storage with per-cell FP16 reference pairs, 2000 steps of the
    rotated SPD medium (24^3 crop): velocity within 1e-3 of the oracle, mass
    drift within 1e-6."""
    big = W.precision(64, 64, 64, storage="fp16")
    p = W.crop(big, 16, 0, 8, 24, 24, 24)
    g = lb.Lattice(p, storage="fp16")
    m0 = g.reduce()[0]
    g.step(2000)
    o = O.Oracle(p)
    o.step(2000)
    _, u, _, _ = g.fields()
    _, ru, _, _ = o.fields()
    assert np.abs(u - ru).max() / np.abs(ru).max() <= 1e-3
    assert abs(g.reduce()[0] / m0 - 1) <= 1e-6


def test_autotune_leaves_state_and_picks_a_shape():
    p = W.miscible(128, 16, 12, seed=4)
    g = lb.Lattice(p, storage="fp32", check_every=1)
    g.step(3)
    f0, h0 = g.populations()
    r0 = g.reduce()
    choice = lb.lb_autotune(g.ctx, 3)
    assert choice in (32, 64, 128, 256, 1032, 1064, 1128)
    f1, h1 = g.populations()
    assert np.array_equal(f0, f1) and np.array_equal(h0, h1)
    assert np.array_equal(r0, g.reduce()) and g.t == 3
    g.step(40)
    o = O.Oracle(p)
    o.step(43)
    compare(g, o, p, "fp32")


def test_reduced_precision_storage_full_protocol():
    """The precision workload's error protocol, 10 000 steps: FP16 / BF16
    storage against the FP32-storage GPU run over the full 256^3 domain and
    against the FP64 oracle on a 32^3 crop. FP16 keeps max|du|/max|u| within
    1e-3 and the mass drift within 1e-6 in both; BF16 (8-bit mantissa) is
    held to 5e-3."""
    steps = 10000
    full = {}
    for st in ("fp32", "fp16", "bf16"):
        g = lb.Lattice(W.precision(storage=st), storage=st, check_every=100)
        m0 = g.reduce()[0]
        g.step(steps)
        _, u, C, _ = g.fields()
        full[st] = (u, C, abs(g.reduce()[0] / m0 - 1))
        g.close()
    u32, C32, _ = full["fp32"]
    big = W.precision(64, 64, 64, storage="fp32")
    crop = W.crop(big, 16, 0, 8, 32, 32, 32)
    o = O.Oracle(crop, threads=os.cpu_count())
    o.step(steps)
    _, ru, rC, _ = o.fields()
    for st, bound in (("fp16", 1e-3), ("bf16", 5e-3)):
        u, C, drift = full[st]
        du_full = np.abs(u - u32).max() / np.abs(u32).max()
        g = lb.Lattice(crop.replace(storage=st), storage=st)
        m0 = g.reduce()[0]
        g.step(steps)
        _, uc, Cc, _ = g.fields()
        du_crop = np.abs(uc - ru).max() / np.abs(ru).max()
        drift_crop = abs(g.reduce()[0] / m0 - 1)
        g.close()
        print(f"{st}: full vs FP32 du {du_full:.2e} dC {np.abs(C - C32).max():.2e} drift "
              f"{drift:.1e}; crop vs oracle du {du_crop:.2e} dC {np.abs(Cc - rC).max():.2e} "
              f"drift {drift_crop:.1e}")
        assert du_full <= bound and du_crop <= bound
        assert drift <= 1e-6 and drift_crop <= 1e-6


@pytest.mark.parametrize("storage,tol", [("fp64", 2e-7), ("fp32", 1e-5)])
@pytest.mark.parametrize("tau", [0.8, 0.5 + np.sqrt(3.0 / 16.0)])
def test_poiseuille_exact_discrete_solution_on_the_gpu(storage, tol, tau):
    """The GPU path on plane Poiseuille flow against the exact steady BGK
    solution with halfway bounce-back walls (the oracle's pin),
    u(y) = G/(2 nu) [y (L - y) + (16 (tau - 1/2)^2 - 3)/12]; FP64 storage to
    the float32 rounding of the exported field, FP32 to the 1e-5 bound."""
    nz, G = 16, 1e-6
    p = W.brinkman(nz=nz, K=1.0, eps=1.0, tau=tau, G=G, nxy=4).replace(K6=None, storage=storage)
    g = lb.Lattice(p, storage=storage)
    nu = (tau - 0.5) / 3.0
    g.step(int(np.ceil(40.0 * nz * nz / (np.pi ** 2 * nu))))
    _, u, _, _ = g.fields()
    u = u.reshape(nz, 4, 4, 3)
    y = np.arange(nz) + 0.5
    exact = G / (2 * nu) * (y * (nz - y) + (16 * (tau - 0.5) ** 2 - 3) / 12)
    assert np.abs(u[..., 0] - exact[:, None, None]).max() <= tol * np.abs(exact).max()
    g.close()


@pytest.mark.parametrize("where", ["pinned", "device"])
def test_init_reads_addressable_inputs_in_place(where):
    """lb_init from pinned host or device arrays (read in place by the
    initialisation) gives the state that pageable arrays (copied) give."""
    torch = pytest.importorskip("torch")
    p = W.random_medium(19, 13, 11, seed=8)
    a = lb.Lattice(p, storage="fp32", init=False)
    b = lb.Lattice(p, storage="fp32", init=False)
    arrs = [np.ascontiguousarray(x, np.float32) for x in (p.rho0, p.u0, p.C0)]
    lb.lb_init(a.ctx, *arrs)
    if where == "pinned":
        ts = [torch.from_numpy(x).pin_memory() for x in arrs]
    else:
        ts = [torch.from_numpy(x).cuda() for x in arrs]
    torch.cuda.synchronize()
    lb.lb_init(b.ctx, *ts)
    b.sync()
    for n in (0, 9):
        a.step(n)
        b.step(n)
        fa, ha = a.populations()
        fb, hb = b.populations()
        assert np.array_equal(fa, fb) and np.array_equal(ha, hb)
