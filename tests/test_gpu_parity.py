"""GPU (sm_103a) parity of the float64 path against the CPU oracle, through the C ABI.

Tolerance: relative L2 over all coefficients <= 1e-12 (the float64 path differs
from the oracle only in the order of roundings; a single RHS agrees to ~1e-15).
Sizes span several element tiles with a ragged last tile (n = 6 gives N = 72,
n = 16 gives N = 512), and the full 256 x 256 workload is checked on one RHS and
one time step in the launch configuration the benchmark times.
"""
import math

import numpy as np
import pytest

from paper_1601_07944_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def dgmod():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1601_07944_gb300 import _build, dg
    _build.build()
    dg.load()
    return dg


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


CASES = [(1, 0), (2, 0), (3, 0), (3, 3), (4, 0), (5, 0)]


def test_volume_points_match(dgmod, oracle_mod):
    mesh = I.periodic_mesh(6)
    for p in (1, 4):
        m = dgmod.Mesh.from_mesh(mesh, p)
        o = oracle_mod.OracleDG.from_mesh(mesh, p)
        assert np.abs(_host(m.volume_points()) - o.volume_points()).max() < 1e-14


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_project_ic_parity(dgmod, oracle_mod, p):
    mesh = I.periodic_mesh(6)
    m = dgmod.Mesh.from_mesh(mesh, p)
    o = oracle_mod.OracleDG.from_mesh(mesh, p)
    got = _host(m.project_function(I.perturbed_vortex))
    ref = o.project_ic(I.perturbed_vortex)
    assert rel_l2(got, ref) < 1e-14


@pytest.mark.parametrize("n", [6, 16])
@pytest.mark.parametrize("p,ne", CASES)
def test_rhs_parity(dgmod, oracle_mod, p, ne, n):
    mesh = I.periodic_mesh(n)
    m = dgmod.Mesh.from_mesh(mesh, p, n_edge_pts=ne)
    o = oracle_mod.OracleDG.from_mesh(mesh, p, n_edge_pts=ne)
    c = o.project_ic(I.perturbed_vortex)
    ref = o.rhs(c)
    got = _host(m.rhs(_dev(c)))
    assert rel_l2(got, ref) < TOL
    assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("p,ne,n,steps", [(1, 0, 16, 100), (2, 0, 16, 20), (3, 0, 16, 20),
                                          (3, 3, 16, 10), (4, 0, 8, 10), (5, 0, 8, 5)])
def test_rk_step_parity(dgmod, oracle_mod, p, ne, n, steps):
    """Whole runs: each side projects the initial data with its own tables and
    advances with SSP-RK3 at the same fixed dt.  (p=1, n=16, 100 steps is the
    512-element vortex workload in full.)"""
    mesh = I.periodic_mesh(n)
    ic = I.vortex if p == 1 else I.perturbed_vortex
    dt = I.fixed_dt(mesh, ic, p)
    m = dgmod.Mesh.from_mesh(mesh, p, n_edge_pts=ne)
    o = oracle_mod.OracleDG.from_mesh(mesh, p, n_edge_pts=ne)
    c = m.project_function(ic)
    m.rk_step(c, dt, steps)
    ref = o.ssp_rk3(o.project_ic(ic), dt, steps)
    got = _host(c)
    assert rel_l2(got, ref) < TOL, rel_l2(got, ref)


def test_totals_parity_and_conservation(dgmod, oracle_mod):
    mesh = I.periodic_mesh(16)
    p = 2
    m = dgmod.Mesh.from_mesh(mesh, p)
    o = oracle_mod.OracleDG.from_mesh(mesh, p)
    c = m.project_function(I.perturbed_vortex)
    t0 = m.conserved_totals(c)
    ref = o.totals(_host(c))
    assert np.all(np.abs(t0 - ref) <= 1e-14 * np.abs(ref))
    assert np.array_equal(t0, m.conserved_totals(c))          # fixed-order reduction
    m.rk_step(c, I.fixed_dt(mesh, I.perturbed_vortex, p), 50)
    t1 = m.conserved_totals(c)
    assert np.all(np.abs(t1 - t0) <= 1e-13 * np.abs(t0))


def test_deterministic(dgmod):
    mesh = I.periodic_mesh(16)
    m = dgmod.Mesh.from_mesh(mesh, 3)
    c0 = m.project_function(I.perturbed_vortex)
    dt = I.fixed_dt(mesh, I.perturbed_vortex, 3)
    a = c0.clone(); b = c0.clone()
    m.rk_step(a, dt, 5)
    m.rk_step(b, dt, 5)
    assert np.array_equal(_host(a), _host(b))


def test_host_entry_matches_device_entry(dgmod):
    import torch
    mesh = I.periodic_mesh(8)
    m = dgmod.Mesh.from_mesh(mesh, 2)
    c = m.project_function(I.vortex)
    dt = I.fixed_dt(mesh, I.vortex, 2)
    h = torch.empty(c.shape, dtype=torch.float64).pin_memory()
    h.copy_(c.cpu())
    m.rk_step(c, dt, 3)
    m.rk_step_host(h, dt, 3)
    assert np.array_equal(_host(c), h.numpy())


@pytest.mark.parametrize("p,steps", [(1, 1), (3, 1), (3, 3)])
def test_host_entry_in_place_on_pinned_memory(dgmod, p, steps):
    """On a mesh the fused small-mesh stepper does not take (9,800 elements), a
    page-locked host state is read in place by the first kernel (the traces
    kernel makes the device copy); a pageable one is copied in.  Both give
    dg_rk_step's bits."""
    import torch
    mesh = I.periodic_mesh(70)
    m = dgmod.Mesh.from_mesh(mesh, p)
    c = m.project_function(I.perturbed_vortex)
    dt = I.fixed_dt(mesh, I.perturbed_vortex, p)
    pinned = torch.empty(c.shape, dtype=torch.float64).pin_memory()
    pinned.copy_(c.cpu())
    pageable = c.cpu().clone()
    m.rk_step(c, dt, steps)
    m.rk_step_host(pinned, dt, steps)
    m.rk_step_host(pageable, dt, steps)
    m.device_status()
    ref = _host(c)
    assert np.array_equal(pinned.numpy(), ref)
    assert np.array_equal(pageable.numpy(), ref)


def test_free_stream_full_size(dgmod):
    """A uniform state is an exact steady solution on the full 1024^2 p=5 mesh:
    the RHS vanishes up to the rounding of its two terms, each of size about
    |F| |grad phi| / h (eps times that is ~4e-12 here)."""
    mesh = I.periodic_mesh(1024)
    p = 5
    m = dgmod.Mesh.from_mesh(mesh, p)
    c = m.project_function(lambda x, y: I.uniform_state(x, y))
    r = _host(m.rhs(c))
    U = I.uniform_state(np.zeros(1), np.zeros(1))[0]
    rho, u, v = U[0], U[1] / U[0], U[2] / U[0]
    pr = 0.4 * (U[3] - 0.5 * rho * (u * u + v * v))
    fmax = max(abs(U[3] + pr) * max(abs(u), abs(v)), abs(U[1] * u + pr), abs(U[2] * v + pr))
    T = dgmod.host_tables(p)
    gmax = max(np.abs(T["dphi_r"]).max(), np.abs(T["dphi_s"]).max())
    scale = np.finfo(float).eps * fmax * gmax / mesh.h
    assert np.abs(r).max() < 16 * scale


@pytest.mark.parametrize("n,p", [(256, 3), (512, 4)])
def test_full_size_parity(dgmod, oracle_mod, n, p):
    """The 256^2 p=3 and 512^2 p=4 workloads at full size: one RHS and one SSP-RK3
    step against the oracle, in the benchmark's launch configuration."""
    mesh = I.periodic_mesh(n)
    ic = I.vortex if n == 256 else I.perturbed_vortex
    m = dgmod.Mesh.from_mesh(mesh, p)
    o = oracle_mod.OracleDG.from_mesh(mesh, p)
    c = o.project_ic(ic)
    # R is the difference of two terms that each grow like 1/h; its rounding error
    # is eps times their size, which at these h exceeds 1e-12 |R|
    ref, vol = o.rhs_and_volume(c)
    got = _host(m.rhs(_dev(c)))
    eps = np.finfo(float).eps
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref) + 16 * eps * np.linalg.norm(vol)
    dt = I.fixed_dt(mesh, ic, p)
    cd = _dev(c)
    m.rk_step(cd, dt, 1)
    assert rel_l2(_host(cd), o.ssp_rk3(c, dt, 1)) < TOL


def test_argument_errors(dgmod):
    import torch
    mesh = I.periodic_mesh(4)
    m = dgmod.Mesh.from_mesh(mesh, 1)
    c = m.project_function(I.vortex)
    with pytest.raises(dgmod.DGError) as ei:
        m.rhs(c, out=c)                       # aliasing input and output
    assert ei.value.status == 1
    with pytest.raises(dgmod.DGError) as ei:
        m.adjoint_step(c, 0.01, c, out=c)
    assert ei.value.status == 1
    with pytest.raises(dgmod.DGError) as ei:
        m.rk_step(c, float("nan"), 1)
    assert ei.value.status == 1
    with pytest.raises(ValueError):
        m.rhs(torch.zeros((3, 4, 3), dtype=torch.float64, device="cuda"))


def test_eval_points_and_l2_error(dgmod, oracle_mod):
    """Point values of the solution (dg_eval_points) and the L2 error built on them
    agree with the oracle's."""
    mesh = I.periodic_mesh(8)
    p = 3
    m = dgmod.Mesh.from_mesh(mesh, p)
    o = oracle_mod.OracleDG.from_mesh(mesh, p)
    c = o.project_ic(I.vortex)
    rng = np.random.default_rng(2)
    r = rng.uniform(0.02, 0.48, 9)
    s = rng.uniform(0.02, 0.48, 9)
    got = _host(m.eval_points(_dev(c), r, s))
    ref = o.eval_points(c, r, s)
    assert rel_l2(got, ref) < 1e-14
    T = dgmod.host_tables(p + 3)
    rule = (T["vol_r"], T["vol_s"], T["vol_w"])
    e_gpu = m.l2_error(_dev(c), lambda x, y: I.vortex(x, y, 0.0), rule=rule)
    e_or = o.l2_error(c, lambda x, y: I.vortex(x, y, 0.0))
    assert abs(e_gpu - e_or) <= 1e-10 * e_or


@pytest.mark.parametrize("p", [1, 2, 3])
def test_vortex_convergence_order(dgmod, p):
    """The closed-form isentropic vortex: the L2 density error of the GPU solver at
    t = 0.5 falls like h^(p+1) on n = 32, 64, 128 (dt fixed from the finest mesh,
    small enough that the time error stays below the spatial one)."""
    import math
    ns = (32, 64, 128)
    T = 0.5
    dt = 0.5 * I.fixed_dt(I.periodic_mesh(ns[-1]), I.vortex, p)
    steps = int(math.ceil(T / dt))
    dt = T / steps
    errs = []
    for n in ns:
        mesh = I.periodic_mesh(n)
        m = dgmod.Mesh.from_mesh(mesh, p)
        c = m.project_function(I.vortex)
        m.rk_step(c, dt, steps)
        errs.append(m.l2_error(c, lambda x, y: I.vortex(x, y, T)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert rates[-1] > p + 1 - 0.3, (errs, rates)


def test_full_size_parity_1024_p5(dgmod, oracle_mod):
    """The 1024^2, p=5 workload (2,097,152 elements, 176 M DOF) at full size: one RHS
    and one SSP-RK3 step against the oracle."""
    mesh = I.periodic_mesh(1024)
    p = 5
    m = dgmod.Mesh.from_mesh(mesh, p)
    o = oracle_mod.OracleDG.from_mesh(mesh, p)
    c = o.project_ic(I.vortex)
    ref, vol = o.rhs_and_volume(c)
    got = _host(m.rhs(_dev(c)))
    eps = np.finfo(float).eps
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref) + 16 * eps * np.linalg.norm(vol)
    del got, ref, vol
    dt = I.fixed_dt(mesh, I.vortex, p)
    cd = _dev(c)
    m.rk_step(cd, dt, 1)
    assert rel_l2(_host(cd), o.ssp_rk3(c, dt, 1)) < TOL


def _full_run_samples():
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "full_run_samples.json")
    with open(path) as fh:
        return json.load(fh)["runs"]


@pytest.mark.parametrize("run", [0, 1])
def test_full_run_parity(dgmod, run):
    """Whole runs at full size against the oracle (tests/golden/full_run_samples.json,
    written by make_full_run_samples.py from the oracle alone): the 256^2 p=3
    vortex after its 200 steps and the 256^2 p=2 perturbed vortex after the 400
    steps of the adjoint workload's forward run; the GPU run replays the 16-step
    CUDA graph.  Sampled coefficients (1024 seeded indices) within 1e-12 relative
    L2, the whole state's norm within 1e-12, the totals within 1e-13."""
    r = _full_run_samples()[run]
    mesh = I.periodic_mesh(r["n"])
    f = getattr(I, r["ic"])
    m = dgmod.Mesh.from_mesh(mesh, r["p"])
    assert list(m.coef_shape) == r["shape"]
    dt = r["dt"]                              # the oracle run's step (libm may differ in the last bit)
    assert abs(I.fixed_dt(mesh, f, r["p"]) - dt) <= 1e-14 * dt
    c = m.project_function(f)
    m.rk_step(c, dt, r["steps"])
    m.device_status()
    got = _host(c).reshape(-1)
    ref = np.array(r["value"])
    sample = got[np.array(r["index"])]
    assert rel_l2(sample, ref) < TOL, rel_l2(sample, ref)
    assert abs(np.linalg.norm(got) - r["l2_norm"]) <= 1e-12 * r["l2_norm"]
    tot = m.conserved_totals(c)
    assert np.all(np.abs(tot - np.array(r["totals"])) <= 1e-13 * np.abs(np.array(r["totals"])))


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_graph_replay_matches_plain_launches(dgmod, prec):
    """A 40-step call (one plain step, two replays of the 16-step CUDA graph, seven
    plain steps) gives bit for bit the state of 40 one-step calls (the separate
    launches: the fused small-mesh stepper is switched off)."""
    mesh = I.periodic_mesh(16)
    m = dgmod.Mesh.from_mesh(mesh, 2)
    m.set_small_mesh_stepper(False)
    c0 = m.project_function(I.perturbed_vortex)
    dt = I.fixed_dt(mesh, I.perturbed_vortex, 2)
    a = c0.clone(); b = c0.clone()
    m.rk_step(a, dt, 40, precision=prec)
    for _ in range(40):
        m.rk_step(b, dt, 1, precision=prec)
    m.device_status()
    assert np.array_equal(_host(a), _host(b))
    m.rk_step(a, dt, 20, precision=prec)          # replay of the cached graph
    for _ in range(20):
        m.rk_step(b, dt, 1, precision=prec)
    assert np.array_equal(_host(a), _host(b))


def test_stable_dt(dgmod, oracle_mod):
    """dg_stable_dt against the same formula evaluated from the oracle's point values."""
    mesh = I.periodic_mesh(12)
    p = 3
    m = dgmod.Mesh.from_mesh(mesh, p)
    o = oracle_mod.OracleDG.from_mesh(mesh, p)
    c = o.project_ic(I.perturbed_vortex)
    r, s, _ = o.volume_rule()
    U = o.eval_points(c, r, s)
    rho, u, v = U[..., 0], U[..., 1] / U[..., 0], U[..., 2] / U[..., 0]
    pr = 0.4 * (U[..., 3] - 0.5 * rho * (u * u + v * v))
    smax = np.max(np.sqrt(u * u + v * v) + np.sqrt(1.4 * pr / rho))
    xy = mesh.elem_xy
    a2 = np.abs((xy[:, 1, 0] - xy[:, 0, 0]) * (xy[:, 2, 1] - xy[:, 0, 1])
                - (xy[:, 1, 1] - xy[:, 0, 1]) * (xy[:, 2, 0] - xy[:, 0, 0]))
    per = sum(np.hypot(*(xy[:, (q + 1) % 3] - xy[:, q]).T) for q in range(3))
    ref = 0.3 * np.min(a2 / per) / ((2 * p + 1) * smax)
    assert abs(m.stable_dt(_dev(c), 0.3) - ref) <= 1e-13 * ref


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_non_physical_state_reported(dgmod, prec):
    """A state with negative density in one element is reported as DG_ENONPHYS by
    dg_device_status (and by dg_stable_dt); the record then clears."""
    mesh = I.periodic_mesh(8)
    m = dgmod.Mesh.from_mesh(mesh, 2)
    c = m.project_function(I.vortex)
    m.device_status()
    bad = c.clone()
    bad[5, 0, 0] = -1.0
    m.rhs(bad, precision=prec)
    with pytest.raises(dgmod.DGError) as ei:
        m.device_status()
    assert ei.value.status == 5
    m.device_status()                       # cleared
    with pytest.raises(dgmod.DGError) as ei:
        m.stable_dt(bad)
    assert ei.value.status == 5
    m.rhs(c, precision=prec)
    m.device_status()


def test_det_j_and_map_points(dgmod, oracle_mod):
    """dg_det_j and dg_map_points (Eq. 2dmap) against the oracle's geometry; the
    library's L2 error is repeatable bit for bit (fixed-order reduction)."""
    mesh = I.periodic_mesh(9)
    m = dgmod.Mesh.from_mesh(mesh, 2)
    o = oracle_mod.OracleDG.from_mesh(mesh, 2)
    assert np.abs(_host(m.det_j()) - o.det_j()).max() <= 1e-15 * np.abs(o.det_j()).max()
    rng = np.random.default_rng(5)
    r = rng.uniform(0.01, 0.49, 7)
    s = rng.uniform(0.01, 0.49, 7)
    xy = _host(m.map_points(r, s))
    ref = o.map_points(r, s)
    assert np.abs(xy - np.asarray(ref).reshape(xy.shape)).max() < 1e-14
    c = m.project_function(I.vortex)
    e1 = m.l2_error(c, lambda x, y: I.vortex(x, y, 0.0))
    assert e1 == m.l2_error(c, lambda x, y: I.vortex(x, y, 0.0)) and e1 > 0.0
