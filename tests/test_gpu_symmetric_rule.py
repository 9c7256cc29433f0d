"""GPU parity on the fully symmetric degree-2p volume rules (Section 4.3.2's kind
of rule, 3 / 6 / 12 / 16 / 25 points at p = 1..5) against the oracle on the
same rule, through the C ABI.

The library derives its rule itself (extended precision) and contracts the
volume term directly on it; the oracle installs its own derivation (50-digit
decimal).  Float64: relative L2 <= 1e-12 for one RHS, for whole runs of every
time integrator (graph replay included), for the discrete adjoint, on periodic
meshes and on a closed box; the tensor-core modes against the float64 GPU run
on the same rule; one step of the 256 x 256, p = 3 workload in the launch
configuration the benchmark times.
"""
import numpy as np
import pytest

from paper_1601_07944_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-12
RULE = "symmetric"


@pytest.fixture(scope="module")
def dgmod():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1601_07944_gb300 import _build, dg
    _build.build()
    dg.load()
    return dg


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _pair(dgmod, oracle_mod, mesh, p, ne=0):
    m = dgmod.Mesh.from_mesh(mesh, p, n_edge_pts=ne, vol_rule=RULE)
    o = oracle_mod.OracleDG.from_mesh(mesh, p, n_edge_pts=ne, vol_rule=RULE)
    assert m.nq == o.nq == {1: 3, 2: 6, 3: 12, 4: 16, 5: 25}[p]
    return m, o


@pytest.mark.parametrize("p,ne", [(1, 0), (2, 0), (3, 0), (3, 3), (4, 0), (5, 0)])
@pytest.mark.parametrize("n", [5, 8])
def test_rhs_parity(dgmod, oracle_mod, p, ne, n):
    """n = 5: 50 elements, n = 8: 128 elements; both end in a ragged tile at
    every p (64, 32 or 16 elements per tile)."""
    m, o = _pair(dgmod, oracle_mod, I.periodic_mesh(n), p, ne)
    c = o.project_ic(I.perturbed_vortex)
    got = _host(m.rhs(_dev(c)))
    ref = o.rhs(c)
    assert rel_l2(got, ref) < TOL, rel_l2(got, ref)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_projection_and_points(dgmod, oracle_mod, p):
    """The library's volume points and projection on the symmetric rule match
    the oracle's."""
    mesh = I.periodic_mesh(6)
    m, o = _pair(dgmod, oracle_mod, mesh, p)
    xy = _host(m.volume_points())
    assert np.abs(xy - o.volume_points()).max() < 1e-13
    c = _host(m.project_function(I.perturbed_vortex))
    ref = o.project_ic(I.perturbed_vortex)
    assert rel_l2(c, ref) < TOL


@pytest.mark.parametrize("method", ["ssp_rk3", "rk2", "rk4"])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_stepping_parity(dgmod, oracle_mod, method, p):
    """20 steps: one plain step, a replayed 16-step graph, three more."""
    mesh = I.periodic_mesh(8)
    m, o = _pair(dgmod, oracle_mod, mesh, p)
    ic = I.perturbed_vortex
    dt = I.fixed_dt(mesh, ic, p)
    c0 = o.project_ic(ic)
    ref = getattr(o, method)(c0, dt, 20)
    c = _dev(c0)
    m.rk_step(c, dt, 20, method=method)
    m.device_status()
    assert rel_l2(_host(c), ref) < TOL, rel_l2(_host(c), ref)


def test_full_size_step(dgmod, oracle_mod):
    """One SSP-RK3 step of the 256 x 256, p = 3 workload on the symmetric rule."""
    mesh = I.periodic_mesh(256)
    m, o = _pair(dgmod, oracle_mod, mesh, 3)
    dt = I.fixed_dt(mesh, I.vortex, 3)
    c0 = o.project_ic(I.vortex)
    c = _dev(c0)
    m.rk_step(c, dt, 1)
    m.device_status()
    ref = o.ssp_rk3(c0, dt, 1)
    assert rel_l2(_host(c), ref) < TOL


@pytest.mark.parametrize("case", ["box", "vortex_state"])
def test_boundary_parity(dgmod, oracle_mod, case):
    if case == "box":
        mesh = I.box_mesh(8)

        def ic(x, y):
            a, th = I.fourier_coefficients()
            d = I.fourier_perturbation(x, y, a, th, 5e-2)
            zero = np.zeros_like(d[0])
            return I.primitive_to_conserved(1.0 + d[0], zero, zero, 1.0 + d[1])
    else:
        mesh = I.box_mesh(8, x_code=I.BC_STATE, y_code=I.BC_STATE)
        ic = I.steady_vortex
    m, o = _pair(dgmod, oracle_mod, mesh, 3)
    if case == "vortex_state":
        xy = _host(m.boundary_points())
        m.set_boundary_state(_dev(ic(xy[..., 0], xy[..., 1])))
        oxy = o.boundary_points()
        o.set_boundary_state(ic(oxy[..., 0], oxy[..., 1]))
    c0 = o.project_ic(ic)
    dt = I.fixed_dt(mesh, ic, 3)
    ref = o.ssp_rk3(c0, dt, 20)
    c = _dev(c0)
    m.rk_step(c, dt, 20)
    m.device_status()
    assert rel_l2(_host(c), ref) < TOL


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_adjoint_parity(dgmod, oracle_mod, p):
    mesh = I.periodic_mesh(6)
    m, o = _pair(dgmod, oracle_mod, mesh, p)
    rng = np.random.default_rng(9)
    c0 = o.project_ic(I.perturbed_vortex)
    lam = rng.standard_normal(c0.shape)
    got = _host(m.rhs_adjoint(_dev(c0), _dev(lam)))
    ref = o.rhs_vjp(c0, lam)
    assert rel_l2(got, ref) < TOL, rel_l2(got, ref)
    dt = I.fixed_dt(mesh, I.perturbed_vortex, p)
    got = _host(m.adjoint_step(_dev(c0), dt, _dev(lam)))
    ref = o.ssp_rk3_vjp(c0, dt, lam)
    assert rel_l2(got, ref) < TOL, rel_l2(got, ref)


def test_limited_stepping_parity(dgmod, oracle_mod):
    mesh = I.periodic_mesh(16)
    m, o = _pair(dgmod, oracle_mod, mesh, 1)
    c0 = o.limit(o.project_ic(I.density_steps))
    dt = I.fixed_dt(mesh, I.density_steps, 1)
    o.set_limiter(True)
    m.set_limiter(True)
    ref = o.rk2(c0, dt, 20)
    c = _dev(c0)
    m.rk_step(c, dt, 20, method="rk2")
    m.device_status()
    assert rel_l2(_host(c), ref) < TOL


@pytest.mark.parametrize("prec,tol", [("tf32x3", 1e-6), ("tf32x1", 1e-3)])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_mixed_vs_fp64(dgmod, p, prec, tol):
    """The tensor-core modes on the symmetric rule: state error against the
    float64 GPU run on the same rule after 20 steps, within the bounds the
    mixed modes meet on the collapsed grid; totals conserved."""
    mesh = I.periodic_mesh(32)
    m = dgmod.Mesh.from_mesh(mesh, p, vol_rule=RULE)
    c0 = m.project_function(I.perturbed_vortex)
    dt = I.fixed_dt(mesh, I.perturbed_vortex, p)
    a = c0.clone(); b = c0.clone()
    m.rk_step(a, dt, 20)
    t0 = m.conserved_totals(b)
    m.rk_step(b, dt, 20, precision=prec)
    m.device_status()
    A, B = _host(a), _host(b)
    assert np.linalg.norm(B - A) / np.linalg.norm(A) < tol
    assert np.all(np.abs(m.conserved_totals(b) - t0) <= 1e-13 * np.abs(t0))


def test_rules_give_different_but_close_solutions(dgmod):
    """Same data on the two rules: the runs differ (aliasing of the nonlinear
    flux) by far less than the discretisation error scale."""
    mesh = I.periodic_mesh(32)
    a = dgmod.Mesh.from_mesh(mesh, 3)
    b = dgmod.Mesh.from_mesh(mesh, 3, vol_rule=RULE)
    dt = I.fixed_dt(mesh, I.vortex, 3)
    ca = a.project_function(I.vortex)
    cb = b.project_function(I.vortex)
    a.rk_step(ca, dt, 20)
    b.rk_step(cb, dt, 20)
    d = np.linalg.norm(_host(ca) - _host(cb)) / np.linalg.norm(_host(ca))
    assert 1e-12 < d < 1e-4
