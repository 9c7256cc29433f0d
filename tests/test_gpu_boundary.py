"""GPU parity of boundary faces (Algorithm 2's ghost states: solid walls and
prescribed states) against the oracle, through the C ABI.

The discrete adjoint runs through the same ghost states.

Meshes: the jittered mesh with walls on x = +-5 (a channel, periodic in y), a
closed box of walls, and a box whose four sides carry the exact values of a
steady vortex (each side evaluates them at its own boundary points).  Float64:
relative L2 <= 1e-12 for one RHS and over 20 SSP-RK3 steps (graph replay
included); the tensor-core modes against the float64 GPU run within the bounds
they meet on periodic meshes.
"""
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


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _acoustic(x, y):
    a, th = I.fourier_coefficients()
    d = I.fourier_perturbation(x, y, a, th, 5e-2)
    zero = np.zeros_like(d[0])
    return I.primitive_to_conserved(1.0 + d[0], zero, zero, 1.0 + d[1])


CASES = {
    "channel": (lambda n: I.box_mesh(n, x_code=I.BC_WALL, y_code=0), _acoustic),
    "box": (lambda n: I.box_mesh(n), _acoustic),
    "vortex_state": (lambda n: I.box_mesh(n, x_code=I.BC_STATE, y_code=I.BC_STATE), I.steady_vortex),
}


def _setup(dgmod, oracle_mod, case, n, p, ne=0):
    make, ic = CASES[case]
    mesh = make(n)
    m = dgmod.Mesh.from_mesh(mesh, p, n_edge_pts=ne)
    o = oracle_mod.OracleDG.from_mesh(mesh, p, n_edge_pts=ne)
    if case == "vortex_state":
        xy = _host(m.boundary_points())
        m.set_boundary_state(_dev(ic(xy[..., 0], xy[..., 1])))
        oxy = o.boundary_points()
        o.set_boundary_state(ic(oxy[..., 0], oxy[..., 1]))
    assert m.n_boundary == o.n_boundary > 0
    return mesh, m, o, ic


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("p,ne", [(1, 0), (2, 0), (3, 0), (3, 3), (4, 0), (5, 0)])
def test_boundary_rhs_parity(dgmod, oracle_mod, case, p, ne):
    mesh, m, o, ic = _setup(dgmod, oracle_mod, case, 6, p, ne)
    c = o.project_ic(ic)
    ref = o.rhs(c)
    got = _host(m.rhs(_dev(c)))
    assert rel_l2(got, ref) < TOL, rel_l2(got, ref)


@pytest.mark.parametrize("case", sorted(CASES))
def test_boundary_rk_step_parity(dgmod, oracle_mod, case):
    mesh, m, o, ic = _setup(dgmod, oracle_mod, case, 16, 3)
    c0 = o.project_ic(ic)
    dt = I.fixed_dt(mesh, ic, 3)
    ref = o.ssp_rk3(c0, dt, 20)
    c = _dev(c0)
    m.rk_step(c, dt, 20)
    m.device_status()
    assert rel_l2(_host(c), ref) < TOL, rel_l2(_host(c), ref)


def test_closed_box_conserves_mass_and_energy(dgmod, oracle_mod):
    mesh, m, o, ic = _setup(dgmod, oracle_mod, "box", 16, 3)
    c = m.project_function(ic)
    t0 = m.conserved_totals(c)
    m.rk_step(c, I.fixed_dt(mesh, ic, 3), 40)
    t1 = m.conserved_totals(c)
    assert abs(t1[0] - t0[0]) <= 1e-13 * abs(t0[0]) and abs(t1[3] - t0[3]) <= 1e-13 * abs(t0[3])


@pytest.mark.parametrize("prec,tol", [("tf32x3", 1e-6), ("tf32x1", 1e-3)])
@pytest.mark.parametrize("case", sorted(CASES))
def test_boundary_mixed_vs_fp64(dgmod, oracle_mod, case, prec, tol):
    mesh, m, o, ic = _setup(dgmod, oracle_mod, case, 32, 3)
    c0 = m.project_function(ic)
    dt = I.fixed_dt(mesh, ic, 3)
    a = c0.clone(); b = c0.clone()
    m.rk_step(a, dt, 20)
    m.rk_step(b, dt, 20, precision=prec)
    m.device_status()
    A, B = _host(a), _host(b)
    assert np.linalg.norm(B - A) / np.linalg.norm(A) < tol


def test_boundary_limiter_parity(dgmod, oracle_mod):
    """p = 1 in a closed box with discontinuous data, every stage limited (a
    boundary face adds no neighbour to the limiter's bounds)."""
    mesh = I.box_mesh(16)
    m = dgmod.Mesh.from_mesh(mesh, 1)
    o = oracle_mod.OracleDG.from_mesh(mesh, 1)
    c0 = o.limit(o.project_ic(I.density_steps))
    dt = I.fixed_dt(mesh, I.density_steps, 1)
    o.set_limiter(True)
    m.set_limiter(True)
    ref = o.ssp_rk3(c0, dt, 20)
    c = _dev(c0)
    m.rk_step(c, dt, 20)
    m.device_status()
    assert rel_l2(_host(c), ref) < TOL, rel_l2(_host(c), ref)


def test_boundary_noalloc_rhs(dgmod, oracle_mod):
    import torch
    mesh, m, o, ic = _setup(dgmod, oracle_mod, "vortex_state", 16, 3)
    c = m.project_function(ic)
    r1 = m.rhs(c)
    r2 = torch.empty_like(c)
    m.rhs_noalloc(c, out=r2)
    assert torch.equal(r1, r2)


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("p", [1, 2, 3])
def test_boundary_adjoint_parity(dgmod, oracle_mod, case, p):
    """(dR/dc)^T lam and the adjoint of one SSP-RK3 step through the ghost states,
    against the oracle's reverse sweep."""
    mesh, m, o, ic = _setup(dgmod, oracle_mod, case, 6, p)
    rng = np.random.default_rng(5)
    c0 = o.project_ic(ic)
    lam = rng.standard_normal(c0.shape)
    got = _host(m.rhs_adjoint(_dev(c0), _dev(lam)))
    ref = o.rhs_vjp(c0, lam)
    assert rel_l2(got, ref) < TOL, rel_l2(got, ref)
    dt = I.fixed_dt(mesh, ic, p)
    got = _host(m.adjoint_step(_dev(c0), dt, _dev(lam)))
    ref = o.ssp_rk3_vjp(c0, dt, lam)
    assert rel_l2(got, ref) < TOL, rel_l2(got, ref)


def test_boundary_refusals(dgmod):
    mesh = I.box_mesh(8, x_code=I.BC_STATE, y_code=I.BC_WALL)
    m = dgmod.Mesh.from_mesh(mesh, 2)
    c = m.project_function(I.steady_vortex)
    with pytest.raises(dgmod.DGError) as e:
        m.rhs(c)                                        # no boundary state yet
    assert e.value.status == 1
    xy = _host(m.boundary_points())
    m.set_boundary_state(_dev(I.steady_vortex(xy[..., 0], xy[..., 1])))
    m.rhs(c)
    bad = I.box_mesh(4)
    bad.nbr[0, 0] = -5 if bad.nbr[0, 0] < 0 else bad.nbr[0, 0]
    bad.nbr[bad.nbr == I.BC_WALL] = -5
    with pytest.raises(dgmod.DGError) as e:
        dgmod.Mesh.from_mesh(bad, 1)
    assert e.value.status == 4                          # DG_EMESH
