"""The fused small-mesh stepper (dg_set_small_mesh_stepper): on a mesh whose
element tiles fit in one wave of the GPU, a float64 Runge-Kutta call runs every
stage in one cooperative launch, the edge, element and (with the limiter on)
limiter phases separated by a barrier over the grid.  It runs the same code as
the separate launches, so the states agree bit for bit; every small-mesh parity
test of the suite (against the oracle) goes through it by default."""
import numpy as np
import pytest

from paper_1601_07944_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dgmod():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1601_07944_gb300 import _build, dg
    _build.build()
    dg.load()
    return dg


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _run(m, c0, dt, steps, method, fused):
    """The state after `steps` steps in one call, and the kernel kinds one more
    call launches (per-kernel timing is on for that call only: it turns the CUDA
    graphs of the separate-launch path off)."""
    m.set_small_mesh_stepper(fused)
    c = c0.clone()
    m.rk_step(c, dt, steps, method=method)
    out = _host(c)
    m.set_timing(True)
    m.rk_step(c, dt, 2, method=method)
    kt = m.kernel_times()
    m.set_timing(False)
    m.device_status()
    return out, kt


@pytest.mark.parametrize("method", ["ssp_rk3", "rk2", "rk4"])
@pytest.mark.parametrize("p,ne,n", [(1, 0, 10), (2, 0, 8), (3, 0, 8), (3, 3, 7), (4, 0, 6), (5, 0, 5)])
def test_fused_equals_separate_launches(dgmod, p, ne, n, method):
    """Ragged last tiles (50 to 200 elements); 20 steps (a 16-step graph replay
    and plain steps on the separate-launch side)."""
    mesh = I.periodic_mesh(n)
    m = dgmod.Mesh.from_mesh(mesh, p, n_edge_pts=ne)
    c0 = m.project_function(I.perturbed_vortex)
    dt = I.fixed_dt(mesh, I.perturbed_vortex, p)
    a, kta = _run(m, c0, dt, 20, method, True)
    b, ktb = _run(m, c0, dt, 20, method, False)
    assert "stepper" in kta and kta["stepper"][0] == 1 and "element" not in kta
    assert "stepper" not in ktb and "element" in ktb
    assert np.array_equal(a, b)


@pytest.mark.parametrize("rule", ["collapsed", "symmetric"])
def test_fused_with_boundary_faces(dgmod, rule):
    """A closed box of walls and a channel with prescribed states on its sides."""
    import torch
    for mesh in (I.box_mesh(10), I.box_mesh(10, x_code=I.BC_STATE, y_code=I.BC_STATE)):
        m = dgmod.Mesh.from_mesh(mesh, 2, vol_rule=rule)
        if m.n_boundary:
            xy = m.boundary_points().cpu().numpy()
            m.set_boundary_state(torch.from_numpy(np.ascontiguousarray(I.steady_vortex(xy[..., 0], xy[..., 1]))).cuda())
        c0 = m.project_function(I.steady_vortex)
        dt = I.fixed_dt(mesh, I.steady_vortex, 2)
        a, kta = _run(m, c0, dt, 12, "ssp_rk3", True)
        b, _ = _run(m, c0, dt, 12, "ssp_rk3", False)
        assert "stepper" in kta
        assert np.array_equal(a, b)


@pytest.mark.parametrize("method", ["ssp_rk3", "rk2", "rk4"])
@pytest.mark.parametrize("n", [10, 16])
def test_fused_with_limiter(dgmod, n, method):
    """p = 1 with every stage limited (density steps: the limiter acts on most
    elements); 200 and 512 elements, ragged last tiles; no limiter launch on the
    fused side."""
    mesh = I.periodic_mesh(n)
    m = dgmod.Mesh.from_mesh(mesh, 1)
    c0 = m.limit(m.project_function(I.density_steps))
    dt = I.fixed_dt(mesh, I.density_steps, 1)
    m.set_limiter(True)
    a, kta = _run(m, c0, dt, 20, method, True)
    b, ktb = _run(m, c0, dt, 20, method, False)
    m.set_limiter(False)
    assert "stepper" in kta and "other" not in kta and "element" not in kta
    assert "stepper" not in ktb and "other" in ktb
    assert np.array_equal(a, b)
    try:
        free, _ = _run(m, c0, dt, 20, method, True)
        assert not np.array_equal(free, a)        # limiting changed the run
    except dgmod.DGError as e:
        assert dgmod.STATUS[e.status] == "DG_ENONPHYS"   # or, without it, the run broke down


def test_fused_matches_oracle(dgmod, oracle_mod):
    """The fused path against the oracle's SSP-RK3 run (relative L2 <= 1e-12)."""
    mesh = I.periodic_mesh(12)
    p = 3
    m = dgmod.Mesh.from_mesh(mesh, p)
    o = oracle_mod.OracleDG.from_mesh(mesh, p)
    dt = I.fixed_dt(mesh, I.perturbed_vortex, p)
    c = m.project_function(I.perturbed_vortex)
    m.set_timing(True)
    m.rk_step(c, dt, 25)
    assert "stepper" in m.kernel_times()
    m.set_timing(False)
    ref = o.ssp_rk3(o.project_ic(I.perturbed_vortex), dt, 25)
    got = _host(c)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12


def test_large_mesh_keeps_separate_launches(dgmod):
    """The fused stepper's tiles hold 4 or 8 elements, at most 4 blocks per SM;
    9,800 elements at p = 3 need 1,225 blocks of 8, more than one wave on 152 SMs:
    the separate launches run."""
    import torch
    mesh = I.periodic_mesh(70)
    m = dgmod.Mesh.from_mesh(mesh, 3)
    props = torch.cuda.get_device_properties(0)
    assert (m.N + 7) // 8 > 4 * props.multi_processor_count
    c = m.project_function(I.vortex)
    m.set_timing(True)
    m.rk_step(c, I.fixed_dt(mesh, I.vortex, 3), 2)
    kt = m.kernel_times()
    m.set_timing(False)
    assert "stepper" not in kt and kt["element"][0] == 6
