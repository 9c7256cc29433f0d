"""GPU parity of the paper's own time integrators (Section 4.3.1: classic RK2,
read as Heun's method, and the classical RK4) against the oracle, through
dg_rk_step_method.

The oracle takes RK4 in Butcher form with every stage derivative kept, the
library with a running sum of its stages (Heun's method is in Shu-Osher form on
both sides), so the two differ only in rounding order: relative L2 <= 1e-12 over
whole runs.
Runs of more than 16 steps go through the replayed CUDA graph.
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


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("method", ["rk2", "rk4"])
@pytest.mark.parametrize("p,ne,n,steps", [(1, 0, 16, 40), (2, 0, 6, 20), (3, 0, 16, 20), (3, 3, 8, 5),
                                          (4, 0, 8, 5), (5, 0, 6, 18)])
def test_classic_rk_parity(dgmod, oracle_mod, method, p, ne, n, steps):
    mesh = I.periodic_mesh(n)
    ic = I.vortex if p == 1 else I.perturbed_vortex
    dt = I.fixed_dt(mesh, ic, p)
    m = dgmod.Mesh.from_mesh(mesh, p, n_edge_pts=ne)
    o = oracle_mod.OracleDG.from_mesh(mesh, p, n_edge_pts=ne)
    c = m.project_function(ic)
    m.rk_step(c, dt, steps, method=method)
    m.device_status()
    ref = getattr(o, method)(o.project_ic(ic), dt, steps)
    assert rel_l2(_host(c), ref) < TOL, rel_l2(_host(c), ref)


@pytest.mark.parametrize("method", ["rk2", "rk4"])
def test_classic_rk_full_size_step(dgmod, oracle_mod, method):
    """One step of the 256 x 256, p = 3 workload in the launch configuration the
    benchmark times, against the oracle's step of the whole mesh."""
    mesh = I.periodic_mesh(256)
    p = 3
    dt = I.fixed_dt(mesh, I.vortex, p)
    m = dgmod.Mesh.from_mesh(mesh, p)
    o = oracle_mod.OracleDG.from_mesh(mesh, p)
    c = m.project_function(I.vortex)
    m.rk_step(c, dt, 1, method=method)
    m.device_status()
    ref = getattr(o, method)(o.project_ic(I.vortex), dt, 1)
    got = _host(c)
    assert rel_l2(got, ref) < TOL, rel_l2(got, ref)


@pytest.mark.parametrize("method", ["ssp_rk3", "rk2", "rk4"])
def test_methods_conserve_totals(dgmod, method):
    mesh = I.periodic_mesh(16)
    m = dgmod.Mesh.from_mesh(mesh, 3)
    c = m.project_function(I.perturbed_vortex)
    dt = I.fixed_dt(mesh, I.perturbed_vortex, 3)
    t0 = m.conserved_totals(c)
    m.rk_step(c, dt, 30, method=method)
    assert np.all(np.abs(m.conserved_totals(c) - t0) <= 1e-13 * np.abs(t0))


@pytest.mark.parametrize("method", ["rk2", "rk4"])
@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_graph_replay_matches_plain_launches(dgmod, method, prec):
    """A 40-step call (one plain step, two graph replays, seven plain steps) gives
    bit for bit the state of 40 one-step calls, for each method."""
    mesh = I.periodic_mesh(16)
    m = dgmod.Mesh.from_mesh(mesh, 2)
    c0 = m.project_function(I.perturbed_vortex)
    dt = I.fixed_dt(mesh, I.perturbed_vortex, 2)
    a = c0.clone(); b = c0.clone()
    m.rk_step(a, dt, 40, precision=prec, method=method)
    for _ in range(40):
        m.rk_step(b, dt, 1, precision=prec, method=method)
    m.device_status()
    assert np.array_equal(_host(a), _host(b))


@pytest.mark.parametrize("method", ["rk2", "rk4"])
@pytest.mark.parametrize("prec,tol", [("tf32x3", 1e-6), ("tf32x1", 1e-3)])
@pytest.mark.parametrize("p", [2, 4])
def test_mixed_classic_rk_vs_fp64(dgmod, method, p, prec, tol):
    """The tensor-core modes with the paper's steppers: state error against the
    float64 GPU run of the same method after 20 steps, within the bound the
    mixed modes meet with SSP-RK3."""
    mesh = I.periodic_mesh(32)
    m = dgmod.Mesh.from_mesh(mesh, p)
    c0 = m.project_function(I.perturbed_vortex)
    dt = I.fixed_dt(mesh, I.perturbed_vortex, p)
    a = c0.clone(); b = c0.clone()
    m.rk_step(a, dt, 20, precision="fp64", method=method)
    m.rk_step(b, dt, 20, precision=prec, method=method)
    m.device_status()
    A, B = _host(a), _host(b)
    assert np.linalg.norm(B - A) / np.linalg.norm(A) < tol


def test_unknown_method_rejected(dgmod):
    import ctypes
    mesh = I.periodic_mesh(4)
    m = dgmod.Mesh.from_mesh(mesh, 1)
    c = m.project_function(I.vortex)
    st = dgmod.load().dg_rk_step_method(m._h, ctypes.c_void_p(c.data_ptr()), 1e-3, 1, 7, 0, None)
    assert st == 1                                   # DG_EINVAL
    with pytest.raises(ValueError):
        m.rk_step(c, 1e-3, 1, method="rk3")
