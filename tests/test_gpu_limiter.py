"""GPU parity of the Barth-Jespersen limiter (p = 1, Section 4.3.5) and of time
stepping with every stage limited (Section 4.3.1), against the oracle.

Both sides start from the same coefficients (the oracle's projection, copied to
the device), so the limiter sees the same inputs on both; they then differ only
in rounding order (relative L2 <= 1e-12).  Sizes: 16 x 16 (512 elements, two
resident blocks' worth of threads and a ragged last block) and 64 x 64.
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


def _state(o, kind):
    if kind == "steps":
        return o.project_ic(I.density_steps)
    c = o.project_ic(I.perturbed_vortex)
    rng = np.random.default_rng(11)
    c[:, :, 1:] += 0.05 * rng.standard_normal(c[:, :, 1:].shape)
    return c


@pytest.mark.parametrize("kind", ["steps", "random_slopes"])
@pytest.mark.parametrize("n", [16, 64])
def test_limit_parity(dgmod, oracle_mod, kind, n):
    mesh = I.periodic_mesh(n)
    o = oracle_mod.OracleDG.from_mesh(mesh, 1)
    m = dgmod.Mesh.from_mesh(mesh, 1)
    c0 = _state(o, kind)
    ref = o.limit(c0)
    got = _host(m.limit(_dev(c0)))
    assert rel_l2(got, ref) < TOL, rel_l2(got, ref)
    assert np.array_equal(got[:, :, 0], c0[:, :, 0])          # means untouched
    assert not np.array_equal(ref, c0)                        # the limiter acted


@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("method", ["ssp_rk3", "rk2", "rk4"])
@pytest.mark.parametrize("kind", ["steps", "random_slopes"])
def test_limited_stepping_parity(dgmod, oracle_mod, method, kind, fused):
    """20 steps: in one launch of the fused small-mesh stepper (its limiter phase),
    or as separate launches (one plain step, then a replayed 16-step graph and
    three more)."""
    mesh = I.periodic_mesh(16)
    o = oracle_mod.OracleDG.from_mesh(mesh, 1)
    m = dgmod.Mesh.from_mesh(mesh, 1)
    m.set_small_mesh_stepper(fused)
    c0 = o.limit(_state(o, kind))
    dt = I.fixed_dt(mesh, I.density_steps, 1)
    o.set_limiter(True)
    m.set_limiter(True)
    ref = getattr(o, method)(c0, dt, 20)
    c = _dev(c0)
    m.rk_step(c, dt, 20, method=method)
    m.device_status()
    got = _host(c)
    assert rel_l2(got, ref) < TOL, rel_l2(got, ref)
    o.set_limiter(False)
    with np.errstate(all="ignore"):
        free = getattr(o, method)(c0, dt, 20)     # unlimited (on the steps it breaks down)
    assert not np.array_equal(free, ref)          # limiting changed the run


def test_limited_graph_replay_matches_plain_launches(dgmod, oracle_mod):
    mesh = I.periodic_mesh(16)
    o = oracle_mod.OracleDG.from_mesh(mesh, 1)
    m = dgmod.Mesh.from_mesh(mesh, 1)
    c0 = o.limit(o.project_ic(I.density_steps))
    dt = I.fixed_dt(mesh, I.density_steps, 1)
    m.set_small_mesh_stepper(False)        # the separate launches and their graph
    m.set_limiter(True)
    a = _dev(c0); b = _dev(c0)
    m.rk_step(a, dt, 40)
    for _ in range(40):
        m.rk_step(b, dt, 1)
    assert np.array_equal(_host(a), _host(b))
    # switching the limiter off drops the captured graph: the run equals plain launches again
    m.set_limiter(False)
    m.rk_step(a, dt, 20)
    for _ in range(20):
        m.rk_step(b, dt, 1)
    assert np.array_equal(_host(a), _host(b))


def test_limiter_errors(dgmod):
    mesh = I.periodic_mesh(8)
    m2 = dgmod.Mesh.from_mesh(mesh, 2)
    with pytest.raises(dgmod.DGError) as e:
        m2.set_limiter(True)
    assert e.value.status == 1                                 # DG_EINVAL
    c2 = m2.project_function(I.vortex)
    with pytest.raises(dgmod.DGError):
        m2.limit(c2)
    m = dgmod.Mesh.from_mesh(mesh, 1)
    m.set_limiter(True)
    c = m.project_function(I.vortex)
    dt = I.fixed_dt(mesh, I.vortex, 1)
    with pytest.raises(dgmod.DGError) as e:
        m.rk_step(c, dt, 1, precision="tf32x3")
    assert e.value.status == 7                                 # DG_ENOTIMPL
    with pytest.raises(dgmod.DGError) as e:
        m.adjoint_step(c, dt, c.clone())
    assert e.value.status == 7
