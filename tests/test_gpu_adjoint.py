"""GPU discrete adjoint against the oracle's reverse sweep and central
differences, through the C ABI (dg_adjoint_step) and the checkpointed
torch.autograd wrapper."""
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


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("n", [6, 16])
@pytest.mark.parametrize("p,ne", [(1, 0), (2, 0), (3, 0), (3, 3), (4, 0), (5, 0)])
def test_adjoint_step_parity(dgmod, oracle_mod, p, ne, n):
    mesh = I.periodic_mesh(n)
    m = dgmod.Mesh.from_mesh(mesh, p, n_edge_pts=ne)
    o = oracle_mod.OracleDG.from_mesh(mesh, p, n_edge_pts=ne)
    rng = np.random.default_rng(n + 10 * p)
    c = o.project_ic(I.perturbed_vortex)
    c = c + 0.002 * rng.standard_normal(c.shape)
    lam = rng.standard_normal(c.shape)
    dt = I.fixed_dt(mesh, I.perturbed_vortex, p)
    ref = o.ssp_rk3_vjp(c, dt, lam)
    got = _host(m.adjoint_step(_dev(c), dt, _dev(lam)))
    assert rel_l2(got, ref) < 1e-12


@pytest.mark.parametrize("n", [6, 16])
@pytest.mark.parametrize("p,ne", [(1, 0), (2, 0), (3, 0), (3, 3), (4, 0), (5, 0)])
def test_rhs_adjoint_parity(dgmod, oracle_mod, p, ne, n):
    mesh = I.periodic_mesh(n)
    m = dgmod.Mesh.from_mesh(mesh, p, n_edge_pts=ne)
    o = oracle_mod.OracleDG.from_mesh(mesh, p, n_edge_pts=ne)
    rng = np.random.default_rng(3 * n + p)
    c = o.project_ic(I.perturbed_vortex) + 0.002 * rng.standard_normal((o.N, 4, o.np))
    lam = rng.standard_normal(c.shape)
    got = _host(m.rhs_adjoint(_dev(c), _dev(lam)))
    assert rel_l2(got, o.rhs_vjp(c, lam)) < 1e-12


@pytest.mark.parametrize("n", [6, 16, 128])
@pytest.mark.parametrize("p,ne", [(1, 0), (2, 0), (3, 0), (5, 0)])
def test_stored_stages_bitwise(dgmod, p, ne, n):
    """dg_rk_step_stages gives dg_rk_step's new state bit for bit, and
    dg_adjoint_step_stages on its stage values gives dg_adjoint_step's lam_n bit
    for bit (6 x 6 and 16 x 16 run the fused small-mesh stepper in dg_rk_step,
    128 x 128 the separate launches)."""
    import torch
    mesh = I.periodic_mesh(n)
    m = dgmod.Mesh.from_mesh(mesh, p, n_edge_pts=ne)
    rng = np.random.default_rng(7 * n + p)
    c = m.project_function(I.perturbed_vortex)
    lam = _dev(rng.standard_normal(tuple(c.shape)))
    dt = I.fixed_dt(mesh, I.perturbed_vortex, p)
    a, b = c.clone(), c.clone()
    u1, u2 = torch.empty_like(c), torch.empty_like(c)
    m.rk_step(a, dt, 1)
    m.rk_step_stages(b, dt, u1, u2)
    assert np.array_equal(_host(a), _host(b))
    ref = _host(m.adjoint_step(c, dt, lam))
    got = _host(m.adjoint_step_stages(c, u1, u2, dt, lam))
    m.device_status()
    assert np.array_equal(got, ref)


def test_stored_stages_errors(dgmod):
    import torch
    mesh = I.periodic_mesh(6)
    m = dgmod.Mesh.from_mesh(mesh, 1)
    c = m.project_function(I.vortex)
    u = torch.empty_like(c)
    with pytest.raises(dgmod.DGError):
        m.rk_step_stages(c, 1e-3, u, u)              # u1 and u2 the same buffer
    with pytest.raises(dgmod.DGError):
        m.rk_step_stages(c, 1e-3, c, u)              # u1 aliases c
    with pytest.raises(dgmod.DGError):
        m.adjoint_step_stages(c, u, u, 1e-3, c, out=u)   # lam_n aliases a stage
    m.set_limiter(True)
    with pytest.raises(dgmod.DGError):
        m.rk_step_stages(c, 1e-3, u, torch.empty_like(c))
    m.set_limiter(False)


def _loss_setup(dgmod, oracle_mod, n, p):
    mesh = I.periodic_mesh(n)
    m = dgmod.Mesh.from_mesh(mesh, p)
    dt = I.fixed_dt(mesh, I.perturbed_vortex, p)
    c0 = m.project_function(I.perturbed_vortex)
    tgt0 = m.project_function(lambda x, y: I.perturbed_vortex(x, y, seed=I.SEED_TARGET))
    return mesh, m, dt, c0, tgt0


@pytest.mark.parametrize("keep_stages", [True, False])
def test_autograd_matches_oracle_reverse_sweep(dgmod, oracle_mod, keep_stages):
    """40 steps, checkpoints every 8: the gradient of the density misfit with
    respect to c0 equals the oracle's step-by-step reverse sweep, with the stage
    values kept by the recomputation or recomputed by each transposed step."""
    import torch
    from paper_1601_07944_gb300 import autograd as AG
    n, p, steps, every = 16, 2, 40, 8
    mesh, m, dt, c0, tgt0 = _loss_setup(dgmod, oracle_mod, n, p)
    target = tgt0.clone()
    m.rk_step(target, dt, steps)
    dJ = m.det_j()
    x = c0.clone().requires_grad_(True)
    loss = AG.density_misfit(dJ, AG.solve(m, x, dt, steps, every, keep_stages=keep_stages), target)
    loss.backward()
    g = _host(x.grad)
    # oracle reverse sweep from the same c0 and target
    o = oracle_mod.OracleDG.from_mesh(mesh, p)
    cn = _host(c0)
    states = [cn]
    for _ in range(steps):
        states.append(o.ssp_rk3(states[-1], dt, 1))
    lam = np.zeros_like(cn)
    dj = o.det_j()
    lam[:, 0, :] = dj[:, None] * (states[-1][:, 0, :] - _host(target)[:, 0, :])
    for s in range(steps - 1, -1, -1):
        lam = o.ssp_rk3_vjp(states[s], dt, lam)
    assert rel_l2(g, lam) < 1e-11


@pytest.mark.parametrize("n,p,steps,every,nfd", [(16, 2, 40, 8, 16), (256, 2, 400, 20, 32)])
def test_autograd_central_differences(dgmod, oracle_mod, n, p, steps, every, nfd):
    """Gradient of the density misfit against central differences (h = 1e-6) on
    random coefficients; the 256^2, p=2, 400-step, every-20 case is the full
    differentiation workload."""
    import torch
    from paper_1601_07944_gb300 import autograd as AG
    mesh, m, dt, c0, tgt0 = _loss_setup(dgmod, oracle_mod, n, p)
    target = tgt0.clone()
    m.rk_step(target, dt, steps)
    dJ = m.det_j()

    def loss_of(c):
        cT = c.clone()
        m.rk_step(cT, dt, steps)
        return float(AG.density_misfit(dJ, cT, target).item())

    x = c0.clone().requires_grad_(True)
    L = AG.density_misfit(dJ, AG.solve(m, x, dt, steps, every), target)
    L.backward()
    g = _host(x.grad)
    rng = np.random.default_rng(I.SEED_FD)
    h = 1e-6
    # a central difference of a loss computed in float64 carries a rounding
    # error of about eps L / h; below that floor no relative check is possible
    floor = 100 * np.finfo(float).eps * float(L.item()) / h
    strong = 0
    for flat in rng.choice(c0.numel(), nfd, replace=False):
        idx = np.unravel_index(flat, tuple(c0.shape))
        cp = c0.clone(); cp[idx] += h
        cm = c0.clone(); cm[idx] -= h
        g_fd = (loss_of(cp) - loss_of(cm)) / (2 * h)
        assert abs(g_fd - g[idx]) <= 1e-6 * abs(g[idx]) + floor, (idx, g_fd, g[idx], floor)
        strong += abs(g[idx]) > 1e3 * floor
    # coefficients of the density's low modes carry gradients far above the floor:
    # there the agreement is 1e-6 relative or better
    for j in range(3):
        idx = (int(rng.integers(0, c0.shape[0])), 0, j)
        cp = c0.clone(); cp[idx] += h
        cm = c0.clone(); cm[idx] -= h
        g_fd = (loss_of(cp) - loss_of(cm)) / (2 * h)
        assert abs(g_fd - g[idx]) <= 1e-6 * abs(g[idx]) + floor, (idx, g_fd, g[idx], floor)
        strong += abs(g[idx]) > 1e3 * floor
    # the relative criterion was exercised: at least the mean-mode coefficients'
    # gradients stand three orders above the rounding floor
    assert strong >= 1, (strong, floor)
    idx0 = (int(rng.integers(0, c0.shape[0])), 0, 0)
    assert abs(g[idx0]) > 1e3 * floor, (g[idx0], floor)
