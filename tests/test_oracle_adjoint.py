"""Pins of the oracle's discrete adjoint (reverse sweep of the RHS and of one
SSP-RK3 step).

  * the Euler flux is homogeneous of degree one, F_n(U) = (dF_n/dU) U, which pins
    the hand-derived flux Jacobian without differentiating anything;
  * the Lax-Friedrichs Jacobians match central differences away from the kinks;
  * the full RHS Jacobian assembled from transposed products equals the one from
    central differences on a rough state (so every transposition is right);
  * the dot-product test <lam, J v> = <J^T lam, v> for one SSP-RK3 step;
  * the gradient of the density misfit through several steps matches central
    differences on random coefficients.
"""
import numpy as np
import pytest

from paper_1601_07944_gb300 import inputs as I


def _rough(o, mesh, seed, amp=0.003):
    rng = np.random.default_rng(seed)
    c = o.project_ic(I.perturbed_vortex)
    return c + amp * rng.standard_normal(c.shape)


def test_flux_jacobian_homogeneity(oracle_mod):
    rng = np.random.default_rng(0)
    for _ in range(20):
        U = I.primitive_to_conserved(*rng.uniform([0.5, -1, -1, 0.5], [1.5, 1, 1, 1.5]))
        th = rng.uniform(0, 2 * np.pi)
        nx, ny = np.cos(th), np.sin(th)
        J = oracle_mod.flux_jacobian(U, nx, ny)
        F1, F2 = oracle_mod.euler_flux(U)
        assert np.allclose(J @ U, F1 * nx + F2 * ny, rtol=1e-14, atol=1e-14)


def test_lax_friedrichs_jacobians_fd(oracle_mod):
    rng = np.random.default_rng(1)
    h = 1e-7
    for _ in range(10):
        U = I.primitive_to_conserved(*rng.uniform([0.5, -1, -1, 0.5], [1.5, 1, 1, 1.5]))
        V = I.primitive_to_conserved(*rng.uniform([0.5, -1, -1, 0.5], [1.5, 1, 1, 1.5]))
        th = rng.uniform(0, 2 * np.pi)
        nx, ny = np.cos(th), np.sin(th)
        Jl, Jr = oracle_mod.lax_friedrichs_jacobians(U, V, nx, ny)
        LF = oracle_mod.lax_friedrichs
        fl = np.stack([(LF(U + h * e, V, nx, ny) - LF(U - h * e, V, nx, ny)) / (2 * h) for e in np.eye(4)], 1)
        fr = np.stack([(LF(U, V + h * e, nx, ny) - LF(U, V - h * e, nx, ny)) / (2 * h) for e in np.eye(4)], 1)
        assert np.abs(fl - Jl).max() < 1e-7 * max(1, np.abs(Jl).max())
        assert np.abs(fr - Jr).max() < 1e-7 * max(1, np.abs(Jr).max())


@pytest.mark.parametrize("rule", ["collapsed", "symmetric"])
@pytest.mark.parametrize("p", [1, 2])
def test_rhs_jacobian_transpose(oracle_mod, p, rule):
    """Central-difference Jacobian of the RHS against the reverse sweep, on both
    volume rules (the sweep's volume term runs over whatever rule is installed)."""
    mesh = I.periodic_mesh(3)
    o = oracle_mod.OracleDG.from_mesh(mesh, p, vol_rule=rule)
    c = _rough(o, mesh, 7)
    n = c.size
    eps = 1e-6
    Jfd = np.zeros((n, n))
    for i in range(n):
        e = np.zeros(n); e[i] = eps
        e = e.reshape(c.shape)
        Jfd[:, i] = ((o.rhs(c + e) - o.rhs(c - e)) / (2 * eps)).ravel()
    Jad = np.zeros((n, n))
    for i in range(n):
        lam = np.zeros(n); lam[i] = 1.0
        Jad[i, :] = o.rhs_vjp(c, lam.reshape(c.shape)).ravel()
    assert np.abs(Jfd - Jad).max() < 1e-8 * np.abs(Jfd).max()


@pytest.mark.parametrize("p", [1, 2])
def test_rhs_jacobian_transpose_with_boundaries(oracle_mod, p):
    """Walls on x = +-5 (the ghost is the reflected interior trace) and prescribed
    states on y = +-5 (a ghost independent of the solution)."""
    mesh = I.box_mesh(3, x_code=I.BC_WALL, y_code=I.BC_STATE)
    o = oracle_mod.OracleDG.from_mesh(mesh, p)
    xy = o.boundary_points()
    o.set_boundary_state(I.steady_vortex(xy[..., 0], xy[..., 1]))
    c = _rough(o, mesh, 8)
    n = c.size
    eps = 1e-6
    Jfd = np.zeros((n, n))
    for i in range(n):
        e = np.zeros(n); e[i] = eps
        e = e.reshape(c.shape)
        Jfd[:, i] = ((o.rhs(c + e) - o.rhs(c - e)) / (2 * eps)).ravel()
    Jad = np.zeros((n, n))
    for i in range(n):
        lam = np.zeros(n); lam[i] = 1.0
        Jad[i, :] = o.rhs_vjp(c, lam.reshape(c.shape)).ravel()
    assert np.abs(Jfd - Jad).max() < 1e-8 * np.abs(Jfd).max()


def test_rk_step_dot_product(oracle_mod):
    mesh = I.periodic_mesh(6)
    o = oracle_mod.OracleDG.from_mesh(mesh, 2)
    c = _rough(o, mesh, 3)
    dt = I.fixed_dt(mesh, I.perturbed_vortex, 2)
    rng = np.random.default_rng(9)
    lam = rng.standard_normal(c.shape)
    v = rng.standard_normal(c.shape)
    eps = 1e-6
    jv = (o.ssp_rk3(c + eps * v, dt, 1) - o.ssp_rk3(c - eps * v, dt, 1)) / (2 * eps)
    a = float(np.sum(lam * jv))
    b = float(np.sum(o.ssp_rk3_vjp(c, dt, lam) * v))
    assert abs(a - b) <= 1e-8 * abs(b)


def test_misfit_gradient_fd(oracle_mod):
    """L(c0) = 1/2 sum_e det J_e sum_j (c_rho(T) - c_rho_target)^2 after k steps;
    the reverse sweep over the steps gives dL/dc0."""
    mesh = I.periodic_mesh(4)
    p, k = 2, 4
    o = oracle_mod.OracleDG.from_mesh(mesh, p)
    c0 = _rough(o, mesh, 5, amp=0.002)
    dt = I.fixed_dt(mesh, I.perturbed_vortex, p)
    target = o.ssp_rk3(o.project_ic(lambda x, y: I.perturbed_vortex(x, y, seed=I.SEED_TARGET)), dt, k)
    dJ = o.det_j()

    def loss(c):
        cT = o.ssp_rk3(c, dt, k)
        return 0.5 * float(np.sum(dJ[:, None] * (cT[:, 0, :] - target[:, 0, :]) ** 2))

    states = [c0]
    for _ in range(k):
        states.append(o.ssp_rk3(states[-1], dt, 1))
    lam = np.zeros_like(c0)
    lam[:, 0, :] = dJ[:, None] * (states[-1][:, 0, :] - target[:, 0, :])
    for s in range(k - 1, -1, -1):
        lam = o.ssp_rk3_vjp(states[s], dt, lam)
    rng = np.random.default_rng(4)
    h = 1e-6
    gmax = np.abs(lam).max()
    for flat in rng.choice(c0.size, 12, replace=False):
        idx = np.unravel_index(flat, c0.shape)
        cp = c0.copy(); cp[idx] += h
        cm = c0.copy(); cm[idx] -= h
        g_fd = (loss(cp) - loss(cm)) / (2 * h)
        assert abs(g_fd - lam[idx]) <= 1e-6 * max(abs(lam[idx]), 1e-3 * gmax), (idx, g_fd, lam[idx])
