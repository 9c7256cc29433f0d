"""Pins of the oracle's time integrators: SSP-RK3 and the paper's own classic
RK2 (Heun) and RK4 (Section 4.3.1).

The semi-discrete system dc/dt = L(c) (Eq. 2ddg0) is integrated on a small mesh
by scipy's DOP853 (an independent, adaptive eighth-order library integrator) at
a tolerance far below the Runge-Kutta errors; the error of each method against
it must fall as dt^q with q its order (2, 3, 4) when dt is halved.  A dropped
stage or a wrong weight or node lowers the observed order.  Any Runge-Kutta
method keeps the domain integrals of a conservative discretisation, so the
totals must stay at rounding level as well.
"""
import numpy as np
import pytest

from paper_1601_07944_gb300 import inputs as I

ORDERS = {"rk2": 2, "ssp_rk3": 3, "rk4": 4}


@pytest.fixture(scope="module")
def setup(oracle_mod):
    # The density wave is smooth and resolved, so the jumps at the edges, where the
    # Lax-Friedrichs flux has its kinks (|v.n| and the max of the wave speeds), are
    # small; on an under-resolved vortex those kinks cap the observed order of RK4.
    mesh = I.periodic_mesh(8)
    p = 2
    o = oracle_mod.OracleDG.from_mesh(mesh, p)
    c0 = o.project_ic(I.density_wave)
    dt = 2.0 * I.fixed_dt(mesh, I.density_wave, p)
    steps = 8
    T = steps * dt
    integrate = pytest.importorskip("scipy.integrate")
    shape = c0.shape
    sol = integrate.solve_ivp(lambda t, y: o.rhs(y.reshape(shape)).ravel(), (0.0, T), c0.ravel(),
                              method="DOP853", rtol=1e-13, atol=1e-15)
    assert sol.success
    exact = sol.y[:, -1].reshape(shape)
    return o, c0, dt, steps, exact


@pytest.mark.parametrize("method", sorted(ORDERS))
def test_temporal_order_against_library_integrator(setup, method):
    o, c0, dt, steps, exact = setup
    step = getattr(o, method)
    errs = []
    for r in (1, 2, 4):
        c = step(c0, dt / r, steps * r)
        errs.append(np.linalg.norm(c - exact) / np.linalg.norm(exact))
    q = ORDERS[method]
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[-1] > 1e-13, errs           # still above the reference's own error
    for r in rates:
        assert q - 0.2 <= r <= q + 0.5, (method, errs, rates)


@pytest.mark.parametrize("method", ["rk2", "rk4"])
def test_classic_rk_conserves_totals(oracle_mod, method):
    mesh = I.periodic_mesh(8)
    o = oracle_mod.OracleDG.from_mesh(mesh, 2)
    c0 = o.project_ic(I.perturbed_vortex)
    dt = I.fixed_dt(mesh, I.perturbed_vortex, 2)
    t0 = o.totals(c0)
    c = getattr(o, method)(c0, dt, 20)
    assert np.all(np.abs(o.totals(c) - t0) <= 1e-13 * np.abs(t0))
