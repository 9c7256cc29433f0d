"""Pins of the oracle's Barth-Jespersen limiter for p = 1 (Section 4.3.5).

What the paper fixes about the limited state, checked from point values this
test evaluates itself (at the centroid and at the edge integration points of
every element) and from the mesh's neighbour arrays:
  * no new extrema: at every edge integration point of element i, each variable
    lies within [U^min, U^max], the smallest and largest centroid values of i and
    its three neighbours (Eqs. limitmax, limitmin);
  * the limiting is as weak as that allows: where the linear part was scaled down
    (alpha < 1) an edge point sits on one of the bounds, and an element whose edge
    values were already within the bounds is left unchanged;
  * only the slope changes (Eq. limit): the centroid value and the direction of the
    gradient are kept and alpha lies in [0, 1];
  * limiting a limited state changes nothing.
Stage-by-stage limiting inside the time steppers keeps the domain integrals.
"""
import numpy as np
import pytest

from paper_1601_07944_gb300 import inputs as I

V = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])


def _edge_points(o):
    x, _ = o.edge_rule()
    r, s = [], []
    for q in range(3):
        a, b = V[q], V[(q + 1) % 3]
        pts = 0.5 * (1 - x)[:, None] * a + 0.5 * (1 + x)[:, None] * b
        r.append(pts[:, 0]); s.append(pts[:, 1])
    return np.concatenate(r), np.concatenate(s)


def _bounds(o, mesh, c):
    cen = o.eval_points(c, np.array([1.0 / 3]), np.array([1.0 / 3]))[:, 0, :]     # [N, 4]
    nb = cen[mesh.nbr]                                                           # [N, 3, 4]
    allv = np.concatenate([cen[:, None, :], nb], axis=1)
    return cen, allv.min(axis=1), allv.max(axis=1)


@pytest.fixture(scope="module", params=["random_slopes", "steps"])
def case(request, oracle_mod):
    mesh = I.periodic_mesh(8)
    o = oracle_mod.OracleDG.from_mesh(mesh, 1)
    if request.param == "random_slopes":
        c = o.project_ic(I.perturbed_vortex)
        rng = np.random.default_rng(11)
        c[:, :, 1:] += 0.05 * rng.standard_normal(c[:, :, 1:].shape)
    else:
        c = o.project_ic(I.density_steps)
    return mesh, o, c


def test_no_new_extrema_at_edge_points(case):
    mesh, o, c = case
    cl = o.limit(c)
    r, s = _edge_points(o)
    _, lo, hi = _bounds(o, mesh, c)
    u = o.eval_points(cl, r, s)                                  # [N, 3 ne, 4]
    tol = 1e-14 * (1.0 + np.abs(u))
    assert np.all(u <= hi[:, None, :] + tol) and np.all(u >= lo[:, None, :] - tol)


def test_limiting_is_as_weak_as_the_bounds_allow(case):
    mesh, o, c = case
    cl = o.limit(c)
    r, s = _edge_points(o)
    _, lo, hi = _bounds(o, mesh, c)
    u0 = o.eval_points(c, r, s)
    u1 = o.eval_points(cl, r, s)
    scale = 1e-12 * (1.0 + np.abs(u1).max(axis=1))
    g0 = np.linalg.norm(c[:, :, 1:], axis=2)
    g1 = np.linalg.norm(cl[:, :, 1:], axis=2)
    scaled = g1 < g0 * (1 - 1e-13)
    touch = np.minimum(np.abs(u1 - hi[:, None, :]), np.abs(u1 - lo[:, None, :])).min(axis=1)
    assert np.all(touch[scaled] <= scale[scaled])
    inside = np.all((u0 <= hi[:, None, :]) & (u0 >= lo[:, None, :]), axis=1)
    assert np.array_equal(c[inside], cl[inside])
    assert scaled.any() and inside.any()                       # both branches are exercised


def test_only_the_slope_changes(case):
    mesh, o, c = case
    cl = o.limit(c)
    assert np.array_equal(cl[:, :, 0], c[:, :, 0])
    g0 = c[:, :, 1:]
    num = np.sum(cl[:, :, 1:] * g0, axis=2)
    den = np.sum(g0 * g0, axis=2)
    alpha = np.where(den > 0, num / np.where(den > 0, den, 1.0), 1.0)
    assert np.all(alpha >= -1e-15) and np.all(alpha <= 1 + 1e-15)
    np.testing.assert_allclose(cl[:, :, 1:], alpha[..., None] * g0, rtol=0, atol=1e-15)


def test_idempotent(case):
    mesh, o, c = case
    cl = o.limit(c)
    np.testing.assert_allclose(o.limit(cl), cl, rtol=0, atol=1e-15)


@pytest.mark.parametrize("method", ["ssp_rk3", "rk2", "rk4"])
def test_limited_stepping_conserves_totals(oracle_mod, method):
    mesh = I.periodic_mesh(8)
    o = oracle_mod.OracleDG.from_mesh(mesh, 1)
    o.set_limiter(True)
    c0 = o.limit(o.project_ic(I.density_steps))
    dt = I.fixed_dt(mesh, I.density_steps, 1)
    t0 = o.totals(c0)
    c = getattr(o, method)(c0, dt, 10)
    assert np.all(np.abs(o.totals(c) - t0) <= 1e-13 * np.abs(t0).max())     # momenta start at 0
    o.set_limiter(False)
    assert not np.array_equal(getattr(o, method)(c0, dt, 10), c)   # the limiter acted


def test_limiter_needs_p1(oracle_mod):
    o = oracle_mod.OracleDG.from_mesh(I.periodic_mesh(4), 2)
    with pytest.raises(Exception):
        o.limit(o.project_ic(I.vortex))
