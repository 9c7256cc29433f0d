"""Pins of the fully symmetric degree-2p volume rules (Section 4.3.2 asks for
rules of degree 2p; Section 6.1 counts 3 points at p = 1 and 16 at p = 4) and of the oracle's
solver running on them.

Facts checked, none of them a re-run of the derivation:
  * exactness: every monomial r^i s^j of degree <= 2p integrates to its exact
    value, computed here by symbolic integration over the triangle (sympy);
  * the rule is a rule of the stated kind: point counts 3/6/12/16/25, weights
    positive and summing to the area 1/2, points strictly inside, and the set
    of weighted points invariant under all six permutations of the vertices;
  * p = 1: the classical three-point rule, points (1/6, 1/6), (2/3, 1/6),
    (1/6, 2/3) with weights 1/6 (closed form);
  * the basis is orthonormal under the rule (Gram = I, degree 2p products);
  * the DG solver on the rule: free-stream preservation, exact discrete
    conservation, and order p+1 on the exact density wave;
  * provenance: the seeded multi-start search (oracle/search_symmetric_rules.py,
    float64 Levenberg-Marquardt on orthogonal-basis moments from random orbit
    parameters) finds, as the rule farthest from the edges, the one the start
    values lead to, and it agrees with the 50-digit solution.
"""
import math

import numpy as np
import pytest

from paper_1601_07944_gb300 import inputs as I

COUNTS = {1: 3, 2: 6, 3: 12, 4: 16, 5: 25}


@pytest.fixture(scope="module")
def rules():
    from oracle.symmetric_rules import symmetric_rule
    return {p: symmetric_rule(p) for p in COUNTS}


@pytest.fixture(scope="module")
def exact_moments():
    sp = pytest.importorskip("sympy")
    r, s = sp.symbols("r s")
    out = {}
    for i in range(11):
        for j in range(11 - i):
            out[(i, j)] = float(sp.integrate(sp.integrate(r ** i * s ** j, (r, 0, 1 - s)), (s, 0, 1)))
    return out


@pytest.mark.parametrize("p", sorted(COUNTS))
def test_exact_to_degree_2p(rules, exact_moments, p):
    r, s, w = rules[p]
    for i in range(2 * p + 1):
        for j in range(2 * p + 1 - i):
            got = float(np.sum(w * r ** i * s ** j))
            ex = exact_moments[(i, j)]
            assert abs(got - ex) <= 2e-15 * ex + 1e-17, (p, i, j, got, ex)


@pytest.mark.parametrize("p", sorted(COUNTS))
def test_rule_shape(rules, p):
    r, s, w = rules[p]
    assert r.size == s.size == w.size == COUNTS[p]
    assert np.all(w > 0)
    assert abs(w.sum() - 0.5) < 1e-15
    assert np.all(r > 0) and np.all(s > 0) and np.all(1 - r - s > 0)


@pytest.mark.parametrize("p", sorted(COUNTS))
def test_invariant_under_vertex_permutations(rules, p):
    r, s, w = rules[p]
    lam = np.stack([1 - r - s, r, s], 1)
    key = np.round(np.c_[lam, w], 12)
    base = sorted(map(tuple, key))
    for perm in [(0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]:
        other = sorted(map(tuple, np.round(np.c_[lam[:, perm], w], 12)))
        assert np.allclose(np.array(other), np.array(base), atol=1e-12)


def test_p1_is_the_classical_three_point_rule(rules):
    r, s, w = rules[1]
    got = sorted(zip(np.round(r, 15), np.round(s, 15)))
    want = sorted([(1 / 6, 1 / 6), (2 / 3, 1 / 6), (1 / 6, 2 / 3)])
    assert np.allclose(np.array(got), np.array(want), atol=1e-15)
    assert np.allclose(w, 1 / 6, atol=1e-15)


@pytest.mark.parametrize("p", sorted(COUNTS))
def test_basis_orthonormal_under_rule(oracle_mod, p):
    o = oracle_mod.OracleDG.from_mesh(I.periodic_mesh(2), p, vol_rule="symmetric")
    assert o.nq == COUNTS[p]
    r, s, w = o.volume_rule()
    phi, _, _ = o.volume_tables()
    G = phi.T @ (w[:, None] * phi)
    # 2e-15: a rule whose points are off by 1e-14 (a float64 solve of the
    # ill-conditioned moment system) already misses this by 100x at p = 5
    assert np.abs(G - np.eye(o.np)).max() < 2e-15


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_free_stream_preservation_symmetric(oracle_mod, p):
    o = oracle_mod.OracleDG.from_mesh(I.periodic_mesh(8), p, vol_rule="symmetric")
    c = o.project_ic(lambda x, y: I.uniform_state(x, y))
    assert np.abs(o.rhs(c)).max() < 1e-13


def test_conservation_symmetric(oracle_mod):
    m = I.periodic_mesh(8)
    o = oracle_mod.OracleDG.from_mesh(m, 2, vol_rule="symmetric")
    c = o.project_ic(I.perturbed_vortex)
    t0 = o.totals(c)
    c1 = o.ssp_rk3(c, I.fixed_dt(m, I.perturbed_vortex, 2), 30)
    assert np.all(np.abs(o.totals(c1) - t0) <= 1e-13 * np.abs(t0))
    assert np.abs(c1 - c).max() > 1e-3


@pytest.mark.parametrize("p,ns", [(1, (8, 16, 32)), (2, (8, 16, 32)), (3, (4, 8, 16))])
def test_density_wave_convergence_symmetric(oracle_mod, p, ns):
    T = 0.4
    dt = min(I.fixed_dt(I.periodic_mesh(n), I.density_wave, p) for n in ns) * 0.5
    steps = int(math.ceil(T / dt))
    dt = T / steps
    errs = []
    for n in ns:
        o = oracle_mod.OracleDG.from_mesh(I.periodic_mesh(n), p, vol_rule="symmetric")
        c = o.ssp_rk3(o.project_ic(I.density_wave), dt, steps)
        errs.append(o.l2_error(c, lambda x, y: I.density_wave(x, y, T)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert rates[-1] > p + 1 - 0.2 and min(rates) > p + 1 - 0.5, (errs, rates)


def test_rules_differ_from_collapsed_grid(oracle_mod):
    """The symmetric rule really replaces the grid: a nonlinear RHS changes (by
    the aliasing error of the flux quadrature), a polynomial-flux state does not."""
    m = I.periodic_mesh(8)
    a = oracle_mod.OracleDG.from_mesh(m, 3)
    b = oracle_mod.OracleDG.from_mesh(m, 3, vol_rule="symmetric")
    assert (a.nq, b.nq) == (16, 12)
    c = a.project_ic(I.perturbed_vortex)
    ra, rb = a.rhs(c), b.rhs(c)
    d = np.linalg.norm(ra - rb) / np.linalg.norm(ra)
    assert 1e-12 < d < 1e-2
    # rho and p linear, velocity constant: the flux is linear in position and
    # both rules integrate the volume term exactly
    kw = dict(rho0=1.0, rx=0.02, ry=-0.015, u=0.4, v=-0.3, p0=1.0, px=0.03, py=0.05)
    cl = a.project_ic(lambda x, y: I.linear_state(x, y, **kw))
    assert np.abs(a.rhs(cl) - b.rhs(cl)).max() < 1e-13


@pytest.mark.parametrize("p", sorted(COUNTS))
def test_start_values_come_from_the_search(rules, p):
    """START (three significant digits) is the search's chosen rule rounded, and
    that rule is the 50-digit rule to float64 search accuracy."""
    from oracle import search_symmetric_rules as S
    found = S.search(p)
    assert found, "no positive-interior rule found"
    can, mb = found[0]
    assert S.as_start(can) == [(k, tuple(v)) for k, v in S.START[p]]
    # the chosen rule's points and weights against the oracle's rule (same orbit
    # order as START after canonical sorting: compare as sets of weighted points)
    x = []
    for o in can:
        x += list(o[1:])
    bary, w = S._points([o[0] for o in can], np.array(x))
    r, s_, wr = rules[p]
    assert len(w) == len(wr)
    for k in range(len(wr)):        # every point of the oracle's rule, found with its weight
        d = np.hypot(bary[:, 1] - r[k], bary[:, 2] - s_[k])
        j = int(np.argmin(d))
        assert d[j] < 1e-9 and abs(w[j] - wr[k]) < 1e-9

