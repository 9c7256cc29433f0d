"""Pins of the oracle's quadrature rules and orthonormal basis.

The oracle is checked against facts fixed by mathematics, never against itself:
textbook Gauss nodes, exact monomial integrals, orthonormality, the closed forms
of the constant and linear modes, and finite differences of the gradients.
"""
import math

import numpy as np
import pytest


def test_gauss_legendre_textbook(oracle_mod):
    O = oracle_mod
    x, w = O.gauss_legendre(2)
    assert np.allclose(x, [-1 / math.sqrt(3), 1 / math.sqrt(3)], atol=1e-15)
    assert np.allclose(w, [1.0, 1.0], atol=1e-15)
    x, w = O.gauss_legendre(3)
    assert np.allclose(x, [-math.sqrt(0.6), 0.0, math.sqrt(0.6)], atol=1e-15)
    assert np.allclose(w, [5 / 9, 8 / 9, 5 / 9], atol=1e-15)


@pytest.mark.parametrize("n", range(1, 9))
def test_gauss_legendre_exactness(oracle_mod, n):
    x, w = oracle_mod.gauss_legendre(n)
    assert np.all(np.diff(x) > 0)
    assert np.allclose(x, -x[::-1], atol=1e-15)          # symmetric: reversal k -> n+1-k
    for k in range(2 * n):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.dot(w, x ** k) - exact) < 1e-14
    # and not exact one degree higher
    k = 2 * n
    assert abs(np.dot(w, x ** k) - 2.0 / (k + 1)) > 1e-6


@pytest.mark.parametrize("n", range(1, 9))
def test_gauss_jacobi_10_exactness(oracle_mod, n):
    # weight (1-x): int_{-1}^{1} (1-x) x^k dx = 2/(k+1) [k even] - 2/(k+2) [k odd]
    x, w = oracle_mod.gauss_jacobi(n, 1.0, 0.0)
    for k in range(2 * n):
        exact = (2.0 / (k + 1)) if k % 2 == 0 else (-2.0 / (k + 2))
        assert abs(np.dot(w, x ** k) - exact) < 1e-14


@pytest.mark.parametrize("n", range(1, 8))
def test_stroud_monomials(oracle_mod, n):
    r, s, w = oracle_mod.stroud(n)
    assert abs(w.sum() - 0.5) < 1e-15
    assert np.all(r > 0) and np.all(s > 0) and np.all(r + s < 1)   # interior points
    for a in range(2 * n):
        for b in range(2 * n - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs(np.dot(w, r ** a * s ** b) - exact) < 1e-15


@pytest.mark.parametrize("p", range(0, 7))
def test_basis_orthonormal(oracle_mod, p):
    O = oracle_mod
    np_ = (p + 1) * (p + 2) // 2
    G = O.dubiner_gram_exact(p)
    assert np.abs(G - np.eye(np_)).max() < 1e-15
    r, s, w = O.stroud(p + 1)                 # exact to degree 2p+1
    phi, _, _ = O.dubiner(p, r, s)
    assert np.abs(phi.T @ (w[:, None] * phi) - np.eye(np_)).max() < 2e-15


@pytest.mark.parametrize("p", range(0, 7))
def test_basis_hierarchy_and_span(oracle_mod, p):
    """Mode j has total degree d_j (ordered by degree) and the modes span all
    polynomials of degree <= p."""
    O = oracle_mod
    C = O.dubiner_monomials(p)
    K = C.shape[1]
    np_ = C.shape[0]
    degs = [d for d in range(p + 1) for _ in range(d + 1)]
    X, Y = np.meshgrid(np.arange(K), np.arange(K), indexing="ij")
    for j in range(np_):
        assert np.all(C[j][X + Y > degs[j]] == 0.0)
        assert np.any(C[j][X + Y == degs[j]] != 0.0)
    mask = (X + Y) <= p
    M = np.stack([C[j][mask] for j in range(np_)])
    assert np.linalg.matrix_rank(M) == np_


def test_basis_closed_forms(oracle_mod):
    """phi_1 = sqrt(2); phi_2 = sqrt(12) (2r + s - 1); phi_3 = 2 (3s - 1).

    These follow by hand from the collapsed-coordinate definition: psi_10 =
    P_1(alpha)(1-s) = 2r + s - 1 and psi_01 = P_1^{(1,0)}(2s-1) = 3s - 1, with
    int (2r+s-1)^2 = 1/12 and int (3s-1)^2 = 1/4 over the reference triangle."""
    rng = np.random.default_rng(5)
    r = rng.uniform(0, 0.5, 50)
    s = rng.uniform(0, 0.5, 50)
    phi, dr, ds = oracle_mod.dubiner(1, r, s)
    assert np.allclose(phi[:, 0], math.sqrt(2), atol=1e-15)
    assert np.allclose(phi[:, 1], math.sqrt(12) * (2 * r + s - 1), atol=1e-14)
    assert np.allclose(phi[:, 2], 2 * (3 * s - 1), atol=1e-14)
    assert np.allclose(dr[:, 1], 2 * math.sqrt(12)) and np.allclose(ds[:, 1], math.sqrt(12))
    assert np.allclose(dr[:, 2], 0.0) and np.allclose(ds[:, 2], 6.0)


@pytest.mark.parametrize("p", [2, 5])
def test_basis_gradients_finite_difference(oracle_mod, p):
    rng = np.random.default_rng(p)
    r = rng.uniform(0.05, 0.45, 20)
    s = rng.uniform(0.05, 0.45, 20)
    h = 1e-5
    _, dr, ds = oracle_mod.dubiner(p, r, s)
    fp, _, _ = oracle_mod.dubiner(p, r + h, s)
    fm, _, _ = oracle_mod.dubiner(p, r - h, s)
    assert np.abs((fp - fm) / (2 * h) - dr).max() < 1e-6 * max(1, np.abs(dr).max())
    fp, _, _ = oracle_mod.dubiner(p, r, s + h)
    fm, _, _ = oracle_mod.dubiner(p, r, s - h)
    assert np.abs((fp - fm) / (2 * h) - ds).max() < 1e-6 * max(1, np.abs(ds).max())


@pytest.mark.parametrize("p", range(0, 6))
def test_basis_integrals(oracle_mod, p):
    I = oracle_mod.dubiner_integrals(p)
    assert abs(I[0] - math.sqrt(0.5)) < 2.3e-16
    assert np.abs(I[1:]).max(initial=0.0) < 1e-16
