"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports every
entry point include/dg.h declares, its own quadrature and basis tables agree with
the oracle's independent ones, and mesh validation rejects bad meshes before any
device work."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1601_07944_gb300 import _build, dg, inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return dg.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "dg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dg_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert "dg_rhs" in names and "dg_rk_step" in names and "dg_adjoint_step" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(dg.EXPORTS)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_host_tables_match_oracle(lib, oracle_mod, p):
    T = dg.host_tables(p)
    r, s, w = oracle_mod.stroud(p + 1)
    assert np.abs(T["vol_r"] - r).max() < 2.3e-16
    assert np.abs(T["vol_s"] - s).max() < 2.3e-16
    assert np.abs(T["vol_w"] - w).max() < 2.3e-16
    x, we = oracle_mod.gauss_legendre(p + 1)
    assert np.abs(T["edge_x"] - x).max() < 2.3e-16
    assert np.abs(T["edge_w"] - we).max() < 2.3e-16
    # volume tables: both sides evaluate at the exact images of the rounded 1D nodes
    o = oracle_mod.OracleDG.from_mesh(I.periodic_mesh(2), p)
    phi, dr, ds = o.volume_tables()

    def rel(a, b):
        return np.abs(a - b).max() / np.abs(b).max()
    # both sides evaluate in extended precision at the same double points
    assert rel(T["phi"], phi) < 4e-16
    assert rel(T["dphi_r"], dr) < 4e-16
    assert rel(T["dphi_s"], ds) < 4e-16
    xi = T["edge_x"]
    V = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    for q in range(3):
        pts = 0.5 * (1 - xi)[:, None] * V[q] + 0.5 * (1 + xi)[:, None] * V[(q + 1) % 3]
        pf, _, _ = oracle_mod.dubiner(p, pts[:, 0], pts[:, 1])
        assert rel(T["phi_face"][q], pf) < 4e-16


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_collapsed_grid_alpha_nodes_are_mirror_pairs(lib, p):
    """The float64 element kernels fold their alpha sums on mirror pairs of
    nodes (P_a(-x) = (-1)^a P_a(x)); that needs the library's alpha nodes to be
    symmetric about 0 with equal weights, and the middle node of an odd count at
    0, to rounding."""
    T = dg.host_tables(p)
    nd = p + 1
    r = T["vol_r"].reshape(nd, nd)          # point index ib * nd + ia
    s = T["vol_s"].reshape(nd, nd)
    w = T["vol_w"].reshape(nd, nd)
    beta = 2.0 * s - 1.0
    alpha = 4.0 * r / (1.0 - beta) - 1.0
    # alpha recovered from the rounded points: the rounding of r grows by 4 / (1 - beta)
    tol = 8 * np.finfo(float).eps / (1.0 - beta).min()
    assert np.abs(alpha - alpha[:1, :]).max() < tol           # the same alpha nodes on every beta line
    assert np.abs(alpha + alpha[:, ::-1]).max() < tol         # alpha_{nd-1-ia} = -alpha_ia
    assert np.abs(w - w[:, ::-1]).max() <= 4 * np.finfo(float).eps * np.abs(w).max()
    if nd % 2:
        assert np.abs(alpha[:, nd // 2]).max() < tol


def test_host_tables_p3_three_edge_points(lib, oracle_mod):
    T = dg.host_tables(3, 3)
    x, w = oracle_mod.gauss_legendre(3)
    assert np.abs(T["edge_x"] - x).max() < 1e-15 and np.abs(T["edge_w"] - w).max() < 1e-15


def _create(lib, xy, nbr, nf, p=2, ne=0, rule=0):
    xy = np.ascontiguousarray(xy, np.float64)
    nbr = np.ascontiguousarray(nbr, np.int64)
    nf = np.ascontiguousarray(nf, np.int8)
    desc = dg._Desc(xy.shape[0], xy.ctypes.data, nbr.ctypes.data, nf.ctypes.data, p, ne, 1.4, rule)
    h = ctypes.c_void_p()
    st = lib.dg_mesh_create(ctypes.byref(desc), ctypes.byref(h))
    return st, lib.dg_last_error().decode()


def test_mesh_validation_errors(lib):
    m = I.periodic_mesh(4)
    xy = m.elem_xy.copy()
    xy[3] = xy[3][::-1]                           # clockwise element
    st, msg = _create(lib, xy, m.nbr, m.nbr_face)
    assert st == 4 and "counter-clockwise" in msg
    nbr = m.nbr.copy()
    nbr[5, 1] = (nbr[5, 1] + 1) % m.n_elem          # asymmetric neighbour
    st, msg = _create(lib, m.elem_xy, nbr, m.nbr_face)
    assert st == 4 and "symmetric" in msg
    nbr = m.nbr.copy()
    nbr[0, 0] = I.BC_WALL                         # a wall on one side of an interior face only
    st, msg = _create(lib, m.elem_xy, nbr, m.nbr_face)
    assert st == 4 and "symmetric" in msg
    b = I.box_mesh(4)
    nbr = b.nbr.copy()
    nbr[nbr == I.BC_WALL] = -7                    # not a boundary code
    st, msg = _create(lib, b.elem_xy, nbr, b.nbr_face)
    assert st == 4 and "boundary code" in msg
    xy = m.elem_xy.copy()
    xy[7, 1] += 1e-3                              # edge no longer matches its neighbour's
    xy[7, 1] -= 0.0
    st, msg = _create(lib, xy, m.nbr, m.nbr_face)
    assert st == 4
    st, msg = _create(lib, m.elem_xy, m.nbr, m.nbr_face, p=7)
    assert st == 1 and "unsupported" in msg
    st, msg = _create(lib, m.elem_xy, m.nbr, m.nbr_face, p=2, ne=5)
    assert st == 1
    st, msg = _create(lib, m.elem_xy, m.nbr, m.nbr_face, rule=2)
    assert st == 1 and "vol_rule" in msg


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_symmetric_rule_matches_oracle(lib, p):
    """The library derives the symmetric rule on its own (extended precision,
    orthonormal-basis moments) and must land on the oracle's rule (50-digit
    decimal, monomial moments) in the same point order."""
    from oracle.symmetric_rules import symmetric_rule
    r, s, w, phi = dg.volume_rule(p, "symmetric")
    R, S, W = symmetric_rule(p)
    assert r.size == {1: 3, 2: 6, 3: 12, 4: 16, 5: 25}[p]
    assert np.abs(r - R).max() <= 2e-16 and np.abs(s - S).max() <= 2e-16 and np.abs(w - W).max() <= 3e-17
    # the basis values at the points agree with the oracle's evaluation there
    o_phi = oracle_basis(p, r, s)
    assert np.abs(phi - o_phi).max() < 1e-13
    # and the collapsed grid is the one dg_host_tables reports
    rc, sc, wc, _ = dg.volume_rule(p, "collapsed")
    T = dg.host_tables(p)
    assert np.array_equal(rc, T["vol_r"]) and np.array_equal(wc, T["vol_w"])
    nq = ctypes.c_int()
    assert lib.dg_volume_rule(p, 5, ctypes.byref(nq), None, None, None, None) == 1
    assert lib.dg_volume_rule(9, 1, ctypes.byref(nq), None, None, None, None) == 1


def oracle_basis(p, r, s):
    import oracle
    return oracle.dubiner(p, r, s)[0]


def test_null_arguments(lib):
    assert lib.dg_mesh_create(None, None) == 1
    assert lib.dg_rhs(None, None, None, 0, None) == 1
    assert lib.dg_mesh_destroy(None) == 0
