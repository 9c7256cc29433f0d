"""Degenerate and boundary-size cases of the GPU path against the oracle.

  * one triangle closed by walls on all three sides (N = 1: a single, partly
    empty tile, three boundary faces and no interior face);
  * a square of two triangles with walls and prescribed states (one interior
    face);
  * the smallest periodic mesh the generator makes (2 x 2 squares, 8 elements);
  * zero steps: the state is left untouched, bit for bit, in every mode.
Float64 parity: relative L2 <= 1e-12, on both volume rules; the 3xTF32 RHS on
the tiny meshes within the mixed-mode bound 2e-6 (||R|| + ||V||), V the volume
term.
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


def _wavy(x, y):
    r = 1.0 + 0.1 * np.sin(x + 2.0 * y)
    return I.primitive_to_conserved(r, 0.1 * np.cos(y), -0.05 * np.sin(x), 1.0 + 0.05 * np.cos(x))


class _Mesh:
    def __init__(self, xy, nbr, nf):
        self.elem_xy = np.asarray(xy, np.float64)
        self.nbr = np.asarray(nbr, np.int64)
        self.nbr_face = np.asarray(nf, np.int8)
        self.n_elem = self.elem_xy.shape[0]


def _triangle():
    return _Mesh([[[-1.0, -0.8], [1.2, -0.5], [0.1, 1.1]]], [[I.BC_WALL] * 3], [[-1] * 3])


def _square():
    # (a, b, c) and (a, c, d) of the unit square, split along a-c: face 2 of the
    # first (c -> a) is face 0 of the second (a -> c)
    a, b, c, d = (0.0, 0.0), (1.0, 0.0), (1.0, 1.0), (0.0, 1.0)
    return _Mesh([[a, b, c], [a, c, d]], [[I.BC_WALL, I.BC_STATE, 1], [0, I.BC_WALL, I.BC_STATE]],
                 [[-1, -1, 0], [2, -1, -1]])


def _pair(dgmod, oracle_mod, mesh, p, rule, ic):
    m = dgmod.Mesh.from_mesh(mesh, p, vol_rule=rule)
    o = oracle_mod.OracleDG.from_mesh(mesh, p, vol_rule=rule)
    if m.n_boundary and (np.asarray(mesh.nbr) == I.BC_STATE).any():
        xy = _host(m.boundary_points())
        m.set_boundary_state(_dev(ic(xy[..., 0], xy[..., 1])))
        oxy = o.boundary_points()
        o.set_boundary_state(ic(oxy[..., 0], oxy[..., 1]))
    return m, o


@pytest.mark.parametrize("rule", ["collapsed", "symmetric"])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("kind", ["triangle", "square", "periodic2"])
def test_tiny_meshes(dgmod, oracle_mod, kind, p, rule):
    mesh = {"triangle": _triangle, "square": _square, "periodic2": lambda: I.periodic_mesh(2)}[kind]()
    m, o = _pair(dgmod, oracle_mod, mesh, p, rule, _wavy)
    c0 = o.project_ic(_wavy)
    got = _host(m.rhs(_dev(c0)))
    ref, vol = o.rhs_and_volume(c0)
    assert rel_l2(got, ref) < TOL, rel_l2(got, ref)
    # the tensor-core path on the same tiny mesh (one partly empty tile), within
    # the 3xTF32 bound of the mixed-mode tests: 2e-6 (||R|| + ||V||)
    mixed = _host(m.rhs(_dev(c0), precision="tf32x3"))
    assert np.linalg.norm(mixed - ref) <= 2e-6 * (np.linalg.norm(ref) + np.linalg.norm(vol))
    dt = 2e-3
    for method in ("ssp_rk3", "rk4"):
        c = _dev(c0)
        m.rk_step(c, dt, 18, method=method)
        m.device_status()
        ref = getattr(o, method)(c0, dt, 18)
        assert rel_l2(_host(c), ref) < TOL
    if kind == "triangle":
        # closed by walls: mass and energy stay put
        c = _dev(c0)
        t0 = m.conserved_totals(c)
        m.rk_step(c, dt, 18)
        t1 = m.conserved_totals(c)
        assert abs(t1[0] - t0[0]) <= 1e-14 * abs(t0[0]) and abs(t1[3] - t0[3]) <= 1e-14 * abs(t0[3])


@pytest.mark.parametrize("p", [1, 3])
def test_tiny_mesh_adjoint(dgmod, oracle_mod, p):
    mesh = _square()
    m, o = _pair(dgmod, oracle_mod, mesh, p, "collapsed", _wavy)
    c0 = o.project_ic(_wavy)
    lam = np.random.default_rng(4).standard_normal(c0.shape)
    got = _host(m.adjoint_step(_dev(c0), 2e-3, _dev(lam)))
    ref = o.ssp_rk3_vjp(c0, 2e-3, lam)
    assert rel_l2(got, ref) < TOL


@pytest.mark.parametrize("prec", ["fp64", "tf32x3", "tf32x1"])
@pytest.mark.parametrize("method", ["ssp_rk3", "rk2", "rk4"])
def test_zero_steps_is_a_no_op(dgmod, method, prec):
    mesh = I.periodic_mesh(8)
    m = dgmod.Mesh.from_mesh(mesh, 2)
    c = m.project_function(I.perturbed_vortex)
    before = _host(c).copy()
    m.rk_step(c, 1e-3, 0, precision=prec, method=method)
    m.device_status()
    assert np.array_equal(_host(c), before)
