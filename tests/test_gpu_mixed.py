"""Mixed-precision path (tcgen05 TF32 tensor-core contractions) on the GPU.

Error model: the contractions run on TF32 inputs with FP32 accumulation, the
volume flux in FP32.  The RHS is the small difference of the volume and surface
terms, so its error is measured against the size of those terms (the oracle's
volume term V / det J):
    3xTF32: ||R_mixed - R|| <= 2e-6 (||R|| + ||V||)   (FP32-level arithmetic)
    1xTF32: ||R_mixed - R|| <= 4e-3 (||R|| + ||V||)   (10-bit TF32 mantissa)
The edge traces come from the tensor-core contraction (float32 accumulation) in
dg_rhs as in every Runge-Kutta stage; the edge flux is evaluated from them in
float64 (its dissipation coefficient alpha included), and the mean mode is
lifted in float64 from each edge's float64 flux integral, which its two elements
take with opposite signs.  So the conserved totals drift only at float64
rounding, while the mean mode's error follows the traces': it is bounded at the
mode's tolerance against the size of the surface term S / det J = V / det J - R.
"""
import numpy as np
import pytest

from paper_1601_07944_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"tf32x3": 2e-6, "tf32x1": 4e-3}
CASES = [(1, 0), (2, 0), (3, 0), (3, 3), (4, 0), (5, 0)]


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


def test_arithmetic_helpers_match_hardware(dgmod):
    assert dgmod.self_test() == (0, 0, 0, 0)


@pytest.mark.parametrize("prec", ["tf32x3", "tf32x1"])
@pytest.mark.parametrize("n", [6, 16])
@pytest.mark.parametrize("p,ne", CASES)
def test_mixed_rhs_vs_oracle(dgmod, oracle_mod, p, ne, n, prec):
    mesh = I.periodic_mesh(n)
    m = dgmod.Mesh.from_mesh(mesh, p, n_edge_pts=ne)
    o = oracle_mod.OracleDG.from_mesh(mesh, p, n_edge_pts=ne)
    c = o.project_ic(I.perturbed_vortex)
    ref, vol = o.rhs_and_volume(c)
    got = _host(m.rhs(_dev(c), precision=prec))
    m.device_status()
    err = np.linalg.norm(got - ref)
    assert err <= TOL[prec] * (np.linalg.norm(ref) + np.linalg.norm(vol)), err / np.linalg.norm(ref)
    # mean mode: no volume term, so its error is the surface term's, whose inputs
    # (the traces) carry the contraction's rounding
    assert np.abs(got[:, :, 0] - ref[:, :, 0]).max() <= TOL[prec] * np.abs(vol - ref).max()


@pytest.mark.parametrize("prec", ["tf32x3", "tf32x1"])
def test_mixed_conservation_and_determinism(dgmod, prec):
    mesh = I.periodic_mesh(16)
    p = 3
    m = dgmod.Mesh.from_mesh(mesh, p)
    c0 = m.project_function(I.perturbed_vortex)
    dt = I.fixed_dt(mesh, I.perturbed_vortex, p)
    t0 = m.conserved_totals(c0)
    a = c0.clone(); b = c0.clone()
    m.rk_step(a, dt, 30, precision=prec)
    m.rk_step(b, dt, 30, precision=prec)
    m.device_status()
    assert np.array_equal(_host(a), _host(b))
    t1 = m.conserved_totals(a)
    assert np.all(np.abs(t1 - t0) <= 1e-13 * np.abs(t0))


@pytest.mark.parametrize("prec,tol", [("tf32x3", 1e-6), ("tf32x1", 1e-3)])
@pytest.mark.parametrize("p", [2, 4])
def test_mixed_state_vs_fp64(dgmod, p, prec, tol):
    """State error of the mixed run against the float64 GPU run after 20 steps."""
    mesh = I.periodic_mesh(32)
    m = dgmod.Mesh.from_mesh(mesh, p)
    c0 = m.project_function(I.perturbed_vortex)
    dt = I.fixed_dt(mesh, I.perturbed_vortex, p)
    a = c0.clone(); b = c0.clone()
    m.rk_step(a, dt, 20, precision="fp64")
    m.rk_step(b, dt, 20, precision=prec)
    m.device_status()
    A, B = _host(a), _host(b)
    assert np.linalg.norm(B - A) / np.linalg.norm(A) < tol


# -- full size: more tiles than resident CTAs ---------------------------------
# The tensor-core element kernel runs a resident grid (at most 8 CTAs per SM, so
# at most 1,216 CTAs on 152 SMs) whose CTAs loop over 32-element tiles, loading
# the next tile's inputs one tile ahead and carrying the mbarrier phase across
# tiles; the edge-flux kernel gives each block an equal slice of the edges.  The
# 256^2 (4,096 tiles) and 512^2 (16,384 tiles) meshes make every CTA run many
# tiles, in the launch configuration the benchmark times.

_ORACLE = {}


def _oracle_rhs(oracle_mod, n, p, rule):
    key = (n, p, rule)
    if key not in _ORACLE:
        _ORACLE.clear()
        mesh = I.periodic_mesh(n)
        o = oracle_mod.OracleDG.from_mesh(mesh, p, vol_rule=rule)
        ic = I.vortex if (n, p) == (256, 3) else I.perturbed_vortex
        c = o.project_ic(ic)
        ref, vol = o.rhs_and_volume(c)
        _ORACLE[key] = (mesh, o, ic, c, ref, vol)
    return _ORACLE[key]


@pytest.mark.parametrize("prec", ["tf32x3", "tf32x1"])
@pytest.mark.parametrize("n,p,rule", [(256, 3, "collapsed"), (512, 4, "collapsed"), (256, 3, "symmetric")])
def test_mixed_full_size_rhs_vs_oracle(dgmod, oracle_mod, n, p, rule, prec):
    mesh, o, _, c, ref, vol = _oracle_rhs(oracle_mod, n, p, rule)
    m = dgmod.Mesh.from_mesh(mesh, p, vol_rule=rule)
    assert (m.N + 31) // 32 > 152 * 8                 # many tiles per CTA
    got = _host(m.rhs(_dev(c), precision=prec))
    m.device_status()
    err = np.linalg.norm(got - ref)
    assert err <= TOL[prec] * (np.linalg.norm(ref) + np.linalg.norm(vol)), err / np.linalg.norm(ref)
    assert np.abs(got[:, :, 0] - ref[:, :, 0]).max() <= TOL[prec] * np.abs(vol - ref).max()
    # the same call again: bit for bit (one writer per output slot, no atomics)
    assert np.array_equal(got, _host(m.rhs(_dev(c), precision=prec)))


@pytest.mark.parametrize("prec", ["tf32x3", "tf32x1"])
@pytest.mark.parametrize("rule", ["collapsed", "symmetric"])
def test_mixed_full_size_step_vs_oracle(dgmod, oracle_mod, rule, prec):
    """One SSP-RK3 step of the 256^2 p=3 vortex in a tensor-core mode against the
    oracle's float64 step: the increment c1 - c0 = dt (k1/6 + k2/6 + 2 k3/3) carries
    each stage's RHS error with weights summing to one, so it is bounded by dt
    times the RHS bound (twice, for the stages' inputs differing from the
    oracle's); the state itself within the mode's state bound."""
    mesh, o, ic, c, ref, vol = _oracle_rhs(oracle_mod, 256, 3, rule)
    m = dgmod.Mesh.from_mesh(mesh, 3, vol_rule=rule)
    dt = I.fixed_dt(mesh, ic, 3)
    want = o.ssp_rk3(c, dt, 1)
    cd = _dev(c)
    m.rk_step(cd, dt, 1, precision=prec)
    m.device_status()
    got = _host(cd)
    inc_err = np.linalg.norm((got - c) - (want - c))
    assert inc_err <= 2 * TOL[prec] * dt * (np.linalg.norm(ref) + np.linalg.norm(vol)), inc_err
    state_tol = {"tf32x3": 1e-6, "tf32x1": 1e-3}[prec]
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < state_tol
