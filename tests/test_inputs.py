"""Pins of the seeded input generators (mesh, random stream, initial data)."""
import numpy as np

from paper_1601_07944_gb300 import inputs as I


def test_splitmix64_published_vector():
    # SplitMix64 seeded with 0: the first outputs of the published generator.
    z = I.splitmix64(0, 3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_range():
    u = I.uniform01(7, 10000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.02


def _area2(xy):
    a, b, c = xy[:, 0], xy[:, 1], xy[:, 2]
    return (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])


def test_mesh_invariants():
    for n in (2, 3, 8, 16):
        m = I.periodic_mesh(n)
        N = m.n_elem
        assert N == 2 * n * n
        a2 = _area2(m.elem_xy)
        assert np.all(a2 > 0)                                   # counter-clockwise
        assert abs(a2.sum() / 2 - 100.0) < 1e-12 * 100         # tiles [-5,5]^2
        e = np.arange(N)[:, None].repeat(3, 1)
        q = np.arange(3)[None, :].repeat(N, 0)
        f, qf = m.nbr, m.nbr_face.astype(np.int64)
        assert np.all(m.nbr[f, qf] == e) and np.all(m.nbr_face[f, qf] == q)
        # the shared edge is the neighbour's edge reversed, up to a period shift
        xy = m.elem_xy
        p0 = xy[e, q]; p1 = xy[e, (q + 1) % 3]
        r0 = xy[f, qf]; r1 = xy[f, (qf + 1) % 3]
        s0 = p0 - r1; s1 = p1 - r0
        assert np.allclose(s0, s1, atol=1e-12)
        k = s0 / 10.0
        assert np.allclose(k, np.round(k), atol=1e-12)


def test_jitter_bounds_and_boundary_lattice():
    n = 16
    m0 = I.periodic_mesh(n, jitter=0.0)
    m1 = I.periodic_mesh(n)
    d = np.abs(m1.elem_xy - m0.elem_xy)
    assert d.max() <= 0.1 * m1.h + 1e-14
    assert d.max() > 0.05 * m1.h
    # vertex 0 of triangle 0 of square (0, j) or (i, 0) lies on the lattice
    xy = m1.elem_xy.reshape(n, n, 2, 3, 2)
    assert np.all(xy[0, :, 0, 0, 1] == -5.0)
    assert np.all(xy[:, 0, 0, 0, 0] == -5.0)


def test_vortex_closed_form():
    # centre: u, v equal to the free stream; density and pressure at their minimum
    U = I.vortex(np.array([0.0]), np.array([0.0]))[0]
    g = 1.4
    T0 = 1.0 - (g - 1) * 25.0 / (8 * g * np.pi ** 2) * np.e
    rho0 = T0 ** (1 / (g - 1))
    assert abs(U[0] - rho0) < 1e-15
    assert abs(U[1] / U[0] - 1.0) < 1e-15 and abs(U[2] / U[0] - 1.0) < 1e-15
    # isentropic: p = rho^gamma everywhere
    x = np.linspace(-5, 5, 37)
    X, Y = np.meshgrid(x, x)
    rho, u, v, p = I.vortex_primitive(X, Y)
    assert np.allclose(p, rho ** g, rtol=1e-14)
    # translation by (t, t)
    a = I.vortex(X, Y, t=1.3)
    b = I.vortex(X - 1.3, Y - 1.3)
    assert np.allclose(a, b, rtol=1e-13, atol=1e-14)


def test_fourier_perturbation_normalised():
    a, th = I.fourier_coefficients()
    assert np.allclose(np.abs(a).reshape(2, -1).sum(1), 1.0)
    assert th.min() >= 0 and th.max() < 2 * np.pi
    x = np.random.default_rng(0).uniform(-5, 5, 1000)
    d = I.fourier_perturbation(x, x[::-1], a, th, 1e-2)
    assert np.abs(d).max() <= 1e-2 + 1e-15
    # periodic on the period-10 domain
    d2 = I.fourier_perturbation(x + 10, x[::-1] - 10, a, th, 1e-2)
    assert np.allclose(d, d2, atol=1e-15)
