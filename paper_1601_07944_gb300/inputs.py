"""Seeded synthetic workloads: jittered periodic triangle meshes and initial data.

This module generates *inputs* only.  It holds none of the discontinuous Galerkin
method's arithmetic (no basis, quadrature, geometry, flux or time stepping), so
both the CPU oracle and the CUDA path can take their meshes and initial states
from it.  Everything here is a plain function of a seed.

Mesh (stand-in for the paper's unstructured GMSH meshes, Section 5): the periodic
square [-5, 5]^2 is cut into n x n squares of side h = 10/n; square (i, j) has
corners a=(i,j), b=(i+1,j), c=(i+1,j+1), d=(i,j+1) and is split along a-c into
the counter-clockwise triangles (a,b,c) and (a,c,d).  Vertices with
1 <= i, j <= n-1 are moved by independent uniform offsets in [-0.1h, 0.1h]; the
vertices on the domain boundary stay on the lattice so that the periodic cell is
exactly [-5, 5]^2.  Coordinates are stored per element and *unwrapped*: a vertex
index that wraps past n-1 back to 0 is placed at +10, so each triangle is a
genuine triangle in the plane and the shared edge of a periodic neighbour is a
translate of this element's edge.

Random numbers come from SplitMix64 (state += 0x9E3779B97F4A7C15, then the
published SplitMix64 finaliser); a uniform double is (next() >> 11) * 2^-53.
Jitter draws run j outer, i inner, dx then dy, over the interior vertices only.

Element e = 2*(j*n + i) + t holds triangle t of square (i, j).  Local face q of an
element runs from its vertex q to vertex (q+1) mod 3.  ``nbr[e, q]`` is the
element across face q and ``nbr_face[e, q]`` that neighbour's local index of the
same edge.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

GAMMA = 1.4
DOMAIN_LO = -5.0
DOMAIN_L = 10.0

# Seeds of the workloads: mesh jitter, Fourier perturbation, adjoint target,
# finite-difference index selection.
SEED_MESH = 1
SEED_PERTURB = 2
SEED_TARGET = 3
SEED_FD = 4


def splitmix64(seed: int, count: int) -> np.ndarray:
    """The first ``count`` SplitMix64 outputs for ``seed`` (uint64 array).

    The k-th output (k = 1, 2, ...) mixes state seed + k*golden, so the stream is
    evaluated in closed form without a sequential loop.
    """
    k = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + k * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) from SplitMix64: (next() >> 11) * 2^-53."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


class Mesh:
    """A periodic jittered split-square triangle mesh (host arrays)."""

    def __init__(self, n: int, elem_xy: np.ndarray, nbr: np.ndarray, nbr_face: np.ndarray,
                 jitter: float, seed: int):
        self.n = n
        self.elem_xy = elem_xy          # float64 [N, 3, 2], CCW, unwrapped per element
        self.nbr = nbr                  # int64   [N, 3]
        self.nbr_face = nbr_face        # int8    [N, 3]
        self.jitter = jitter
        self.seed = seed

    @property
    def n_elem(self) -> int:
        return int(self.elem_xy.shape[0])

    @property
    def h(self) -> float:
        return DOMAIN_L / self.n


def periodic_mesh(n: int, jitter: float = 0.1, seed: int = SEED_MESH) -> Mesh:
    """Jittered periodic mesh of 2 n^2 triangles on [-5, 5]^2 (see module doc)."""
    if n < 2:
        raise ValueError("periodic_mesh needs n >= 2")
    h = DOMAIN_L / n
    vx = DOMAIN_LO + h * np.arange(n, dtype=np.float64)[None, :].repeat(n, 0)   # [j, i]
    vy = DOMAIN_LO + h * np.arange(n, dtype=np.float64)[:, None].repeat(n, 1)
    if jitter != 0.0:
        m = n - 1
        u = uniform01(seed, 2 * m * m).reshape(m, m, 2)        # [j-1, i-1, (dx, dy)]
        d = (2.0 * u - 1.0) * (jitter * h)
        vx[1:, 1:] += d[:, :, 0]
        vy[1:, 1:] += d[:, :, 1]

    jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")

    def vert(i, j):
        # unwrapped position of lattice vertex (i, j) with 0 <= i, j <= n
        iw, jw = i % n, j % n
        x = vx[jw, iw] + DOMAIN_L * (i // n)
        y = vy[jw, iw] + DOMAIN_L * (j // n)
        return np.stack([x, y], axis=-1)

    a = vert(ii, jj)
    b = vert(ii + 1, jj)
    c = vert(ii + 1, jj + 1)
    d = vert(ii, jj + 1)
    N = 2 * n * n
    xy = np.empty((n, n, 2, 3, 2), dtype=np.float64)
    xy[:, :, 0, 0], xy[:, :, 0, 1], xy[:, :, 0, 2] = a, b, c
    xy[:, :, 1, 0], xy[:, :, 1, 1], xy[:, :, 1, 2] = a, c, d
    xy = xy.reshape(N, 3, 2)

    def eid(i, j, t):
        return 2 * ((j % n) * n + (i % n)) + t

    nbr = np.empty((n, n, 2, 3), dtype=np.int64)
    nf = np.empty((n, n, 2, 3), dtype=np.int8)
    # triangle (a,b,c): face 0 = a->b (bottom), 1 = b->c (right), 2 = c->a (diagonal)
    nbr[:, :, 0, 0] = eid(ii, jj - 1, 1); nf[:, :, 0, 0] = 1
    nbr[:, :, 0, 1] = eid(ii + 1, jj, 1); nf[:, :, 0, 1] = 2
    nbr[:, :, 0, 2] = eid(ii, jj, 1);     nf[:, :, 0, 2] = 0
    # triangle (a,c,d): face 0 = a->c (diagonal), 1 = c->d (top), 2 = d->a (left)
    nbr[:, :, 1, 0] = eid(ii, jj, 0);     nf[:, :, 1, 0] = 2
    nbr[:, :, 1, 1] = eid(ii, jj + 1, 0); nf[:, :, 1, 1] = 0
    nbr[:, :, 1, 2] = eid(ii - 1, jj, 0); nf[:, :, 1, 2] = 1
    return Mesh(n, xy, nbr.reshape(N, 3), nf.reshape(N, 3), jitter, seed)


# boundary codes of nbr (the element "across" a boundary face): a solid wall, or a
# state prescribed by the caller at the face's quadrature points
BC_WALL = -1
BC_STATE = -2


def box_mesh(n: int, x_code: int = BC_WALL, y_code: int = BC_WALL, jitter: float = 0.1,
             seed: int = SEED_MESH) -> Mesh:
    """The jittered mesh of periodic_mesh (same vertices, triangles and jitter)
    with the faces on x = -5, 5 given the boundary code x_code and those on
    y = -5, 5 the code y_code (0 keeps that direction periodic).  A boundary face
    has nbr = code (< 0) and nbr_face = -1.  The domain-edge vertices are not
    jittered, so the boundary is the square's sides exactly."""
    mesh = periodic_mesh(n, jitter, seed)
    nbr = mesh.nbr.reshape(n, n, 2, 3).copy()
    nf = mesh.nbr_face.reshape(n, n, 2, 3).copy()
    if x_code:
        nbr[:, n - 1, 0, 1] = x_code; nf[:, n - 1, 0, 1] = -1      # right side, face b->c
        nbr[:, 0, 1, 2] = x_code;     nf[:, 0, 1, 2] = -1          # left side, face d->a
    if y_code:
        nbr[0, :, 0, 0] = y_code;     nf[0, :, 0, 0] = -1          # bottom, face a->b
        nbr[n - 1, :, 1, 1] = y_code; nf[n - 1, :, 1, 1] = -1      # top, face c->d
    N = mesh.n_elem
    return Mesh(n, mesh.elem_xy, nbr.reshape(N, 3), nf.reshape(N, 3), jitter, seed)


# ----------------------------------------------------------------------------
# Initial data (functions of physical position), returned as conserved
# variables (rho, rho*u, rho*v, E) with E = p/(gamma-1) + rho*(u^2+v^2)/2.
# ----------------------------------------------------------------------------

def primitive_to_conserved(rho, u, v, p, gamma: float = GAMMA) -> np.ndarray:
    rho = np.asarray(rho, dtype=np.float64)
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return np.stack([rho, rho * u, rho * v, E + 0.0 * rho], axis=-1)


def _wrap(d):
    """Nearest periodic image of a displacement on the period-10 domain."""
    return d - DOMAIN_L * np.floor((d + 0.5 * DOMAIN_L) / DOMAIN_L)


def vortex_primitive(x, y, t: float = 0.0, beta: float = 5.0, gamma: float = GAMMA):
    """Isentropic vortex (strength beta, centre (0,0) at t=0) on a uniform stream
    rho=u=v=p=1, advected by (t, t); the centre is the nearest periodic image."""
    xr = _wrap(np.asarray(x, dtype=np.float64) - t)
    yr = _wrap(np.asarray(y, dtype=np.float64) - t)
    r2 = xr * xr + yr * yr
    g = np.exp(0.5 * (1.0 - r2))
    du = -beta / (2.0 * math.pi) * g * yr
    dv = beta / (2.0 * math.pi) * g * xr
    dT = -(gamma - 1.0) * beta * beta / (8.0 * gamma * math.pi ** 2) * g * g
    rho = (1.0 + dT) ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    return rho, 1.0 + du, 1.0 + dv, p


def steady_vortex(x, y, cx: float = 3.0, cy: float = 0.0, beta: float = 5.0,
                  gamma: float = GAMMA) -> np.ndarray:
    """The isentropic vortex on a fluid at rest (rho = p = 1 far away, no mean
    flow): an exact steady solution of the Euler equations.  Centred at (cx, cy),
    by default near the right side of [-5, 5]^2, where it is far from uniform
    (no periodic images: for bounded domains with prescribed boundary states)."""
    xr = np.asarray(x, dtype=np.float64) - cx
    yr = np.asarray(y, dtype=np.float64) - cy
    r2 = xr * xr + yr * yr
    g = np.exp(0.5 * (1.0 - r2))
    u = -beta / (2.0 * math.pi) * g * yr
    v = beta / (2.0 * math.pi) * g * xr
    dT = -(gamma - 1.0) * beta * beta / (8.0 * gamma * math.pi ** 2) * g * g
    rho = (1.0 + dT) ** (1.0 / (gamma - 1.0))
    return primitive_to_conserved(rho, u, v, rho ** gamma, gamma)


def fourier_coefficients(seed: int = SEED_PERTURB, kmax: int = 4):
    """Perturbation amplitudes and phases: for rho then p, kx outer, ky inner,
    a ~ U[-1,1] then theta ~ U[0, 2pi); amplitudes normalised to sum |a| = 1."""
    cnt = 2 * kmax * kmax * 2
    u = uniform01(seed, cnt).reshape(2, kmax, kmax, 2)
    a = 2.0 * u[..., 0] - 1.0
    th = 2.0 * math.pi * u[..., 1]
    a = a / np.abs(a).reshape(2, -1).sum(axis=1)[:, None, None]
    return a, th


def fourier_perturbation(x, y, a: np.ndarray, th: np.ndarray, amp: float):
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    kmax = a.shape[-1]
    out = np.zeros((2,) + x.shape)
    for v in range(2):
        for kx in range(1, kmax + 1):
            for ky in range(1, kmax + 1):
                out[v] += a[v, kx - 1, ky - 1] * np.sin(
                    2.0 * math.pi * (kx * x + ky * y) / DOMAIN_L + th[v, kx - 1, ky - 1])
    return amp * out


def vortex(x, y, t: float = 0.0, gamma: float = GAMMA) -> np.ndarray:
    """Conserved state of the isentropic vortex at (x, y, t)."""
    rho, u, v, p = vortex_primitive(x, y, t, gamma=gamma)
    return primitive_to_conserved(rho, u, v, p, gamma)


def perturbed_vortex(x, y, seed: int = SEED_PERTURB, amp: float = 1e-2,
                     gamma: float = GAMMA) -> np.ndarray:
    """Vortex plus seeded smooth Fourier perturbations (wavenumbers 1..4) added to
    the density and the pressure."""
    rho, u, v, p = vortex_primitive(x, y, 0.0, gamma=gamma)
    a, th = fourier_coefficients(seed)
    d = fourier_perturbation(x, y, a, th, amp)
    return primitive_to_conserved(rho + d[0], u, v, p + d[1], gamma)


def density_wave(x, y, t: float = 0.0, gamma: float = GAMMA) -> np.ndarray:
    """rho = 1 + 0.2 sin(2 pi (x + y - 2t)/10), u = v = p = 1: an exact Euler
    solution translated by (t, t)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    rho = 1.0 + 0.2 * np.sin(2.0 * math.pi * ((x - t) + (y - t)) / DOMAIN_L)
    one = np.ones_like(rho)
    return primitive_to_conserved(rho, one, one, one, gamma)


def density_steps(x, y, gamma: float = GAMMA) -> np.ndarray:
    """Piecewise constant data with jumps (periodic): rho = 1, p = 1 inside the
    band |x| < 2.5 and rho = 0.125, p = 0.1 outside it, at rest; a discontinuous
    state of the kind the paper's limiter is for."""
    x = np.asarray(x, dtype=np.float64)
    inside = np.abs(x) < 0.25 * DOMAIN_L
    rho = np.where(inside, 1.0, 0.125)
    p = np.where(inside, 1.0, 0.1)
    zero = np.zeros_like(rho)
    return primitive_to_conserved(rho, zero, zero, p, gamma)


def uniform_state(x, y, rho=1.0, u=0.3, v=-0.2, p=0.8, gamma: float = GAMMA) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    one = np.ones_like(x)
    return primitive_to_conserved(rho * one, u * one, v * one, p * one, gamma)


def linear_state(x, y, rho0=1.0, rx=0.02, ry=-0.015, u=0.4, v=-0.3, p0=1.0, px=0.03,
                 py=0.05, gamma: float = GAMMA) -> np.ndarray:
    """Constant velocity with density and pressure linear in (x, y).  Every Euler
    flux component is then a linear function of position."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    rho = rho0 + rx * x + ry * y
    p = p0 + px * x + py * y
    one = np.ones_like(x)
    return primitive_to_conserved(rho, u * one, v * one, p, gamma)


def max_wave_speed(U: np.ndarray, gamma: float = GAMMA) -> float:
    """max(|v| + sqrt(gamma p / rho)) over conserved states U[..., 4]."""
    rho = U[..., 0]
    u = U[..., 1] / rho
    v = U[..., 2] / rho
    p = (gamma - 1.0) * (U[..., 3] - 0.5 * rho * (u * u + v * v))
    return float(np.max(np.sqrt(u * u + v * v) + np.sqrt(gamma * p / rho)))


def fixed_dt(mesh: Mesh, ic, p: int, cfl: float = 0.3, gamma: float = GAMMA) -> float:
    """Time step of a workload, fixed once from the mesh and the initial data:
    dt = cfl * min_e r_in(e) / ((2p+1) * s), with r_in the inscribed radius
    (twice the area over the perimeter) and s the largest |v| + c of the initial
    data sampled at element vertices and centroids."""
    xy = mesh.elem_xy
    e0 = xy[:, 1] - xy[:, 0]
    e1 = xy[:, 2] - xy[:, 1]
    e2 = xy[:, 0] - xy[:, 2]
    area2 = e0[:, 0] * (-e2[:, 1]) - e0[:, 1] * (-e2[:, 0])
    per = (np.hypot(e0[:, 0], e0[:, 1]) + np.hypot(e1[:, 0], e1[:, 1])
           + np.hypot(e2[:, 0], e2[:, 1]))
    r_in = float(np.min(area2 / per))
    pts = np.concatenate([xy.reshape(-1, 2), xy.mean(axis=1)], axis=0)
    s = max_wave_speed(ic(pts[:, 0], pts[:, 1]), gamma)
    return cfl * r_in / ((2 * p + 1) * s)
