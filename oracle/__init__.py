"""CPU oracle of the modal DG method (FP64, plain C), with a ctypes wrapper.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product path (the CUDA
library and its Python binding) never imports this package.

``build()`` compiles ``dg_oracle.c`` into ``liboracle.so`` beside it with gcc
(no fast-math, no FMA contraction, so the arithmetic is plain IEEE FP64).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

M = 4


def build(force: bool = False) -> str:
    """Compile the oracle if the shared object is missing or older than its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                               "-D_DEFAULT_SOURCE", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        L = ctypes.c_int64
        sigs = {
            "or_gauss_jacobi": (I, [I, D, D, P, P]),
            "or_gauss_legendre": (I, [I, P, P]),
            "or_stroud": (I, [I, P, P, P]),
            "or_dubiner_eval": (I, [I, I, P, P, P, P, P]),
            "or_dubiner_integrals": (I, [I, P]),
            "or_dubiner_gram_exact": (I, [I, P]),
            "or_dubiner_monomials": (I, [I, P]),
            "or_opmax": (I, []),
            "or_create": (P, [I, I, I, D, L, P, P, P]),
            "or_destroy": (None, [P]),
            "or_info": (I, [P, P]),
            "or_volume_rule": (I, [P, P, P, P]),
            "or_set_volume_rule": (I, [P, I, P, P, P]),
            "or_volume_tables": (I, [P, P, P, P]),
            "or_edge_rule": (I, [P, P, P]),
            "or_edges": (I, [P, P, P, P, P, P, P, P]),
            "or_det_j": (I, [P, P]),
            "or_map_points": (I, [P, I, P, P, P]),
            "or_volume_points": (I, [P, P]),
            "or_eval_points": (I, [P, P, I, P, P, P]),
            "or_project": (I, [P, P, P]),
            "or_lax_friedrichs": (I, [D, P, P, D, D, P]),
            "or_euler_flux": (I, [D, P, P, P]),
            "or_rhs": (I, [P, P, P]),
            "or_last_volume_term": (I, [P, P]),
            "or_ssp_rk3": (I, [P, P, D, I]),
            "or_rk2": (I, [P, P, D, I]),
            "or_rk4": (I, [P, P, D, I]),
            "or_limit_bj": (I, [P, P]),
            "or_n_boundary": (L, [P]),
            "or_boundary_points": (I, [P, P]),
            "or_set_boundary_state": (I, [P, P]),
            "or_set_limiter": (I, [P, I]),
            "or_totals": (I, [P, P, P]),
            "or_lax_friedrichs_jacobians": (I, [D, P, P, D, D, P, P]),
            "or_flux_jacobian": (I, [D, P, D, D, P]),
            "or_rhs_vjp": (I, [P, P, P, P]),
            "or_ssp_rk3_vjp": (I, [P, P, D, P, P]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _chk(rc):
    if rc != 0:
        raise RuntimeError("oracle call failed (%d)" % rc)


# ---------------------------------------------------------------------------
# quadrature and basis
# ---------------------------------------------------------------------------

def gauss_jacobi(n: int, a: float, b: float):
    x = np.zeros(n); w = np.zeros(n)
    _chk(_load().or_gauss_jacobi(n, a, b, _ptr(x), _ptr(w)))
    return x, w


def gauss_legendre(n: int):
    return gauss_jacobi(n, 0.0, 0.0)


def stroud(n: int):
    r = np.zeros(n * n); s = np.zeros(n * n); w = np.zeros(n * n)
    _chk(_load().or_stroud(n, _ptr(r), _ptr(s), _ptr(w)))
    return r, s, w


def n_modes(p: int) -> int:
    return (p + 1) * (p + 2) // 2


def dubiner(p: int, r, s):
    """Values and reference gradients [npts, Np] of the orthonormal basis."""
    r = np.ascontiguousarray(r, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.float64)
    n, np_ = r.size, n_modes(p)
    phi = np.zeros((n, np_)); dr = np.zeros((n, np_)); ds = np.zeros((n, np_))
    _chk(_load().or_dubiner_eval(p, n, _ptr(r), _ptr(s), _ptr(phi), _ptr(dr), _ptr(ds)))
    return phi, dr, ds


def dubiner_integrals(p: int):
    out = np.zeros(n_modes(p))
    _chk(_load().or_dubiner_integrals(p, _ptr(out)))
    return out


def dubiner_gram_exact(p: int):
    G = np.zeros((n_modes(p), n_modes(p)))
    _chk(_load().or_dubiner_gram_exact(p, _ptr(G)))
    return G


def dubiner_monomials(p: int):
    K = _load().or_opmax() + 1
    out = np.zeros((n_modes(p), K, K))
    _chk(_load().or_dubiner_monomials(p, _ptr(out)))
    return out


def lax_friedrichs(Ul, Ur, nx, ny, gamma=1.4):
    Ul = np.ascontiguousarray(Ul, dtype=np.float64)
    Ur = np.ascontiguousarray(Ur, dtype=np.float64)
    out = np.zeros(4)
    _chk(_load().or_lax_friedrichs(gamma, _ptr(Ul), _ptr(Ur), nx, ny, _ptr(out)))
    return out


def euler_flux(U, gamma=1.4):
    U = np.ascontiguousarray(U, dtype=np.float64)
    F1 = np.zeros(4); F2 = np.zeros(4)
    _chk(_load().or_euler_flux(gamma, _ptr(U), _ptr(F1), _ptr(F2)))
    return F1, F2


def lax_friedrichs_jacobians(Ul, Ur, nx, ny, gamma=1.4):
    Ul = np.ascontiguousarray(Ul, dtype=np.float64)
    Ur = np.ascontiguousarray(Ur, dtype=np.float64)
    Jl = np.zeros((4, 4)); Jr = np.zeros((4, 4))
    _chk(_load().or_lax_friedrichs_jacobians(gamma, _ptr(Ul), _ptr(Ur), nx, ny, _ptr(Jl), _ptr(Jr)))
    return Jl, Jr


def flux_jacobian(U, nx, ny, gamma=1.4):
    U = np.ascontiguousarray(U, dtype=np.float64)
    J = np.zeros((4, 4))
    _chk(_load().or_flux_jacobian(gamma, _ptr(U), nx, ny, _ptr(J)))
    return J


# ---------------------------------------------------------------------------
# solver
# ---------------------------------------------------------------------------

class OracleDG:
    """FP64 CPU DG solver on one mesh (coefficients c[N, M, Np])."""

    def __init__(self, elem_xy, nbr, nbr_face, p: int, n_edge_pts: int = 0, n_vol_dir: int = 0,
                 gamma: float = 1.4, vol_rule: str = "collapsed"):
        """vol_rule: "collapsed" (the (p+1)^2-point collapsed Gauss grid, or
        n_vol_dir^2 points) or "symmetric" (the fully symmetric degree-2p rule
        of oracle/symmetric_rules.py)."""
        lib = _load()
        self._xy = np.ascontiguousarray(elem_xy, dtype=np.float64)
        self._nbr = np.ascontiguousarray(nbr, dtype=np.int64)
        self._nf = np.ascontiguousarray(nbr_face, dtype=np.int8)
        N = self._xy.shape[0]
        h = lib.or_create(p, n_edge_pts, n_vol_dir, gamma, N, _ptr(self._xy), _ptr(self._nbr),
                          _ptr(self._nf))
        if not h:
            raise ValueError("oracle rejected the mesh or the order")
        self._h = h
        if vol_rule == "symmetric":
            from .symmetric_rules import symmetric_rule
            r, s, w = (np.ascontiguousarray(v) for v in symmetric_rule(p))
            _chk(lib.or_set_volume_rule(h, r.size, _ptr(r), _ptr(s), _ptr(w)))
        elif vol_rule != "collapsed":
            raise ValueError("vol_rule must be 'collapsed' or 'symmetric'")
        self.vol_rule = vol_rule
        info = np.zeros(5, dtype=np.int64)
        lib.or_info(h, _ptr(info))
        self.N, self.np, self.nq, self.ne, self.n_edges = (int(v) for v in info)
        self.p = p
        self.gamma = gamma

    @classmethod
    def from_mesh(cls, mesh, p: int, **kw):
        return cls(mesh.elem_xy, mesh.nbr, mesh.nbr_face, p, **kw)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.or_destroy(h)
            self._h = None

    def coef_shape(self):
        return (self.N, M, self.np)

    def volume_rule(self):
        r = np.zeros(self.nq); s = np.zeros(self.nq); w = np.zeros(self.nq)
        _lib.or_volume_rule(self._h, _ptr(r), _ptr(s), _ptr(w))
        return r, s, w

    def volume_tables(self):
        """phi, dphi/dr, dphi/ds [nq, Np] at the volume points (evaluated at the
        exact images of the rounded 1D nodes)."""
        a = np.zeros((self.nq, self.np)); b = np.zeros((self.nq, self.np)); c = np.zeros((self.nq, self.np))
        _chk(_lib.or_volume_tables(self._h, _ptr(a), _ptr(b), _ptr(c)))
        return a, b, c

    def edge_rule(self):
        x = np.zeros(self.ne); w = np.zeros(self.ne)
        _lib.or_edge_rule(self._h, _ptr(x), _ptr(w))
        return x, w

    def edges(self):
        n = self.n_edges
        el = np.zeros(n, np.int64); er = np.zeros(n, np.int64)
        eL = np.zeros(n, np.int32); eR = np.zeros(n, np.int32)
        nx = np.zeros(n); ny = np.zeros(n); ln = np.zeros(n)
        _lib.or_edges(self._h, _ptr(el), _ptr(er), _ptr(eL), _ptr(eR), _ptr(nx), _ptr(ny), _ptr(ln))
        return dict(left=el, right=er, L=eL, R=eR, nx=nx, ny=ny, length=ln)

    def det_j(self):
        out = np.zeros(self.N)
        _lib.or_det_j(self._h, _ptr(out))
        return out

    def map_points(self, r, s):
        r = np.ascontiguousarray(r, dtype=np.float64)
        s = np.ascontiguousarray(s, dtype=np.float64)
        out = np.zeros((self.N, r.size, 2))
        _chk(_lib.or_map_points(self._h, r.size, _ptr(r), _ptr(s), _ptr(out)))
        return out

    def volume_points(self):
        out = np.zeros((self.N, self.nq, 2))
        _chk(_lib.or_volume_points(self._h, _ptr(out)))
        return out

    def eval_points(self, c, r, s):
        c = np.ascontiguousarray(c, dtype=np.float64)
        r = np.ascontiguousarray(r, dtype=np.float64)
        s = np.ascontiguousarray(s, dtype=np.float64)
        out = np.zeros((self.N, r.size, M))
        _chk(_lib.or_eval_points(self._h, _ptr(c), r.size, _ptr(r), _ptr(s), _ptr(out)))
        return out

    def project(self, u_qp):
        u = np.ascontiguousarray(u_qp, dtype=np.float64).reshape(self.N, self.nq, M)
        c = np.zeros(self.coef_shape())
        _chk(_lib.or_project(self._h, _ptr(u), _ptr(c)))
        return c

    def project_ic(self, ic):
        """Project a function ic(x, y) -> conserved state [..., 4]."""
        xy = self.volume_points()
        return self.project(ic(xy[..., 0], xy[..., 1]))

    def rhs(self, c):
        c = np.ascontiguousarray(c, dtype=np.float64)
        R = np.zeros(self.coef_shape())
        _chk(_lib.or_rhs(self._h, _ptr(c), _ptr(R)))
        return R

    def rhs_and_volume(self, c):
        """(R, V / det J): the RHS and its volume term, whose size bounds the
        rounding error of R (R is the small difference of the volume and surface
        terms, each of which grows like 1/h)."""
        R = self.rhs(c)
        V = np.zeros(self.coef_shape())
        _chk(_lib.or_last_volume_term(self._h, _ptr(V)))
        return R, V

    def ssp_rk3(self, c, dt: float, nsteps: int):
        out = np.array(c, dtype=np.float64, copy=True, order="C")
        _chk(_lib.or_ssp_rk3(self._h, _ptr(out), dt, nsteps))
        return out

    def rk2(self, c, dt: float, nsteps: int):
        """Heun's two-stage method (the paper's classic RK2), nsteps steps."""
        out = np.array(c, dtype=np.float64, copy=True, order="C")
        _chk(_lib.or_rk2(self._h, _ptr(out), dt, nsteps))
        return out

    def rk4(self, c, dt: float, nsteps: int):
        """The classical four-stage RK4 (the paper's RK4), nsteps steps."""
        out = np.array(c, dtype=np.float64, copy=True, order="C")
        _chk(_lib.or_rk4(self._h, _ptr(out), dt, nsteps))
        return out

    @property
    def n_boundary(self) -> int:
        return int(_lib.or_n_boundary(self._h))

    def boundary_points(self):
        """Physical points of the boundary faces [Nb, ne, 2] (element order, then
        local face; points counter-clockwise along the element)."""
        out = np.zeros((self.n_boundary, self.ne, 2))
        _chk(_lib.or_boundary_points(self._h, _ptr(out)))
        return out

    def set_boundary_state(self, u):
        """Conserved state prescribed at the boundary points [Nb, ne, 4]."""
        u = np.ascontiguousarray(u, dtype=np.float64)
        assert u.shape == (self.n_boundary, self.ne, M)
        _chk(_lib.or_set_boundary_state(self._h, _ptr(u)))

    def limit(self, c):
        """Barth-Jespersen limiter (p = 1) applied to a copy of c."""
        out = np.array(c, dtype=np.float64, copy=True, order="C")
        _chk(_lib.or_limit_bj(self._h, _ptr(out)))
        return out

    def set_limiter(self, on: bool):
        """Limit every stage value and new state of rk2 / ssp_rk3 / rk4 (p = 1)."""
        _chk(_lib.or_set_limiter(self._h, 1 if on else 0))

    def rhs_vjp(self, c, lam):
        """(dR/dc)^T lam."""
        c = np.ascontiguousarray(c, dtype=np.float64)
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        out = np.zeros(self.coef_shape())
        _chk(_lib.or_rhs_vjp(self._h, _ptr(c), _ptr(lam), _ptr(out)))
        return out

    def ssp_rk3_vjp(self, c_n, dt: float, lam_np1):
        """(d c_{n+1} / d c_n)^T lam_np1 for one SSP-RK3 step from c_n."""
        c_n = np.ascontiguousarray(c_n, dtype=np.float64)
        lam = np.ascontiguousarray(lam_np1, dtype=np.float64)
        out = np.zeros(self.coef_shape())
        _chk(_lib.or_ssp_rk3_vjp(self._h, _ptr(c_n), dt, _ptr(lam), _ptr(out)))
        return out

    def totals(self, c):
        c = np.ascontiguousarray(c, dtype=np.float64)
        out = np.zeros(M)
        _chk(_lib.or_totals(self._h, _ptr(c), _ptr(out)))
        return out

    def l2_error(self, c, exact, var: int = 0, n_dir: int = 0):
        """sqrt(sum over elements of int (U_h - U_exact)^2) for one variable, with a
        collapsed rule exact to degree 2p+6 (n_dir = p+4 points per direction)."""
        nd = n_dir or (self.p + 4)
        r, s, w = stroud(nd)
        vals = self.eval_points(c, r, s)[..., var]
        xy = self.map_points(r, s)
        ex = exact(xy[..., 0], xy[..., 1])[..., var]
        dJ = self.det_j()
        return float(np.sqrt(np.sum(dJ[:, None] * w[None, :] * (vals - ex) ** 2)))
