"""Thin Python binding of the C ABI in include/dg.h (ctypes).

Argument marshalling only: every step of the solver runs in libdg.so's CUDA
kernels.  State tensors are torch float64 CUDA tensors of shape [N, 4, N_p]
(element-major coefficients); calls run on torch's current CUDA stream.

If libdg.so is missing this module raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdg.so")

DG_OK = 0
STATUS = {0: "DG_OK", 1: "DG_EINVAL", 2: "DG_ENOMEM", 3: "DG_ECUDA", 4: "DG_EMESH",
          5: "DG_ENONPHYS", 6: "DG_ETIMEOUT", 7: "DG_ENOTIMPL"}
PRECISION = {"fp64": 0, "tf32x1": 1, "tf32x3": 2}
METHOD = {"ssp_rk3": 0, "rk2": 1, "rk4": 2}
VOL_RULE = {"collapsed": 0, "symmetric": 1}

# every entry point declared in include/dg.h
EXPORTS = ("dg_mesh_create", "dg_mesh_destroy", "dg_mesh_info", "dg_volume_points",
           "dg_project_ic", "dg_rhs", "dg_rk_step", "dg_rk_step_host", "dg_adjoint_step",
           "dg_conserved_totals", "dg_last_error", "dg_host_tables", "dg_set_timing",
           "dg_kernel_times", "dg_probe_fma_rate", "dg_device_status", "dg_rhs_noalloc", "dg_self_test", "dg_eval_points", "dg_rhs_adjoint", "dg_stable_dt",
           "dg_rk_step_method", "dg_limit", "dg_set_limiter", "dg_boundary_points",
           "dg_set_boundary_state", "dg_volume_rule", "dg_set_small_mesh_stepper", "dg_rk_step_stages", "dg_adjoint_step_stages", "dg_det_j",
           "dg_map_points", "dg_l2_error")
KERNEL_KINDS = ("traces", "face", "element", "project", "totals", "adjoint", "other", "stepper")


class DGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class _Desc(ctypes.Structure):
    _fields_ = [("n_elem", ctypes.c_int64), ("elem_xy", ctypes.c_void_p), ("nbr", ctypes.c_void_p),
                ("nbr_face", ctypes.c_void_p), ("p", ctypes.c_int), ("n_edge_pts", ctypes.c_int),
                ("gamma", ctypes.c_double), ("vol_rule", ctypes.c_int)]


class _Info(ctypes.Structure):
    _fields_ = [("n_elem", ctypes.c_int64), ("n_face", ctypes.c_int64), ("p", ctypes.c_int),
                ("n_modes", ctypes.c_int), ("n_vol_pts", ctypes.c_int), ("n_edge_pts", ctypes.c_int),
                ("gamma", ctypes.c_double), ("n_boundary_face", ctypes.c_int64)]


_lib = None


def load(path: str = None):
    """Loads libdg.so (raises if it has not been built).  The environment variable
    DG_LIB names another build of the library to load instead (for example the
    index-checking libdg_debug.so of ``_build.build(debug=True)``)."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = os.environ.get("DG_LIB") or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("libdg.so not found at %s: run __graft_entry__.build() (or "
                           "python -m paper_1601_07944_gb300._build) first" % path)
    lib = ctypes.CDLL(path)
    P, I, D, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    sig = {
        "dg_mesh_create": [P, P],
        "dg_mesh_destroy": [P],
        "dg_mesh_info": [P, P],
        "dg_volume_points": [P, P, P],
        "dg_project_ic": [P, P, P, P],
        "dg_rhs": [P, P, P, I, P],
        "dg_rk_step": [P, P, D, I, I, P],
        "dg_rk_step_method": [P, P, D, I, I, I, P],
        "dg_limit": [P, P, P],
        "dg_boundary_points": [P, P, P],
        "dg_set_boundary_state": [P, P, P],
        "dg_set_limiter": [P, I],
        "dg_set_small_mesh_stepper": [P, I],
        "dg_rk_step_stages": [P, P, D, P, P, P],
        "dg_adjoint_step_stages": [P, P, P, P, D, P, P, P],
        "dg_det_j": [P, P, P],
        "dg_map_points": [P, I, P, P, P, P],
        "dg_l2_error": [P, I, P, P, P, P, P, I, P, P],
        "dg_rk_step_host": [P, P, D, I, I, P],
        "dg_adjoint_step": [P, P, D, P, P, P],
        "dg_conserved_totals": [P, P, P, P],
        "dg_host_tables": [I, I, P, P, P, P, P, P, P, P, P],
        "dg_set_timing": [P, I],
        "dg_kernel_times": [P, P, P],
        "dg_probe_fma_rate": [P, P, P],
        "dg_device_status": [P, P],
        "dg_rhs_noalloc": [P, P, P, I, P],
        "dg_self_test": [P, P],
        "dg_eval_points": [P, I, P, P, P, P, P],
        "dg_rhs_adjoint": [P, P, P, P, P],
        "dg_stable_dt": [P, P, D, P, P],
        "dg_volume_rule": [I, I, P, P, P, P, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = I
    lib.dg_last_error.argtypes = []
    lib.dg_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(st: int):
    if st != DG_OK:
        raise DGError(st, load().dg_last_error().decode(errors="replace"))


def _np_ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_ptr(t, name: str, shape=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError("%s must be a float64 CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s has shape %s, expected %s" % (name, tuple(t.shape), tuple(shape)))
    return ctypes.c_void_p(t.data_ptr())


def _prec(precision) -> int:
    if isinstance(precision, str):
        return PRECISION[precision]
    return int(precision)


def probe_fma_rate(stream=None):
    """(fp64, fp32) sustained FMA rates of the current device, TFLOP/s."""
    a = ctypes.c_double(); b = ctypes.c_double()
    _check(load().dg_probe_fma_rate(ctypes.byref(a), ctypes.byref(b), _stream_ptr(stream)))
    return a.value, b.value


def self_test(stream=None):
    """(float64->float32, float32->float64) bit mismatches of the integer
    conversions against the hardware's, and reciprocals and square roots more
    than 1 ulp from 1/x and sqrt(x), over 2^20 values."""
    out = np.zeros(4, dtype=np.int64)
    _check(load().dg_self_test(_np_ptr(out), _stream_ptr(stream)))
    return tuple(int(v) for v in out)


def host_tables(p: int, ne: int = 0):
    """The library's host-side rules and basis tables (no GPU needed)."""
    ne = ne or p + 1
    np_, nq = (p + 1) * (p + 2) // 2, (p + 1) ** 2
    out = dict(vol_r=np.zeros(nq), vol_s=np.zeros(nq), vol_w=np.zeros(nq), edge_x=np.zeros(ne),
               edge_w=np.zeros(ne), phi=np.zeros((nq, np_)), dphi_r=np.zeros((nq, np_)),
               dphi_s=np.zeros((nq, np_)), phi_face=np.zeros((3, ne, np_)))
    _check(load().dg_host_tables(p, ne, *[_np_ptr(out[k]) for k in (
        "vol_r", "vol_s", "vol_w", "edge_x", "edge_w", "phi", "dphi_r", "dphi_s", "phi_face")]))
    return out


def volume_rule(p: int, rule: str = "collapsed"):
    """The library's volume rule for degree p (no GPU needed): points r, s,
    weights w and the basis phi [nq, N_p] at the points."""
    lib = load()
    nq = ctypes.c_int()
    _check(lib.dg_volume_rule(p, VOL_RULE[rule], ctypes.byref(nq), None, None, None, None))
    n, np_ = nq.value, (p + 1) * (p + 2) // 2
    r, s, w, phi = np.zeros(n), np.zeros(n), np.zeros(n), np.zeros((n, np_))
    _check(lib.dg_volume_rule(p, VOL_RULE[rule], ctypes.byref(nq), _np_ptr(r), _np_ptr(s), _np_ptr(w),
                              _np_ptr(phi)))
    return r, s, w, phi


class Mesh:
    """A mesh handle (geometry, tables and work buffers on the current GPU).

    vol_rule: "collapsed" (the (p+1)^2-point collapsed Gauss grid, the default)
    or "symmetric" (the fully symmetric degree-2p rule with the paper's point
    counts, 3 / 6 / 12 / 16 / 25 at p = 1..5)."""

    def __init__(self, elem_xy, nbr, nbr_face, p: int, n_edge_pts: int = 0, gamma: float = 1.4,
                 vol_rule: str = "collapsed"):
        if vol_rule not in VOL_RULE:
            raise ValueError("vol_rule must be one of %s" % sorted(VOL_RULE))
        lib = load()
        xy = np.ascontiguousarray(elem_xy, dtype=np.float64)
        nb = np.ascontiguousarray(nbr, dtype=np.int64)
        nf = np.ascontiguousarray(nbr_face, dtype=np.int8)
        if xy.ndim != 3 or xy.shape[1:] != (3, 2) or nb.shape != (xy.shape[0], 3) or nf.shape != nb.shape:
            raise ValueError("mesh arrays must be elem_xy[N,3,2], nbr[N,3], nbr_face[N,3]")
        desc = _Desc(xy.shape[0], xy.ctypes.data, nb.ctypes.data, nf.ctypes.data, p, n_edge_pts, gamma,
                     VOL_RULE[vol_rule])
        h = ctypes.c_void_p()
        _check(lib.dg_mesh_create(ctypes.byref(desc), ctypes.byref(h)))
        self._h = h
        self._xy = xy
        info = _Info()
        _check(lib.dg_mesh_info(h, ctypes.byref(info)))
        self.N, self.n_face, self.p = info.n_elem, info.n_face, info.p
        self.np, self.nq, self.ne, self.gamma = info.n_modes, info.n_vol_pts, info.n_edge_pts, info.gamma
        self.n_boundary = info.n_boundary_face
        self.vol_rule = vol_rule

    @classmethod
    def from_mesh(cls, mesh, p: int, **kw):
        return cls(mesh.elem_xy, mesh.nbr, mesh.nbr_face, p, **kw)

    @property
    def handle(self):
        return self._h

    @property
    def coef_shape(self):
        return (self.N, 4, self.np)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().dg_mesh_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def det_j(self, stream=None):
        """det J of every element (twice its area), a float64 device tensor [N] (dg_det_j)."""
        import torch
        out = torch.empty(self.N, dtype=torch.float64, device="cuda")
        _check(load().dg_det_j(self._h, _dev_ptr(out, "detj"), _stream_ptr(stream)))
        return out

    def map_points(self, r, s, stream=None):
        """Physical points [N, npts, 2] (device) of reference points (r, s) of every element."""
        import torch
        r = np.ascontiguousarray(r, dtype=np.float64)
        s = np.ascontiguousarray(s, dtype=np.float64)
        out = torch.empty((self.N, r.size, 2), dtype=torch.float64, device="cuda")
        _check(load().dg_map_points(self._h, r.size, _np_ptr(r), _np_ptr(s), _dev_ptr(out, "xy"),
                                    _stream_ptr(stream)))
        return out

    # -- diagnostics --------------------------------------------------------
    def set_timing(self, enable: bool):
        _check(load().dg_set_timing(self._h, 1 if enable else 0))

    def device_status(self, stream=None):
        """Synchronises and raises DGError(DG_ETIMEOUT) if a bounded device wait expired."""
        _check(load().dg_device_status(self._h, _stream_ptr(stream)))

    def kernel_times(self):
        """{kind: (launches, total ms)} since timing was enabled (synchronises)."""
        ms = np.zeros(8); n = np.zeros(8, dtype=np.int64)
        _check(load().dg_kernel_times(self._h, _np_ptr(ms), _np_ptr(n)))
        return {KERNEL_KINDS[k]: (int(n[k]), float(ms[k])) for k in range(8) if n[k]}

    # -- calls ------------------------------------------------------------
    def volume_points(self, stream=None):
        import torch
        xy = torch.empty((self.N, self.nq, 2), dtype=torch.float64, device="cuda")
        _check(load().dg_volume_points(self._h, _dev_ptr(xy, "xy"), _stream_ptr(stream)))
        return xy

    def eval_points(self, c, r, s, stream=None):
        """Solution values [N, npts, 4] at reference points (r, s) of every element."""
        import torch
        r = np.ascontiguousarray(r, dtype=np.float64)
        s = np.ascontiguousarray(s, dtype=np.float64)
        out = torch.empty((self.N, r.size, 4), dtype=torch.float64, device="cuda")
        _check(load().dg_eval_points(self._h, r.size, _np_ptr(r), _np_ptr(s), _dev_ptr(c, "c", self.coef_shape),
                                     _dev_ptr(out, "out"), _stream_ptr(stream)))
        return out

    def l2_error(self, c, exact, var: int = 0, n_dir: int = 0, rule=None, stream=None):
        """sqrt(sum_e int_e (U_h - U_exact)^2) for one variable (dg_l2_error).  `rule` =
        (r, s, w) is a reference-triangle rule (default: the library's collapsed rule
        with p+4 points per direction, exact to degree 2p+7); exact(x, y) -> [..., 4]
        is evaluated on the host at the physical points (dg_map_points)."""
        import torch
        if rule is None:
            T = host_tables(n_dir - 1 if n_dir else self.p + 3)
            r, s, w = T["vol_r"], T["vol_s"], T["vol_w"]
        else:
            r, s, w = rule
        r = np.ascontiguousarray(r, dtype=np.float64)
        s = np.ascontiguousarray(s, dtype=np.float64)
        w = np.ascontiguousarray(w, dtype=np.float64)
        xy = self.map_points(r, s, stream).cpu().numpy()
        ex = torch.from_numpy(np.ascontiguousarray(exact(xy[..., 0], xy[..., 1]), dtype=np.float64)).cuda()
        out = ctypes.c_double()
        _check(load().dg_l2_error(self._h, r.size, _np_ptr(r), _np_ptr(s), _np_ptr(w),
                                  _dev_ptr(c, "c", self.coef_shape), _dev_ptr(ex, "exact", (self.N, r.size, 4)),
                                  int(var), ctypes.byref(out), _stream_ptr(stream)))
        return out.value

    def project_ic(self, u, out=None, stream=None):
        import torch
        c = out if out is not None else torch.empty(self.coef_shape, dtype=torch.float64, device="cuda")
        _check(load().dg_project_ic(self._h, _dev_ptr(u, "u", (self.N, self.nq, 4)),
                                    _dev_ptr(c, "c", self.coef_shape), _stream_ptr(stream)))
        return c

    def rhs(self, c, out=None, precision="fp64", stream=None):
        import torch
        r = out if out is not None else torch.empty(self.coef_shape, dtype=torch.float64, device="cuda")
        _check(load().dg_rhs(self._h, _dev_ptr(c, "c", self.coef_shape), _dev_ptr(r, "r", self.coef_shape),
                             _prec(precision), _stream_ptr(stream)))
        return r

    def rhs_noalloc(self, c, out, precision="fp64", stream=None):
        """dg_rhs without any device allocation: the work space comes from the
        library's fixed 64 MiB device array (meshes that need more are rejected).
        For callers that cannot allocate when they evaluate the RHS; `out` must be
        given.  Calls that overlap on the GPU race on the shared array."""
        _check(load().dg_rhs_noalloc(self._h, _dev_ptr(c, "c", self.coef_shape), _dev_ptr(out, "r", self.coef_shape),
                                     _prec(precision), _stream_ptr(stream)))
        return out

    def rk_step(self, c, dt: float, nsteps: int = 1, precision="fp64", stream=None, method="ssp_rk3"):
        """nsteps Runge-Kutta steps in place on the device tensor c: "ssp_rk3"
        (dg_rk_step), or the paper's "rk2" (Heun) or "rk4" (dg_rk_step_method)."""
        if method == "ssp_rk3":
            _check(load().dg_rk_step(self._h, _dev_ptr(c, "c", self.coef_shape), float(dt), int(nsteps),
                                     _prec(precision), _stream_ptr(stream)))
            return c
        if method not in METHOD:
            raise ValueError("method must be one of %s" % sorted(METHOD))
        _check(load().dg_rk_step_method(self._h, _dev_ptr(c, "c", self.coef_shape), float(dt), int(nsteps),
                                        METHOD[method], _prec(precision), _stream_ptr(stream)))
        return c

    def boundary_points(self, stream=None):
        """Physical points of the boundary faces, a device tensor [Nb, n_e, 2]."""
        import torch
        out = torch.empty((self.n_boundary, self.ne, 2), dtype=torch.float64, device="cuda")
        if self.n_boundary:
            _check(load().dg_boundary_points(self._h, ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out

    def set_boundary_state(self, u, stream=None):
        """Conserved state prescribed at the boundary points: device tensor [Nb, n_e, 4]."""
        import torch
        if not (isinstance(u, torch.Tensor) and u.is_cuda and u.dtype == torch.float64 and u.is_contiguous()
                and tuple(u.shape) == (self.n_boundary, self.ne, 4)):
            raise TypeError("u must be a contiguous float64 CUDA tensor of shape %s"
                            % ((self.n_boundary, self.ne, 4),))
        _check(load().dg_set_boundary_state(self._h, ctypes.c_void_p(u.data_ptr()), _stream_ptr(stream)))

    def limit(self, c, stream=None):
        """Barth-Jespersen limiter (p = 1) in place on the device tensor c."""
        _check(load().dg_limit(self._h, _dev_ptr(c, "c", self.coef_shape), _stream_ptr(stream)))
        return c

    def set_small_mesh_stepper(self, on: bool):
        """Run rk_step on a small mesh (float64) as one fused launch per call (on
        by default) or as separate launches."""
        _check(load().dg_set_small_mesh_stepper(self._h, 1 if on else 0))

    def set_limiter(self, on: bool):
        """Limit every stage value and new state of rk_step (p = 1, float64)."""
        _check(load().dg_set_limiter(self._h, 1 if on else 0))

    def rk_step_host(self, c_host, dt: float, nsteps: int = 1, precision="fp64", stream=None):
        """nsteps SSP-RK3 steps on a host array (numpy or CPU tensor, ideally pinned), in place."""
        import torch
        if isinstance(c_host, torch.Tensor):
            if c_host.is_cuda or c_host.dtype != torch.float64 or not c_host.is_contiguous():
                raise TypeError("c_host must be a contiguous float64 CPU tensor")
            if tuple(c_host.shape) != self.coef_shape:
                raise ValueError("c_host has the wrong shape")
            ptr = ctypes.c_void_p(c_host.data_ptr())
        else:
            if c_host.dtype != np.float64 or not c_host.flags.c_contiguous or c_host.shape != self.coef_shape:
                raise TypeError("c_host must be a contiguous float64 array of shape %s" % (self.coef_shape,))
            ptr = _np_ptr(c_host)
        _check(load().dg_rk_step_host(self._h, ptr, float(dt), int(nsteps), _prec(precision),
                                      _stream_ptr(stream)))
        return c_host

    def rhs_adjoint(self, c, lam, out=None, stream=None):
        """(dR/dc)^T lam at c."""
        import torch
        o = out if out is not None else torch.empty(self.coef_shape, dtype=torch.float64, device="cuda")
        _check(load().dg_rhs_adjoint(self._h, _dev_ptr(c, "c", self.coef_shape), _dev_ptr(lam, "lam", self.coef_shape),
                                     _dev_ptr(o, "out", self.coef_shape), _stream_ptr(stream)))
        return o

    def adjoint_step(self, c_n, dt: float, lam_np1, out=None, stream=None):
        import torch
        lam = out if out is not None else torch.empty(self.coef_shape, dtype=torch.float64, device="cuda")
        _check(load().dg_adjoint_step(self._h, _dev_ptr(c_n, "c_n", self.coef_shape), float(dt),
                                      _dev_ptr(lam_np1, "lam_np1", self.coef_shape),
                                      _dev_ptr(lam, "lam_n", self.coef_shape), _stream_ptr(stream)))
        return lam

    def rk_step_stages(self, c, dt: float, u1, u2, stream=None):
        """One float64 SSP-RK3 step on c in place (the same bits as rk_step) that
        also writes its stage values into u1 and u2."""
        _check(load().dg_rk_step_stages(self._h, _dev_ptr(c, "c", self.coef_shape), float(dt),
                                        _dev_ptr(u1, "u1", self.coef_shape), _dev_ptr(u2, "u2", self.coef_shape),
                                        _stream_ptr(stream)))
        return c

    def adjoint_step_stages(self, c_n, u1, u2, dt: float, lam_np1, out=None, stream=None):
        """adjoint_step with the step's stage values given (rk_step_stages)."""
        import torch
        lam = out if out is not None else torch.empty(self.coef_shape, dtype=torch.float64, device="cuda")
        _check(load().dg_adjoint_step_stages(self._h, _dev_ptr(c_n, "c_n", self.coef_shape),
                                             _dev_ptr(u1, "u1", self.coef_shape), _dev_ptr(u2, "u2", self.coef_shape),
                                             float(dt), _dev_ptr(lam_np1, "lam_np1", self.coef_shape),
                                             _dev_ptr(lam, "lam_n", self.coef_shape), _stream_ptr(stream)))
        return lam

    def stable_dt(self, c, cfl: float = 0.3, stream=None) -> float:
        """cfl * r_min / ((2p+1) max(|v| + c)) over the volume points of c."""
        out = ctypes.c_double()
        _check(load().dg_stable_dt(self._h, _dev_ptr(c, "c", self.coef_shape), float(cfl), ctypes.byref(out),
                                   _stream_ptr(stream)))
        return out.value

    def conserved_totals(self, c, stream=None):
        out = np.zeros(4)
        _check(load().dg_conserved_totals(self._h, _dev_ptr(c, "c", self.coef_shape), _np_ptr(out),
                                          _stream_ptr(stream)))
        return out

    def project_function(self, ic, stream=None):
        """Projects a function ic(x, y) -> [..., 4] (evaluated on the host) onto the basis."""
        import torch
        xy = self.volume_points(stream).cpu().numpy()
        u = torch.from_numpy(np.ascontiguousarray(ic(xy[..., 0], xy[..., 1]))).cuda()
        return self.project_ic(u, stream=stream)
