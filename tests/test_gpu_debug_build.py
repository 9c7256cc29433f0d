"""The index-checking build (libdg_debug.so, -DDG_DEBUG): every kernel checks each
connectivity index it reads before using it and records a bad one, which
dg_device_status reports as DG_EMESH (compute-sanitizer is not available, so this
build stands in for a memory checker).  A fresh process loads that build and runs
every kind of call -- all precisions, steppers, the limiter, boundary faces, the
adjoint and the no-allocation RHS, on both volume rules -- on meshes with ragged
last tiles, then
requires a clean device record and parity with the oracle.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
import oracle
from paper_1601_07944_gb300 import dg, inputs as I
lib = dg.load()
assert lib._name.endswith("libdg_debug.so"), lib._name

def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))

for mesh, ic in ((I.periodic_mesh(6), I.perturbed_vortex),
                 (I.box_mesh(6, x_code=I.BC_WALL, y_code=I.BC_STATE), I.steady_vortex)):
    for p, rule in ((1, "collapsed"), (3, "collapsed"), (5, "collapsed"), (2, "symmetric"), (5, "symmetric")):
        m = dg.Mesh.from_mesh(mesh, p, vol_rule=rule)
        o = oracle.OracleDG.from_mesh(mesh, p, vol_rule=rule)
        if m.n_boundary:
            xy = m.boundary_points().cpu().numpy()
            m.set_boundary_state(torch.from_numpy(ic(xy[..., 0], xy[..., 1])).cuda())
            oxy = o.boundary_points()
            o.set_boundary_state(ic(oxy[..., 0], oxy[..., 1]))
        c0 = o.project_ic(ic)
        c = torch.from_numpy(c0).cuda()
        assert rel(m.rhs(c).cpu().numpy(), o.rhs(c0)) < 1e-12
        r = torch.empty_like(c)
        m.rhs_noalloc(c, out=r)
        for prec in ("tf32x3", "tf32x1"):
            m.rhs(c, precision=prec)
        dt = I.fixed_dt(mesh, ic, p)
        for method in ("ssp_rk3", "rk2", "rk4"):
            x = c.clone()
            m.rk_step(x, dt, 18, method=method)
            assert rel(x.cpu().numpy(), getattr(o, method)(c0, dt, 18)) < 1e-12
            y = c.clone()
            m.rk_step(y, dt, 3, precision="tf32x3", method=method)
        m.adjoint_step(c, dt, torch.randn_like(c))
        if p == 1:
            m.set_limiter(True)
            z = c.clone()
            m.limit(z)
            m.rk_step(z, dt, 5)
            m.set_limiter(False)
        m.device_status()                 # raises on DG_EMESH (an index out of range)
print("debug build clean")
'''


def test_index_checking_build_runs_clean(oracle_mod):
    from paper_1601_07944_gb300 import _build
    lib = _build.build(debug=True)
    env = dict(os.environ, DG_LIB=lib)
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + SCRIPT], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "debug build clean" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
