"""dg_rhs_noalloc: the RHS for callers that cannot allocate device memory when
they evaluate it (a host whose GPU memory is all held by another allocator, or a
loop that must not pay an allocation's cost).  Its work space is the library's
fixed 64 MiB static device array.  The test calls it through the C ABI twice in a
row, on two different states, in every precision mode (float64, 1xTF32, 3xTF32:
the tensor-core modes lay out float32 traces, float32 fluxes and the fluxes'
float64 mean-mode integrals inside the array) and on both volume rules, and
compares each result with dg_rhs at the same precision: the launches are the
same, so the results agree bit for bit.  It also checks that a mesh needing more
work space than the array holds is refused.  Kept in a file of its own that
pytest collects last."""
import ctypes

import numpy as np
import pytest

from paper_1601_07944_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-12      # the float64 parity bound of the GPU tests


@pytest.fixture(scope="module")
def dgmod():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1601_07944_gb300 import _build, dg
    _build.build()
    dg.load()
    return dg


PREC = {"fp64": 0, "tf32x1": 1, "tf32x3": 2}


def _call_noalloc(dgmod, m, c, r, prec="fp64"):
    import torch
    lib = dgmod.load()
    st = lib.dg_rhs_noalloc(m.handle, ctypes.c_void_p(c.data_ptr()), ctypes.c_void_p(r.data_ptr()), PREC[prec],
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, lib.dg_last_error().decode()


@pytest.mark.parametrize("prec", ["fp64", "tf32x1", "tf32x3"])
@pytest.mark.parametrize("rule", ["collapsed", "symmetric"])
def test_noalloc_rhs_matches_rhs_on_two_calls(dgmod, prec, rule):
    import torch
    mesh = I.periodic_mesh(16)
    m = dgmod.Mesh.from_mesh(mesh, 3, vol_rule=rule)
    states = [m.project_function(I.vortex), m.project_function(I.perturbed_vortex)]
    for c in states:
        ref = m.rhs(c, precision=prec)
        out = torch.full_like(c, float("nan"))
        st, msg = _call_noalloc(dgmod, m, c, out, prec)
        assert st == 0, msg
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.array_equal(a, b), np.linalg.norm(a - b) / np.linalg.norm(b)
        assert np.linalg.norm(a - b) <= TOL * np.linalg.norm(b)
    m.device_status()


def test_noalloc_rejects_meshes_beyond_the_array(dgmod):
    import torch
    mesh = I.periodic_mesh(256)           # needs 9,437,184 doubles of work space
    m = dgmod.Mesh.from_mesh(mesh, 3)
    c = torch.zeros(m.coef_shape, dtype=torch.float64, device="cuda")
    r = torch.empty_like(c)
    st, msg = _call_noalloc(dgmod, m, c, r)
    assert st == 1 and "8388608" in msg and "9437184" in msg
