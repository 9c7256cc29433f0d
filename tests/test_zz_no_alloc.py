"""dg_rhs_noalloc: the RHS for callers that cannot allocate device memory when
they evaluate it (a host whose GPU memory is all held by another allocator, or a
loop that must not pay an allocation's cost).  Its work space is the library's
fixed 64 MiB static device array.  The test calls it through the C ABI twice in a
row, on two different states, and compares each result with dg_rhs; it also
checks that a mesh needing more work space than the array holds is refused.
Kept in a file of its own that pytest collects last."""
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


def _call_noalloc(dgmod, m, c, r):
    import torch
    lib = dgmod.load()
    st = lib.dg_rhs_noalloc(m.handle, ctypes.c_void_p(c.data_ptr()), ctypes.c_void_p(r.data_ptr()), 0,
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, lib.dg_last_error().decode()


def test_noalloc_rhs_matches_rhs_on_two_calls(dgmod):
    import torch
    mesh = I.periodic_mesh(16)
    m = dgmod.Mesh.from_mesh(mesh, 3)
    states = [m.project_function(I.vortex), m.project_function(I.perturbed_vortex)]
    for c in states:
        ref = m.rhs(c)
        out = torch.full_like(c, float("nan"))
        st, msg = _call_noalloc(dgmod, m, c, out)
        assert st == 0, msg
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.linalg.norm(a - b) <= TOL * np.linalg.norm(b)


def test_noalloc_rejects_meshes_beyond_the_array(dgmod):
    import torch
    mesh = I.periodic_mesh(256)           # needs 9,437,184 doubles of work space
    m = dgmod.Mesh.from_mesh(mesh, 3)
    c = torch.zeros(m.coef_shape, dtype=torch.float64, device="cuda")
    r = torch.empty_like(c)
    st, msg = _call_noalloc(dgmod, m, c, r)
    assert st == 1 and "8388608" in msg and "9437184" in msg
