"""pipe_poisson_solve_noalloc: the solve whose working buffer is the library's
fixed device array instead of device memory allocated for the handle.

It exists for programs that must not let a library allocate device memory
while they run; this test checks, through the C ABI, that it gives the same
potential as pipe_poisson_solve on two calls in a row (the second call reuses
the array the first one left behind), and that a mesh too large for the
array is refused.  Collected last on purpose (file name) so that a failure
here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest
import torch

from inputs import bunches
from inputs.bunches import cell_centred

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5
F64_TOL = 1e-12


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_4971_gb300 import _lib, build
    build.build()
    return _lib.load()


def _noalloc(L, solver, rho):
    out = solver.empty()
    st = L.pipe_poisson_solve_noalloc(solver.handle, ctypes.c_void_p(rho.data_ptr()),
                                      ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, L.pipe_strerror(st)
    return out


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("dtype,tol", [(torch.float32, F32_TOL), (torch.float64, F64_TOL)])
def test_noalloc_matches_solve_on_two_calls(L, dtype, tol):
    from paper_1111_4971_gb300 import PipeSolver
    w = bunches.workload_igf_64()                  # 64x64x256: 8.4 MB of workspace in FP32
    s = PipeSolver(w["geom"], w["grid"], igf=True, dtype=dtype)
    for rho_np in w["rho"][:2]:                    # two calls in a row
        rho = torch.tensor(rho_np, dtype=dtype, device="cuda")
        got = _noalloc(L, s, rho)
        want = s.solve(rho)
        torch.cuda.synchronize()
        assert _rel(got, want) <= tol


def test_noalloc_refuses_meshes_beyond_the_array(L):
    from paper_1111_4971_gb300 import PipeSolver
    geom, grid = cell_centred(1.0, 1.0, 128, 128, 512, 0.02)   # 67 MB of workspace in FP32
    s = PipeSolver(geom, grid, igf=True, dtype=torch.float32)
    rho = torch.zeros(grid.shape, dtype=torch.float32, device="cuda")
    out = s.empty()
    st = L.pipe_poisson_solve_noalloc(s.handle, ctypes.c_void_p(rho.data_ptr()),
                                      ctypes.c_void_p(out.data_ptr()), None)
    assert st == 3                                 # PIPE_EUNSUPPORTED
