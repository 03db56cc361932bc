"""pipe_poisson_solve_noalloc: the solve whose working buffer is the library's
fixed device array instead of device memory allocated for the handle.

It exists for programs that must not let a library allocate device memory
while they run (a host that has handed the GPU's memory to its own pool, a
loop that cannot risk an allocation stalling or failing).  Through the C ABI
this test checks, on two calls in a row (the second call reuses the array the
first one left behind), that it gives bit for bit the potential of
pipe_poisson_solve (the same kernels on the same plan, only the working
buffer differs) and agrees with the FP64 oracle; that a call takes no device
memory (free memory unchanged across it); and that a mesh too large for the
array is refused.  Both forms of the solve run through it: the padded
transforms (including the staged transverse kernel at 128 x 128) and the
mode-space form.  Collected last on purpose (file name) so that a failure
here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest
import torch

from inputs import bunches
from inputs.bunches import cell_centred, gaussian_bunch
from oracle import pipe

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


def _noalloc(L, solver, rho, out):
    st = L.pipe_poisson_solve_noalloc(solver.handle, ctypes.c_void_p(rho.data_ptr()),
                                      ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, L.pipe_strerror(st)
    return out


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _plan(s, form):
    if form == "modes":
        s.set_plan(t_kind=3)
    else:
        p = s.plan
        kind = 2 if (s.dtype == torch.float32 and s.shape[0] == 128) else 1
        s.set_plan(z_warps=p["z_warps"], z_pipe=0, t_h=1, t_threads=256, t_kind=kind)


CASES = [
    # 64x64x256 IGF rectangular pipe, the three seeded bunches
    ("igf64", "transforms", torch.float32), ("igf64", "transforms", torch.float64),
    ("igf64", "modes", torch.float32), ("igf64", "modes", torch.float64),
    # 128x128x256 FP32: 33.7 MB of transform workspace, the staged transverse kernel
    ("cc128x256", "transforms", torch.float32), ("cc128x256", "modes", torch.float32),
]


def _workload(name):
    if name == "igf64":
        w = bunches.workload_igf_64()
        return w["geom"], w["grid"], w["rho"][:2]
    geom, grid = cell_centred(1.0, 1.0, 128, 128, 256, 0.03)
    rhos = [gaussian_bunch(geom, grid, (0.5, 0.5, 3.8), (0.15, 0.15, 1.0)),
            gaussian_bunch(geom, grid, (0.4, 0.55, 3.0), (0.1, 0.2, 0.6))]
    return geom, grid, rhos


@pytest.mark.parametrize("name,form,dtype", CASES)
def test_noalloc_equals_solve_bitwise_matches_oracle_and_allocates_nothing(L, name, form, dtype):
    from paper_1111_4971_gb300 import PipeSolver
    geom, grid, rhos = _workload(name)
    s = PipeSolver(geom, grid, igf=True, dtype=dtype)
    _plan(s, form)
    tol = F32_TOL if dtype == torch.float32 else F64_TOL
    out = s.empty()
    for k, rho_np in enumerate(rhos):                 # two calls in a row
        rho = torch.tensor(rho_np, dtype=dtype, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        _noalloc(L, s, rho, out)
        torch.cuda.synchronize()
        if k > 0:                                     # the first call may load the module's code
            assert torch.cuda.mem_get_info()[0] == free0
        want = s.solve(rho)
        torch.cuda.synchronize()
        assert torch.equal(out, want)
        assert _rel(out.double().cpu().numpy(), pipe.fft_solve(rho_np, geom, grid, 1)) <= tol


def test_noalloc_refuses_meshes_beyond_the_array(L):
    from paper_1111_4971_gb300 import PipeSolver
    geom, grid = cell_centred(1.0, 1.0, 128, 128, 512, 0.02)   # 67 MB of transform workspace in FP32
    s = PipeSolver(geom, grid, igf=True, dtype=torch.float32)
    _plan(s, "transforms")
    rho = torch.zeros(grid.shape, dtype=torch.float32, device="cuda")
    out = s.empty()
    st = L.pipe_poisson_solve_noalloc(s.handle, ctypes.c_void_p(rho.data_ptr()),
                                      ctypes.c_void_p(out.data_ptr()), None)
    assert st == 3                                 # PIPE_EUNSUPPORTED
