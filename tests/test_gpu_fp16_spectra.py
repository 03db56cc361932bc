"""Complex-FP16 spectra with per-slab scales (PIPE_F32_C16) against the FP64
oracle.  FP16 keeps 11 significant bits (unit roundoff u = 2^-11 = 4.9e-4).
The spectrum is rounded to FP16 after the z transform and after the
transverse stage, and both operands of the Green product are rounded, so the
relative L2 error of the potential is a small multiple of u: the bound used
here is 8u = 3.9e-3.  The FP32 path is checked against the same oracle to
show what the FP16 storage costs."""
import numpy as np
import pytest
import torch

from inputs import bunches
from inputs.bunches import cell_centred, random_density
from oracle import pipe
from test_gpu_parity import F32_TOL, dev, host, rel

pytestmark = pytest.mark.gpu

U16 = 2.0 ** -11
TOL16 = 8 * U16


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_4971_gb300 import build
    build.build()


def solvers(geom, grid, igf):
    from paper_1111_4971_gb300 import PipeSolver
    return (PipeSolver(geom, grid, igf=igf, dtype=torch.float32, fp16_spectra=True),
            PipeSolver(geom, grid, igf=igf, dtype=torch.float32))


@pytest.mark.parametrize("shape,modes", [((16, 16, 32), 20), ((32, 32, 64), 20), ((64, 64, 128), 20),
                                         ((128, 128, 32), 20)])
def test_fp16_spectra_against_oracle(shape, modes):
    nx, ny, nz = shape
    geom, grid = cell_centred(1.5, 1.0, nx, ny, nz, 0.05, modes=modes)
    rho = random_density(grid.shape, nx + nz, sparsity=0.3)
    for igf in (0, 1):
        want = pipe.fft_solve(rho, geom, grid, igf)
        want_adj = pipe.fft_adjoint(rho, geom, grid, igf)
        s16, s32 = solvers(geom, grid, igf)
        e16 = rel(host(s16.solve(dev(rho, torch.float32))), want)
        e32 = rel(host(s32.solve(dev(rho, torch.float32))), want)
        a16 = rel(host(s16.adjoint(dev(rho, torch.float32))), want_adj)
        print(f"{shape} igf={igf}: FP16 spectra {e16:.2e} (adjoint {a16:.2e}), FP32 {e32:.2e}")
        assert e16 <= TOL16 and a16 <= TOL16
        assert e32 <= F32_TOL
        assert e16 > e32                     # the FP16 rounding is visible


def test_fp16_spectra_bench_bunch_and_gradient_budget():
    """The 128^2 x 1024 long bunch: error of the FP16 variant against the FP64
    GPU path, and the field energy to FP16 accuracy."""
    from paper_1111_4971_gb300 import PipeSolver, field_energy
    w = bunches.workload_throughput_128()
    geom, grid, rho = w["geom"], w["grid"], w["rho"][0]
    p64 = host(PipeSolver(geom, grid, igf=True, dtype=torch.float64).solve(dev(rho, torch.float64)))
    s16 = PipeSolver(geom, grid, igf=True, dtype=torch.float32, fp16_spectra=True)
    r16 = dev(rho, torch.float32)
    p16 = s16.solve(r16)
    e = rel(host(p16), p64)
    print(f"128^2x1024 long bunch: FP16 spectra vs FP64 path {e:.2e}")
    assert e <= TOL16
    W16 = float(field_energy(r16, p16))
    W64 = 0.5 * float(np.sum(rho * p64))
    assert abs(W16 - W64) <= TOL16 * abs(W64)


def test_fp16_spectra_refused_where_not_built():
    from paper_1111_4971_gb300 import PipeError, PipeSolver
    geom, grid = bunches.Geometry(1.0, 0.5, 0.0, 0.0, 12, 9), bunches.Grid(16, 16, 64, 1 / 16, 0.5 / 16, 0.05)
    with pytest.raises(PipeError):                         # x0 = 0 (s = 0): n-point routine only
        PipeSolver(geom, grid, igf=True, dtype=torch.float32, fp16_spectra=True)
    geom, grid = cell_centred(1.0, 1.0, 16, 16, 32, 0.05)
    s = PipeSolver(geom, grid, igf=True, dtype=torch.float32, fp16_spectra=True)
    with pytest.raises(PipeError):
        s.stage_transverse(s.spectrum_buffer())
    with pytest.raises(PipeError):
        PipeSolver(geom, grid, igf=True, dtype=torch.float32, fp16_spectra=True, banded=1)
