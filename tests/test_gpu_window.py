"""Transverse-window meshes (Sec. 5: a small transverse mesh inside the pipe,
not spanning it, at any origin) through the general four-table form of
Eq. 10, against the FP64 oracle: the transformed tables, the transverse
stage, solves and adjoints, and the window of a spanning-mesh solve."""
import numpy as np
import pytest
import torch

from inputs.bunches import Geometry, Grid, cell_centred, gaussian_bunch, random_density
from oracle import pipe
from test_gpu_parity import F32_TOL, F64_TOL, _transverse_reference, dev, host, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_4971_gb300 import build
    build.build()


def solver(geom, grid, igf, dtype, threads=None):
    from paper_1111_4971_gb300 import PipeSolver
    s = PipeSolver(geom, grid, igf=igf, dtype=dtype)
    if threads:
        p = s.plan
        s.set_plan(z_warps=p["z_warps"], z_pipe=p["z_pipe"], t_h=1, t_threads=threads, t_kind=0)
    return s


WINDOWS = {
    # a 16 x 16 window of spacing 0.1 at an arbitrary origin in a 3 x 2 pipe
    "w16x16x32": (Geometry(3.0, 2.0, 0.37, 0.21, 12, 10), Grid(16, 16, 32, 0.1, 0.08, 0.05)),
    # a centred 32 x 32 window, a quarter of the pipe width
    "w32x32x64": (Geometry(1.0, 1.0, 0.375 + 0.5 / 128, 0.375 + 0.5 / 128, 20, 20),
                  Grid(32, 32, 64, 1 / 128, 1 / 128, 0.02)),
    # a 64 x 64 window, the largest plane of the general form
    "w64x64x32": (Geometry(2.0, 1.0, 0.3, 0.1, 20, 20), Grid(64, 64, 32, 0.02, 0.012, 0.04)),
}


@pytest.mark.parametrize("igf", [0, 1])
def test_window_spectra(igf):
    geom, grid = WINDOWS["w16x16x32"]
    s = solver(geom, grid, igf, torch.float64)
    got = s.green_spectrum()                                # (4, nz+1, 2ny, 2nx) complex
    T = pipe.green_tables(geom, grid, igf)
    scale = pipe.h3(grid) / (8.0 * grid.nx * grid.ny * grid.nz)
    for t, key in enumerate(("cc", "cr", "rc", "rr")):
        want = scale * np.fft.fftn(T[key])[:, :, :grid.nz + 1].transpose(2, 1, 0)
        assert np.abs(got[t] - want).max() <= 1e-12 * np.abs(want).max(), key


@pytest.mark.parametrize("threads", [128, 256])
@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 5e-6)])
@pytest.mark.parametrize("key", list(WINDOWS))
def test_window_stage_transverse(key, dtype, tol, threads):
    geom, grid = WINDOWS[key]
    s = solver(geom, grid, 1, dtype, threads)
    rng = np.random.default_rng(grid.nx + threads)
    P = rng.standard_normal((grid.nz + 1, grid.nx, grid.ny)) \
        + 1j * rng.standard_normal((grid.nz + 1, grid.nx, grid.ny))
    cdt = torch.complex128 if dtype == torch.float64 else torch.complex64
    for adj in (0, 1):
        spec = torch.tensor(P, dtype=cdt, device="cuda")
        s.stage_transverse(spec, adjoint=adj)
        want = _transverse_reference(P, geom, grid, 1, adj)
        assert rel(spec.cpu().numpy(), want) < tol, (adj, rel(spec.cpu().numpy(), want))


@pytest.mark.parametrize("igf", [0, 1])
@pytest.mark.parametrize("key", list(WINDOWS))
def test_window_solve_and_adjoint_against_oracle(key, igf):
    geom, grid = WINDOWS[key]
    rho = random_density(grid.shape, 500 + igf, sparsity=0.3)
    spectra = pipe.green_spectra(geom, grid, igf)
    want = pipe.fft_solve(rho, geom, grid, igf, spectra=spectra)
    want_adj = pipe.fft_adjoint(rho, geom, grid, igf, spectra=spectra)
    for dtype, tol in ((torch.float64, F64_TOL), (torch.float32, F32_TOL)):
        s = solver(geom, grid, igf, dtype)
        assert rel(host(s.solve(dev(rho, dtype))), want) <= tol
        assert rel(host(s.adjoint(dev(rho, dtype))), want_adj) <= tol


def test_window_equals_spanning_mesh_inside_it():
    """A bunch that lives inside a central window: the window solve equals the
    spanning-mesh solve on the window's nodes (same discrete sum, Eq. 4), one
    path using the real octant and the other the four general tables."""
    geom_f, grid_f = cell_centred(1.0, 1.0, 128, 128, 64, 0.02, modes=20)
    rho_f = gaussian_bunch(geom_f, grid_f, (0.5, 0.5, 0.63), (0.03, 0.03, 0.15), total_charge=None)
    i0 = 48                                               # window nodes 48..79 of the full mesh
    assert not rho_f[:i0].any() and not rho_f[i0 + 32:].any()
    assert not rho_f[:, :i0].any() and not rho_f[:, i0 + 32:].any()
    geom_w = Geometry(1.0, 1.0, geom_f.x0 + i0 * grid_f.hx, geom_f.y0 + i0 * grid_f.hy, 20, 20)
    grid_w = Grid(32, 32, 64, grid_f.hx, grid_f.hy, grid_f.hz)
    rho_w = rho_f[i0:i0 + 32, i0:i0 + 32, :]
    for dtype, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
        full = host(solver(geom_f, grid_f, 1, dtype).solve(dev(rho_f, dtype)))[i0:i0 + 32, i0:i0 + 32]
        win = host(solver(geom_w, grid_w, 1, dtype).solve(dev(rho_w, dtype)))
        assert rel(win, full) <= tol
