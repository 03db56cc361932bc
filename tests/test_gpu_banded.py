"""The banded reduction of Sec. 5 (Eq. 17-18) through the C ABI against the
FP64 oracle: its 2-D Green spectra, solves for several band widths, the full
band, symmetry of the operator, and the entry points that refuse it."""
import numpy as np
import pytest
import torch

from inputs.bunches import Geometry, Grid, cell_centred, gaussian_bunch, random_density
from oracle import pipe
from test_gpu_parity import F32_TOL, F64_TOL, dev, host, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_4971_gb300 import build
    build.build()


def solver(geom, grid, igf, n_nb, dtype):
    from paper_1111_4971_gb300 import PipeSolver
    return PipeSolver(geom, grid, igf=igf, dtype=dtype, banded=n_nb)


CASES = {
    "cc16x16x32": cell_centred(2.0, 2.0, 16, 16, 32, 0.1, modes=20),
    "rect32x32x64": cell_centred(2.0, 1.0, 32, 32, 64, 0.0625, modes=20),
    "rect64x64x32": cell_centred(3.0, 1.0, 64, 64, 32, 0.05, modes=20),
    "sq128x128x32": cell_centred(1.0, 1.0, 128, 128, 32, 0.02, modes=20),
}


@pytest.mark.parametrize("igf", [0, 1])
def test_banded_green_spectra(igf):
    geom, grid = CASES["rect32x32x64"]
    n_nb = 3
    got = solver(geom, grid, igf, n_nb, torch.float64).green_spectrum()     # [d][ky][kx]
    T = pipe.green_tables(geom, grid, igf)["cc"]
    scale = pipe.h3(grid) / (4.0 * grid.nx * grid.ny)
    for d in range(n_nb + 1):
        S = np.fft.fft2(T[:, :, d])[:grid.nx + 1, :grid.ny + 1]             # [kx][ky]
        assert np.abs(S.imag).max() <= 1e-12 * np.abs(S.real).max()
        want = scale * S.real.T
        assert np.abs(got[d] - want).max() <= 1e-13 * np.abs(want).max()


@pytest.mark.parametrize("threads", [128, 256, 512])
@pytest.mark.parametrize("n_nb", [0, 1, 3])
@pytest.mark.parametrize("key", list(CASES))
def test_banded_solve_against_oracle(key, n_nb, threads):
    geom, grid = CASES[key]
    rho = random_density(grid.shape, 300 + n_nb, sparsity=0.3)
    for igf in (0, 1):
        want = pipe.banded_solve(rho, geom, grid, igf, n_nb)
        for dtype, tol in ((torch.float64, F64_TOL), (torch.float32, F32_TOL)):
            if dtype == torch.float64 and grid.nx > 64:
                continue
            s = solver(geom, grid, igf, n_nb, dtype)
            s.set_plan(z_warps=8, z_pipe=0, t_h=1, t_threads=threads, t_kind=1)
            got = host(s.solve(dev(rho, dtype)))
            assert rel(got, want) <= tol, (igf, dtype, rel(got, want))


def test_full_band_equals_full_solve_and_operator_is_symmetric():
    geom, grid = CASES["cc16x16x32"]
    rho = random_density(grid.shape, 41)
    full = pipe.fft_solve(rho, geom, grid, 1)
    s = solver(geom, grid, 1, grid.nz - 1, torch.float64)
    assert rel(host(s.solve(dev(rho, torch.float64))), full) <= F64_TOL
    s = solver(geom, grid, 1, 2, torch.float64)
    r1, r2 = random_density(grid.shape, 42), random_density(grid.shape, 43)
    a1 = host(s.solve(dev(r1, torch.float64)))
    t2 = host(s.adjoint(dev(r2, torch.float64)))
    assert abs(np.sum(a1 * r2) - np.sum(r1 * t2)) <= 1e-13 * abs(np.sum(a1 * r2))
    assert np.array_equal(host(s.adjoint(dev(r1, torch.float64))), a1)


def test_long_bunch_band_converges_at_the_slowest_mode_rate():
    """A bunch 30 pipe widths long on a coarse z mesh (hz = 1.875 a): every
    further neighbour plane cuts the difference to the full solve by the
    fall-off of the slowest mode over one plane, e^{-kappa_11 hz} with
    kappa_11 = pi sqrt(1/a^2 + 1/b^2) (Eq. 9, 15) -- the reason Sec. 5 can
    keep only a few planes."""
    geom, grid = cell_centred(1.0, 1.0, 64, 64, 128, 240.0 / 128, modes=20)
    rho = gaussian_bunch(geom, grid, (0.5, 0.5, 120.0), (0.15, 0.15, 30.0))
    from paper_1111_4971_gb300 import PipeSolver
    full = host(PipeSolver(geom, grid, igf=True, dtype=torch.float64).solve(dev(rho, torch.float64)))
    e = {}
    for n_nb in (0, 1, 2):
        e[n_nb] = rel(host(solver(geom, grid, 1, n_nb, torch.float64).solve(dev(rho, torch.float64))), full)
    print("banded vs full, long bunch:", e)
    r = np.exp(-np.pi * np.sqrt(2.0) * grid.hz)
    assert 0.05 < e[0] < 0.2
    assert 0.5 * r < e[1] / e[0] < 2.0 * r
    assert 0.5 * r < e[2] / e[1] < 2.0 * r


def test_banded_handle_refused_by_other_entry_points():
    from paper_1111_4971_gb300 import PipeError, PipeSolver, solve_batched
    geom, grid = CASES["cc16x16x32"]
    s = solver(geom, grid, 1, 1, torch.float32)
    spec = s.spectrum_buffer()
    with pytest.raises(PipeError):
        s.stage_transverse(spec)
    other = PipeSolver(geom, grid, igf=True, dtype=torch.float32)
    rho = dev(random_density(grid.shape, 1), torch.float32)
    with pytest.raises(PipeError):
        solve_batched([s, other], [rho, rho], [s.empty(), other.empty()])
    with pytest.raises(PipeError):
        solver(geom, grid, 1, grid.nz, torch.float32)
    # a banded handle the mode form cannot take either (more than 32 modes on a
    # wall-node mesh, which the banded transform kernels do not take)
    with pytest.raises(PipeError):
        solver(type(geom)(geom.a, geom.b, 0.0, 0.0, 40, 40), grid, 1, 1, torch.float32)


# the banded operator in mode space (plan t_kind 3): projection, a
# (2 n_nb + 1)-tap stencil on each mode column, back-projection
MODE_CASES = dict(CASES)
# node on the wall, unequal mode counts: only the mode form takes it
MODE_CASES["wall32x16x64"] = (Geometry(1.0, 0.5, 0.0, 0.0, 12, 9), Grid(32, 16, 64, 1 / 32, 0.5 / 16, 0.05))
# nx != ny, not a power of two
MODE_CASES["cc48x32x64"] = cell_centred(1.5, 1.0, 48, 32, 64, 0.05, modes=16)


@pytest.mark.parametrize("n_nb", [0, 1, 3])
@pytest.mark.parametrize("key", list(MODE_CASES))
def test_banded_mode_form_against_oracle(key, n_nb):
    geom, grid = MODE_CASES[key]
    rho = random_density(grid.shape, 500 + n_nb, sparsity=0.3)
    for igf in (0, 1):
        want = pipe.banded_solve(rho, geom, grid, igf, n_nb)
        for dtype, tol in ((torch.float64, F64_TOL), (torch.float32, F32_TOL)):
            s = solver(geom, grid, igf, n_nb, dtype)
            if s.plan["t_kind"] != 3:
                s.set_plan(t_kind=3)
            assert s.plan["t_kind"] == 3
            got = host(s.solve(dev(rho, dtype)))
            assert rel(got, want) <= tol, (igf, dtype, rel(got, want))
            # symmetric operator: the adjoint is the same computation
            assert torch.equal(s.adjoint(dev(rho, dtype)), s.solve(dev(rho, dtype)))


def test_banded_mode_form_full_band_and_default():
    """The band covering every plane is the full operator; on 64^2 and wider
    planes (modes at most half the mesh) the mode form is the banded default."""
    from paper_1111_4971_gb300 import PipeSolver
    geom, grid = MODE_CASES["cc48x32x64"]
    rho = random_density(grid.shape, 44)
    full = host(PipeSolver(geom, grid, igf=True, dtype=torch.float64).solve(dev(rho, torch.float64)))
    s = solver(geom, grid, 1, grid.nz - 1, torch.float64)
    assert s.plan["t_kind"] == 3
    assert rel(host(s.solve(dev(rho, torch.float64))), full) <= F64_TOL
    g64, gr64 = CASES["rect64x64x32"]
    assert solver(g64, gr64, 1, 2, torch.float32).plan["t_kind"] == 3
