"""The n-point transverse routine (plan t_kind = 1, cell-centred meshes) and
its staged persistent form (t_kind = 2: rows copied in by TMA bulk copies,
one CTA per SM looping over planes) against the same references as the
default routine: the padded four-term transverse stage per kz plane, and full
solves against the FP64 oracle."""
import numpy as np
import pytest
import torch

from inputs.bunches import Geometry, Grid, cell_centred, random_density
from oracle import pipe
from test_gpu_parity import F32_TOL, F64_TOL, GEOMS, _transverse_reference, dev, host, rel, solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_4971_gb300 import build
    build.build()


CELL = {
    "cc16x16x32": GEOMS["cc16x16x32"],
    "rect32x32x64": GEOMS["rect32x32x64"],
    "aliased32x32x32": GEOMS["aliased32x32x32"],
    "rect64x64x32": cell_centred(3.0, 1.0, 64, 64, 32, 0.05, modes=20),
    "sq128x128x32": cell_centred(1.0, 1.0, 128, 128, 32, 0.02, modes=20),
}


def _plan(s, threads, kind=1):
    p = s.plan
    s.set_plan(z_warps=p["z_warps"], z_pipe=p["z_pipe"], t_h=1, t_threads=threads, t_kind=kind)


def _staged_fits(nx, dtype, threads):
    """Shared memory of the staged form (plane, phases, FFT scratch, staged rows)."""
    c = 16 if dtype == torch.float64 else 8
    g = 4 if nx <= 32 else 8
    sstride = (nx // g) * (g + 1) + 8
    rows = min((threads // 32) * (32 // g), nx)
    return c * (nx * nx + 2 * nx + (threads // g) * sstride + rows * nx) + 32 <= 227 * 1024


@pytest.mark.parametrize("kind", [1, 2])
@pytest.mark.parametrize("threads", [128, 256, 512])
@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 5e-6)])
@pytest.mark.parametrize("key", list(CELL))
def test_stage_transverse_npoint(key, dtype, tol, threads, kind):
    geom, grid = CELL[key]
    if dtype == torch.float64 and grid.nx > 64 and threads == 512:
        pytest.skip("FP64 128^2 planes (global scratch) run at 128 or 256 threads")
    if kind == 2 and not _staged_fits(grid.nx, dtype, threads):
        pytest.skip("staged form does not fit in shared memory at this size")
    s = solver(geom, grid, 1, dtype)
    _plan(s, threads, kind)
    rng = np.random.default_rng(grid.nx + threads)
    P = rng.standard_normal((grid.nz + 1, grid.nx, grid.ny)) \
        + 1j * rng.standard_normal((grid.nz + 1, grid.nx, grid.ny))
    cdt = torch.complex128 if dtype == torch.float64 else torch.complex64
    for adj in (0, 1):
        spec = torch.tensor(P, dtype=cdt, device="cuda")
        s.stage_transverse(spec, adjoint=adj)
        want = _transverse_reference(P, geom, grid, 1, adj)
        assert rel(spec.cpu().numpy(), want) < tol, (adj, rel(spec.cpu().numpy(), want))
    assert s.status() == 0


@pytest.mark.parametrize("kind", [1, 2])
@pytest.mark.parametrize("igf", [0, 1])
@pytest.mark.parametrize("key", ["rect32x32x64", "rect64x64x32", "sq128x128x32"])
def test_solve_and_adjoint_npoint_against_oracle(key, igf, kind):
    geom, grid = CELL[key]
    rho = random_density(grid.shape, 200 + igf, sparsity=0.3)
    spectra = pipe.green_spectra(geom, grid, igf)
    want = pipe.fft_solve(rho, geom, grid, igf, spectra=spectra)
    want_adj = pipe.fft_adjoint(rho, geom, grid, igf, spectra=spectra)
    for dtype, tol in ((torch.float64, F64_TOL), (torch.float32, F32_TOL)):
        if kind == 2 and dtype == torch.float64 and grid.nx > 64:
            continue                                     # FP64 128^2: kind 1 only
        s = solver(geom, grid, igf, dtype)
        threads = 256 if dtype == torch.float64 or grid.nx < 64 or kind == 2 else 512
        _plan(s, threads, kind)
        assert s.plan["t_kind"] == kind
        assert rel(host(s.solve(dev(rho, dtype))), want) <= tol
        assert rel(host(s.adjoint(dev(rho, dtype))), want_adj) <= tol
        assert s.status() == 0


def test_staged_npoint_equals_plane_per_cta_bitwise_on_the_bench_grid():
    """128^2 x 1024 FP32 (1025 planes, about 7 per CTA): the staged persistent
    form does the same arithmetic as the plane-per-CTA form, so the solves
    agree bit for bit, in both directions and on two calls in a row."""
    from inputs import bunches
    w = bunches.workload_throughput_128()
    geom, grid, rho = w["geom"], w["grid"], w["rho"][0]
    s = solver(geom, grid, 1, torch.float32)
    x = dev(rho, torch.float32)
    _plan(s, 256, 1)
    a, a_adj = host(s.solve(x)), host(s.adjoint(x))
    _plan(s, 256, 2)
    for _ in range(2):
        assert np.array_equal(host(s.solve(x)), a)
        assert np.array_equal(host(s.adjoint(x)), a_adj)
    assert s.status() == 0


def test_npoint_matches_padded_routine_on_the_bench_grid():
    """128^2 x 1024 FP32: the two routines agree to rounding on the long bunch."""
    from inputs import bunches
    w = bunches.workload_throughput_128()
    geom, grid, rho = w["geom"], w["grid"], w["rho"][0]
    s = solver(geom, grid, 1, torch.float32)
    s.set_plan(z_warps=8, z_pipe=0, t_h=1, t_threads=512, t_kind=0)
    a = host(s.solve(dev(rho, torch.float32)))
    _plan(s, 512)
    b = host(s.solve(dev(rho, torch.float32)))
    assert rel(b, a) <= 2e-6


def test_npoint_plan_refused_where_it_does_not_apply():
    from paper_1111_4971_gb300 import PipeError
    geom, grid = GEOMS["wall16x16x64"]                  # x0 = 0: s = 0
    s = solver(geom, grid, 1, torch.float64)
    with pytest.raises(PipeError):
        s.set_plan(z_warps=8, z_pipe=0, t_h=1, t_threads=256, t_kind=1)
    geom, grid = CELL["sq128x128x32"]
    s = solver(geom, grid, 1, torch.float64)
    s.set_plan(z_warps=8, z_pipe=0, t_h=1, t_threads=256, t_kind=1)
    assert s.plan["t_kind"] == 1                         # FP64 128^2: global scratch planes
    with pytest.raises(PipeError):                      # one CTA per plane only
        s.set_plan(z_warps=8, z_pipe=0, t_h=2, t_threads=256, t_kind=1)
    with pytest.raises(PipeError):                      # staged form: planes in shared memory only
        s.set_plan(z_warps=8, z_pipe=0, t_h=1, t_threads=256, t_kind=2)
    geom, grid = GEOMS["wall16x16x64"]
    s = solver(geom, grid, 1, torch.float32)
    with pytest.raises(PipeError):
        s.set_plan(z_warps=8, z_pipe=0, t_h=1, t_threads=256, t_kind=2)


def test_staged_wait_gives_up_records_timeout_and_recovers():
    """Failure detection without a GPU fault: the first CTA leaves out one of
    its own bulk copies, so its wait has nothing to wait for.  The bounded
    wait gives up, PIPE_ETIMEOUT reaches the host through pipe_status, the
    kernel still ends, and the next solve is exact again."""
    from paper_1111_4971_gb300 import _lib
    geom, grid = CELL["sq128x128x32"]
    s = solver(geom, grid, 1, torch.float32)
    _plan(s, 256, 2)
    x = dev(random_density(grid.shape, 7, sparsity=0.2), torch.float32)
    want = host(s.solve(x))
    assert s.status() == _lib.PIPE_OK
    for drop in (0, 2):                    # the first plane's first copy; a later one
        s.inject_stage_fault(drop_copy=drop, poll_limit=2048)
        s.solve(x)
        torch.cuda.synchronize()
        assert s.status() == _lib.PIPE_ETIMEOUT
        assert s.status() == _lib.PIPE_OK                # read and cleared
        assert np.array_equal(host(s.solve(x)), want)
        assert s.status() == _lib.PIPE_OK
