"""The mode-space form of the solve (plan t_kind 3) against the FP64 oracle.

The form evaluates the same discrete sum as Eq. 10 with the transverse
transforms pruned to the modes of the truncated series (Eq. 7): projection
onto the sine modes, zero-padded z convolution per mode, back-projection.
Full solves and adjoints are compared with O3 (scipy FFTs of Eq. 10) or O1
(brute force), element by element (relative L2; FP64 <= 1e-12, FP32 <= 1e-5),
on cell-centred, wall-node, window and rectangular (nx != ny) meshes; each
stage is compared with its plain definition; the full-size bench
configuration is checked at sampled nodes against the oracle's direct sum.
"""
import numpy as np
import pytest
import torch

from inputs import bunches
from inputs.bunches import Geometry, Grid, cell_centred, gaussian_bunch, random_density
from oracle import green, pipe

pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
F32_TOL = 1e-5


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def dev(x, dtype):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_4971_gb300 import build
    build.build()


def mode_solver(geom, grid, igf, dtype):
    from paper_1111_4971_gb300 import PipeSolver
    s = PipeSolver(geom, grid, igf=igf, dtype=dtype)
    if s.plan["t_kind"] != 3:
        s.set_plan(t_kind=3)
    assert s.plan["t_kind"] == 3
    return s


# meshes: (geometry, grid); the mode form needs nx, ny multiples of 16
MESHES = {
    # cell-centred, square pipe: symmetric in y (folded tables)
    "cc16x16x32": cell_centred(2.0, 2.0, 16, 16, 32, 0.1, modes=20),
    # rectangular pipe a/b = 2, cell-centred
    "rect32x32x64": cell_centred(2.0, 1.0, 32, 32, 64, 0.0625, modes=20),
    # node on the wall (x0 = y0 = 0): not symmetric in y, unequal modes
    "wall32x16x64": (Geometry(1.0, 0.5, 0.0, 0.0, 12, 9), Grid(32, 16, 64, 1 / 32, 0.5 / 16, 0.05)),
    # nx != ny and not a power of two: only the mode form takes it
    "cc48x32x64": cell_centred(1.5, 1.0, 48, 32, 64, 0.05, modes=16),
    # an off-centre window (Sec. 5): not symmetric, not spanning the pipe
    "window32x32x32": (Geometry(3.0, 2.0, 0.7, 0.45, 20, 20), Grid(32, 32, 32, 0.04, 0.035, 0.06)),
    # a centred window: symmetric in y
    "cwindow16x32x64": (Geometry(2.0, 1.5, 0.5 * (2.0 - 15 * 0.05), 0.5 * (1.5 - 31 * 0.025), 20, 20),
                        Grid(16, 32, 64, 0.05, 0.025, 0.05)),
}


def _density(geom, grid, seed):
    x = random_density(grid.shape, seed, sparsity=0.3)
    zc = 0.5 * (grid.nz - 1) * grid.hz
    xc = geom.x0 + 0.5 * (grid.nx - 1) * grid.hx
    yc = geom.y0 + 0.5 * (grid.ny - 1) * grid.hy
    return x + 5.0 * gaussian_bunch(geom, grid, (xc, yc, zc),
                                    (0.2 * grid.nx * grid.hx, 0.2 * grid.ny * grid.hy, 0.2 * grid.nz * grid.hz))


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("igf", [0, 1])
@pytest.mark.parametrize("dtype,tol", [(torch.float64, F64_TOL), (torch.float32, F32_TOL)])
def test_mode_solve_and_adjoint_against_oracle(name, igf, dtype, tol):
    geom, grid = MESHES[name]
    rho = _density(geom, grid, seed=11 + igf)
    want = pipe.fft_solve(rho, geom, grid, igf)
    s = mode_solver(geom, grid, igf, dtype)
    got = host(s.solve(dev(rho, dtype)))
    assert rel(got, want) <= tol, (name, rel(got, want))
    # the operator is symmetric: its adjoint is the oracle's transposed sum
    dphi = random_density(grid.shape, 99 + igf)
    want_adj = pipe.fft_adjoint(dphi, geom, grid, igf)
    got_adj = host(s.adjoint(dev(dphi, dtype)))
    assert rel(got_adj, want_adj) <= tol, (name, rel(got_adj, want_adj))


def test_mode_solve_against_brute_force_sum():
    """Config 1 (16x16x32, ordinary G, FP64) through the mode form against O1."""
    w = bunches.workload_fp64_ordinary_16()
    geom, grid, rho = w["geom"], w["grid"], w["rho"][0]
    want = pipe.direct_sum(rho, geom, grid, 0)
    s = mode_solver(geom, grid, 0, torch.float64)
    assert rel(host(s.solve(dev(rho, torch.float64))), want) <= F64_TOL


def test_mode_and_transform_forms_agree_on_igf64():
    """The IGF 64x64x256 rectangular-pipe workload: the two forms of the same
    operator, FP64, on all three seeded bunches, and the FP32 mode form against
    the FP64 oracle."""
    from paper_1111_4971_gb300 import PipeSolver
    w = bunches.workload_igf_64()
    geom, grid = w["geom"], w["grid"]
    sm = mode_solver(geom, grid, 1, torch.float64)
    sf = PipeSolver(geom, grid, igf=True, dtype=torch.float64)
    p = sf.plan
    if p["t_kind"] == 3:
        sf.set_plan(z_warps=8, z_pipe=0, t_h=1, t_threads=256, t_kind=1)
    s32 = mode_solver(geom, grid, 1, torch.float32)
    for rho in w["rho"]:
        a = host(sm.solve(dev(rho, torch.float64)))
        b = host(sf.solve(dev(rho, torch.float64)))
        assert rel(a, b) <= F64_TOL
        want = pipe.fft_solve(rho, geom, grid, 1)
        assert rel(a, want) <= F64_TOL
        assert rel(host(s32.solve(dev(rho, torch.float32))), want) <= F32_TOL


# ---------------------------------------------------------------------------
# stages against their plain definitions
# ---------------------------------------------------------------------------

def _tables(s, geom, grid):
    """The sine tables of the layout (slot -> mode) and the mode numbers."""
    mx, mxp, myp, fold, xb = s.mode_layout()
    x = geom.x0 + grid.hx * np.arange(grid.nx)
    y = geom.y0 + grid.hy * np.arange(grid.ny)
    mslot = np.arange(1, mxp + 1)
    if fold:
        nslot = np.array([2 * q + 1 if q < myp // 2 else 2 * (q - myp // 2) + 2 for q in range(myp)])
    else:
        nslot = np.arange(1, myp + 1)
    sx = np.sin(np.pi * mslot[:, None] * x[None, :] / geom.a) * (mslot <= geom.modes_m)[:, None]
    sy = np.sin(np.pi * nslot[:, None] * y[None, :] / geom.b) * (nslot <= geom.modes_n)[:, None]
    return sx, sy, mslot, nslot, (mx, mxp, myp, fold, xb)


@pytest.mark.parametrize("name", ["cc16x16x32", "wall32x16x64", "cc48x32x64"])
@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-13), (torch.float32, 2e-6)])
def test_mode_stages(name, dtype, tol):
    geom, grid = MESHES[name]
    igf = 1
    s = mode_solver(geom, grid, igf, dtype)
    sx, sy, mslot, nslot, (mx, mxp, myp, fold, xb) = _tables(s, geom, grid)
    rho = _density(geom, grid, seed=5)
    part, psi = s.mode_buffers()
    # projection, per block of x rows
    s.stage_modes(0, dev(rho, dtype), part)
    rows = grid.nx // xb
    want = np.stack([np.einsum("mi,nj,ijk->mnk", sx[:, b * rows:(b + 1) * rows], sy,
                               rho[b * rows:(b + 1) * rows]).reshape(mxp * myp, grid.nz)
                     for b in range(xb)])
    assert rel(host(part), want) <= tol
    # z convolution: the linear convolution with K_mn(d), d = k - k'
    pin = want.sum(axis=0)
    s.stage_modes(1, dev(want, dtype), psi)
    kap = green.kappa(mslot[:, None], nslot[None, :], geom.a, geom.b)       # (mxp, myp)
    d = (np.arange(grid.nz)[:, None] - np.arange(grid.nz)[None, :]) * grid.hz
    prof = green.z_profile(d[None, None], kap[:, :, None, None], grid.hz, igf) / kap[:, :, None, None]
    live = (mslot[:, None] <= geom.modes_m) & (nslot[None, :] <= geom.modes_n)
    K = green.prefactor_G(geom) * grid.hx * grid.hy * grid.hz * prof * live[:, :, None, None]
    want_psi = np.einsum("mnkq,mnq->mnk", K, pin.reshape(mxp, myp, grid.nz)).reshape(mxp * myp, grid.nz)
    assert rel(host(psi), want_psi) <= tol
    # back-projection
    phi = s.empty()
    s.stage_modes(2, dev(want_psi, dtype), phi)
    want_phi = np.einsum("mi,nj,mnk->ijk", sx, sy, want_psi.reshape(mxp, myp, grid.nz))
    assert rel(host(phi), want_phi) <= tol


def test_mode_spectrum_is_the_dct_of_the_kernel_table():
    """pipe_mode_spectrum against the DFT of the doubled z table of K_mn
    (free slot d = nz filled by the formula), divided by 2 nz."""
    geom, grid = MESHES["rect32x32x64"]
    for igf in (0, 1):
        s = mode_solver(geom, grid, igf, torch.float64)
        sx, sy, mslot, nslot, (mx, mxp, myp, fold, xb) = _tables(s, geom, grid)
        got = s.mode_spectrum().reshape(mxp, myp, grid.nz + 1)
        nz = grid.nz
        r = np.arange(2 * nz)
        w = np.where(r <= nz, r, r - 2 * nz) * grid.hz
        kap = green.kappa(mslot[:, None], nslot[None, :], geom.a, geom.b)
        tab = green.z_profile(w[None, None, :], kap[:, :, None], grid.hz, igf) / kap[:, :, None]
        live = (mslot[:, None] <= geom.modes_m) & (nslot[None, :] <= geom.modes_n)
        want = np.fft.fft(tab, axis=2).real[:, :, :nz + 1] / (2 * nz)
        want *= green.prefactor_G(geom) * grid.hx * grid.hy * grid.hz * live[:, :, None]
        assert rel(got, want) <= 1e-13


# ---------------------------------------------------------------------------
# the bench configuration and planes beyond the transform form's sizes
# ---------------------------------------------------------------------------

NODES_128 = [(64, 64, 512), (0, 0, 0), (127, 127, 1023), (5, 100, 300), (90, 30, 700), (63, 64, 511),
             (1, 126, 2), (127, 0, 1000), (64, 10, 256), (30, 90, 768), (100, 100, 100), (17, 71, 900),
             (120, 60, 40), (45, 45, 450), (80, 20, 620), (10, 10, 10)]


def test_bench_configuration_is_the_mode_form_and_matches_the_direct_sum():
    """128x128x1024 IGF FP32 (the bench's solve, default plan) and FP64 against
    the oracle's exact sum at 16 sampled nodes, and against each other."""
    from paper_1111_4971_gb300 import PipeSolver
    w = bunches.workload_throughput_128()
    geom, grid, rho = w["geom"], w["grid"], w["rho"][0]
    s32 = PipeSolver(geom, grid, igf=True, dtype=torch.float32)
    assert s32.plan["t_kind"] == 3
    s64 = PipeSolver(geom, grid, igf=True, dtype=torch.float64)
    p32 = host(s32.solve(dev(rho, torch.float32)))
    p64 = host(s64.solve(dev(rho, torch.float64)))
    want = pipe.direct_sum_at(rho, geom, grid, 1, NODES_128)
    scale = np.abs(p64).max()
    assert np.abs(np.array([p64[n] for n in NODES_128]) - want).max() <= 1e-12 * scale
    assert np.abs(np.array([p32[n] for n in NODES_128]) - want).max() <= 1e-5 * scale
    assert rel(p32, p64) <= F32_TOL


def test_256_planes_against_oracle():
    """256x256x32 (beyond the transform form): FP64 and FP32 against O3."""
    geom, grid = cell_centred(1.0, 1.0, 256, 256, 32, 0.1, modes=20)
    rho = gaussian_bunch(geom, grid, (0.5, 0.45, 1.6), (0.15, 0.1, 0.6))
    want = pipe.fft_solve(rho, geom, grid, 1)
    for dtype, tol in ((torch.float64, F64_TOL), (torch.float32, F32_TOL)):
        s = mode_solver(geom, grid, 1, dtype)
        assert rel(host(s.solve(dev(rho, dtype))), want) <= tol


def test_512_planes_at_sampled_nodes():
    """512x512x1024 (the accuracy study's reference grid) FP32 and FP64 at
    16 nodes against the oracle's exact sum."""
    geom, grid = cell_centred(1.0, 1.0, 512, 512, 1024, 24.0 / 1024, modes=20)
    rho = gaussian_bunch(geom, grid, (0.5, 0.5, 12.0), (0.15, 0.15, 3.0))
    nodes = [(4 * i + 1, 4 * j + 2, k) for (i, j, k) in NODES_128]
    want = pipe.direct_sum_at(rho, geom, grid, 1, nodes)
    for dtype, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
        s = mode_solver(geom, grid, 1, dtype)
        got = host(s.solve(dev(rho, dtype)))
        scale = np.abs(got).max()
        assert np.abs(np.array([got[n] for n in nodes]) - want).max() <= tol * scale
        del s, got
        torch.cuda.empty_cache()


def test_refusals():
    from paper_1111_4971_gb300 import PipeError, PipeSolver
    geom, grid = MESHES["cc48x32x64"]
    s = PipeSolver(geom, grid, igf=True, dtype=torch.float32)
    assert s.plan["t_kind"] == 3
    with pytest.raises(PipeError):
        s.set_plan(z_warps=8, z_pipe=0, t_h=1, t_threads=256, t_kind=1)
    spec = torch.empty((grid.nz + 1, grid.nx, grid.ny), dtype=torch.complex64, device="cuda")
    with pytest.raises(PipeError):
        s.stage_z_forward(dev(np.zeros(grid.shape), torch.float32), spec)
    # more modes than the form's tables hold: the transform form only
    g40, gr = cell_centred(1.0, 1.0, 32, 32, 32, 0.04, modes=40)
    s40 = PipeSolver(g40, gr, igf=True, dtype=torch.float32)
    assert s40.plan["t_kind"] != 3
    with pytest.raises(PipeError):
        s40.set_plan(t_kind=3)


@pytest.mark.parametrize("modes", [(1, 1), (1, 7), (32, 32), (5, 32)])
def test_mode_counts_at_the_limits(modes):
    """One mode, unequal counts, and the largest count the form takes
    (32 per axis; in FP64 the back-projection's mode columns must fit in
    shared memory, which 32 x 32 does not): solves and adjoints against O3."""
    from paper_1111_4971_gb300 import PipeError
    m, n = modes
    geom = Geometry(1.3, 1.0, 1.3 / 64, 1.0 / 64, m, n)
    grid = Grid(32, 32, 32, 1.3 / 32, 1.0 / 32, 0.05)
    rho = _density(geom, grid, 71 + m + n)
    for igf in (0, 1):
        want = pipe.fft_solve(rho, geom, grid, igf)
        for dtype, tol in ((torch.float64, F64_TOL), (torch.float32, F32_TOL)):
            if dtype == torch.float64 and m * n > 880:
                with pytest.raises(PipeError):
                    mode_solver(geom, grid, igf, dtype)
                continue
            s = mode_solver(geom, grid, igf, dtype)
            assert rel(host(s.solve(dev(rho, dtype))), want) <= tol, (modes, igf, dtype)
            assert rel(host(s.adjoint(dev(rho, dtype))), want) <= tol, (modes, igf, dtype)


def test_zero_density_and_point_charge():
    """Zero in, zero out (every stage is linear); a unit charge on one node
    against the oracle's exact sum at nodes near and far from it, on the
    bench's own launch shapes (128^2 cell-centred, the fast FP32 kernels)."""
    geom, grid = cell_centred(1.0, 1.0, 128, 128, 64, 0.02, modes=20)
    for dtype in (torch.float64, torch.float32):
        s = mode_solver(geom, grid, 1, dtype)
        phi = s.solve(torch.zeros(grid.shape, dtype=dtype, device="cuda"))
        assert torch.count_nonzero(phi).item() == 0
    rho = np.zeros(grid.shape)
    rho[40, 77, 31] = 1.0
    nodes = [(40, 77, 31), (41, 77, 31), (40, 77, 33), (10, 100, 5), (127, 0, 63), (64, 64, 32)]
    want = pipe.direct_sum_at(rho, geom, grid, 1, nodes)
    for dtype, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
        got = host(mode_solver(geom, grid, 1, dtype).solve(dev(rho, dtype)))
        scale = np.abs(got).max()
        assert np.abs(np.array([got[n] for n in nodes]) - want).max() <= tol * scale, dtype
