"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances (relative L2 over the physical block): FP64 path <= 1e-12, FP32 path
<= 1e-5 -- the two accuracy targets of the solver.
"""
import numpy as np
import pytest
import torch

from inputs import bunches
from inputs.bunches import Geometry, Grid, cell_centred, random_density
from oracle import pipe

pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
F32_TOL = 1e-5


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    a = a.astype(np.complex128 if np.iscomplexobj(a) else np.float64)
    b = b.astype(np.complex128 if np.iscomplexobj(b) else np.float64)
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


def solver(geom, grid, igf, dtype=torch.float64):
    from paper_1111_4971_gb300 import PipeSolver
    return PipeSolver(geom, grid, igf=igf, dtype=dtype)


GEOMS = {
    "cc16x16x32": cell_centred(2.0, 2.0, 16, 16, 32, 0.1, modes=20),
    "rect32x32x64": cell_centred(2.0, 1.0, 32, 32, 64, 0.0625, modes=20),
    "wall16x16x64": (Geometry(1.0, 0.5, 0.0, 0.0, 12, 9), Grid(16, 16, 64, 1 / 16, 0.5 / 16, 0.05)),
    "aliased32x32x32": cell_centred(1.0, 1.0, 32, 32, 32, 0.04, modes=40),
}


# ---------------------------------------------------------------------------
# setup: Green spectrum (tabulation + transforms, FP64)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("igf", [0, 1])
@pytest.mark.parametrize("key", list(GEOMS))
def test_green_spectrum(key, igf):
    geom, grid = GEOMS[key]
    s = solver(geom, grid, igf)
    got = s.green_spectrum()                                   # [kz][ky][kx]
    want = pipe.green_spectrum_octant(geom, grid, igf)         # [kx][ky][kz]
    assert np.abs(want.imag).max() <= 1e-12 * np.abs(want.real).max()
    want = want.real.transpose(2, 1, 0)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


def test_free_space_spectrum():
    from paper_1111_4971_gb300 import PipeSolver
    grid = Grid(32, 32, 64, 0.1, 0.12, 0.07)
    s = PipeSolver(None, grid, dtype=torch.float64, free_space=True)
    got = s.green_spectrum()
    want = pipe.hockney_spectrum_octant(grid).real.transpose(2, 1, 0)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


# ---------------------------------------------------------------------------
# single stages against numpy transforms
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-13), (torch.float32, 2e-6)])
@pytest.mark.parametrize("nz", [32, 64, 256, 1024])
def test_stage_z_forward(nz, dtype, tol):
    geom, grid = cell_centred(1.0, 1.0, 16, 16, nz, 0.1, modes=4)
    s = solver(geom, grid, 1, dtype)
    rho = random_density(grid.shape, nz)
    spec = s.spectrum_buffer()
    for adj in (0, 1):
        s.stage_z_forward(dev(rho, dtype), spec, adjoint=adj)
        got = spec.cpu().numpy()
        padded = np.concatenate([rho, np.zeros_like(rho)], axis=2)
        want = np.fft.rfft(padded, axis=2).transpose(2, 0, 1)
        if adj:
            want = np.conj(want)
        assert rel(got, want) < tol


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-13), (torch.float32, 2e-6)])
@pytest.mark.parametrize("nz", [32, 128, 512, 1024])
def test_stage_z_inverse(nz, dtype, tol):
    geom, grid = cell_centred(1.0, 1.0, 16, 16, nz, 0.1, modes=4)
    s = solver(geom, grid, 1, dtype)
    full = random_density((16, 16, 2 * nz), 7 + nz)
    spec_np = np.fft.rfft(full, axis=2).transpose(2, 0, 1)
    for adj in (0, 1):
        inp = np.conj(spec_np) if adj else spec_np
        cdt = torch.complex128 if dtype == torch.float64 else torch.complex64
        spec = torch.tensor(np.ascontiguousarray(inp), dtype=cdt, device="cuda")
        phi = s.empty()
        s.stage_z_inverse(spec, phi, adjoint=adj)
        want = full[:, :, :nz] * (2 * nz)
        assert rel(host(phi), want) < tol


def _z_fits(nz, warps, cbytes, pipe):
    """Shared memory of the z kernels within the 227 KB a CTA can have:
    single-tile, the FFT scratch or the staging tile (they share it);
    pipelined, two input or staging tiles plus the FFT scratch."""
    L = nz // 2
    g = 4 if L <= 32 else 8 if L <= 128 else 16 if L <= 512 else 32
    e = L // g
    cols = warps * (32 // (2 * g))
    scr = (32 * warps // g) * (e * (g + 1) + 8)
    stg = cols * (nz + (2 if cbytes == 8 else 1))
    inw = cols * (nz // 2)
    need = max(2 * inw + scr + stg, 2 * stg + scr) if pipe else max(scr, stg)
    return cbytes * need <= 227 * 1024


@pytest.mark.parametrize("zw,zp", [(4, 0), (4, 1), (8, 0), (16, 0), (16, 1), (8, 1)])
@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-13), (torch.float32, 2e-6)])
@pytest.mark.parametrize("nz", [512, 1024])
def test_stage_z_cta_sizes(nz, dtype, tol, zw, zp):
    """Every z CTA size (4, 8, 16 warps) and both tile schedules, forward and
    inverse, against numpy's real FFTs."""
    if not _z_fits(nz, zw, 16 if dtype == torch.float64 else 8, zp):
        pytest.skip("this CTA size does not fit in shared memory at this size")
    geom, grid = cell_centred(1.0, 1.0, 16, 16, nz, 0.1, modes=4)
    s = solver(geom, grid, 1, dtype)
    p = s.plan
    s.set_plan(z_warps=zw, z_pipe=zp, t_h=p["t_h"], t_threads=p["t_threads"], t_kind=p["t_kind"])
    rho = random_density(grid.shape, nz + zw)
    padded = np.concatenate([rho, np.zeros_like(rho)], axis=2)
    spec_np = np.fft.rfft(padded, axis=2).transpose(2, 0, 1)
    cdt = torch.complex128 if dtype == torch.float64 else torch.complex64
    for adj in (0, 1):
        spec = s.spectrum_buffer()
        s.stage_z_forward(dev(rho, dtype), spec, adjoint=adj)
        want = np.conj(spec_np) if adj else spec_np
        assert rel(spec.cpu().numpy(), want) < tol
        phi = s.empty()
        s.stage_z_inverse(torch.tensor(np.ascontiguousarray(want), dtype=cdt, device="cuda"), phi, adjoint=adj)
        assert rel(host(phi), rho * (2 * nz)) < tol


def _transverse_reference(P, geom, grid, igf, adjoint):
    """Per kz plane: padded 2-D DFT, the four-term product with the oracle's
    transformed tables (each F^fff of its own table), unnormalised inverse, crop."""
    nx, ny, nz = grid.shape
    T = pipe.green_tables(geom, grid, igf)
    F = {k: np.fft.fftn(v) for k, v in T.items()}
    scale = pipe.h3(grid) / (8.0 * nx * ny * nz)
    out = np.empty_like(P)

    def refl(a, axis):
        return np.roll(np.flip(a, axis), 1, axis)

    for kz in range(nz + 1):
        pad = np.zeros((2 * nx, 2 * ny), dtype=np.complex128)
        pad[:nx, :ny] = P[kz]
        if not adjoint:
            S = np.fft.fft2(pad)
            tc = {k: F[k][:, :, kz] for k in F}
            Phi = (tc["cc"] * S - tc["cr"] * refl(S, 1) - tc["rc"] * refl(S, 0)
                   + tc["rr"] * refl(refl(S, 0), 1))
            o = np.fft.ifft2(Phi) * (4 * nx * ny)
        else:
            S = np.fft.ifft2(pad) * (4 * nx * ny)
            tc = {k: F[k][:, :, kz] for k in F}
            # transpose of the product: T_t(R_t k) S(R_t k)
            Phi = (tc["cc"] * S - refl(tc["cr"] * S, 1) - refl(tc["rc"] * S, 0)
                   + refl(refl(tc["rr"] * S, 0), 1))
            o = np.fft.fft2(Phi)
        out[kz] = scale * o[:nx, :ny]
    return out


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 5e-6)])
@pytest.mark.parametrize("key", ["cc16x16x32", "rect32x32x64", "wall16x16x64"])
def test_stage_transverse(key, dtype, tol):
    geom, grid = GEOMS[key]
    s = solver(geom, grid, 1, dtype)
    rng = np.random.default_rng(3)
    P = rng.standard_normal((grid.nz + 1, grid.nx, grid.ny)) \
        + 1j * rng.standard_normal((grid.nz + 1, grid.nx, grid.ny))
    cdt = torch.complex128 if dtype == torch.float64 else torch.complex64
    for adj in (0, 1):
        spec = torch.tensor(P, dtype=cdt, device="cuda")
        s.stage_transverse(spec, adjoint=adj)
        want = _transverse_reference(P, geom, grid, 1, adj)
        assert rel(spec.cpu().numpy(), want) < tol


# ---------------------------------------------------------------------------
# full solves against the oracle
# ---------------------------------------------------------------------------

def test_fp64_ordinary_16_against_brute_force():
    w = bunches.workload_fp64_ordinary_16()
    geom, grid, rho = w["geom"], w["grid"], w["rho"][0]
    want = pipe.direct_sum(rho, geom, grid, 0)
    s64 = solver(geom, grid, 0, torch.float64)
    assert rel(host(s64.solve(dev(rho, torch.float64))), want) <= F64_TOL
    s32 = solver(geom, grid, 0, torch.float32)
    assert rel(host(s32.solve(dev(rho, torch.float32))), want) <= F32_TOL


@pytest.mark.parametrize("igf", [0, 1])
@pytest.mark.parametrize("key", list(GEOMS))
def test_random_density_against_fft_oracle(key, igf):
    geom, grid = GEOMS[key]
    rho = random_density(grid.shape, 100 + igf, sparsity=0.2)
    spectra = pipe.green_spectra(geom, grid, igf)
    want = pipe.fft_solve(rho, geom, grid, igf, spectra=spectra)
    for dtype, tol in ((torch.float64, F64_TOL), (torch.float32, F32_TOL)):
        s = solver(geom, grid, igf, dtype)
        got = host(s.solve(dev(rho, dtype)))
        assert rel(got, want) <= tol, (dtype, rel(got, want))
        adj = host(s.adjoint(dev(rho, dtype)))
        want_adj = pipe.fft_adjoint(rho, geom, grid, igf, spectra=spectra)
        assert rel(adj, want_adj) <= tol


@pytest.mark.parametrize("shape", [(64, 64, 128), (128, 128, 32), (32, 32, 1024)])
def test_sizes_spanning_tiles(shape):
    nx, ny, nz = shape
    geom, grid = cell_centred(1.5, 1.0, nx, ny, nz, 0.05, modes=20)
    rho = random_density(grid.shape, nx + nz, sparsity=0.5)
    want = pipe.fft_solve(rho, geom, grid, 1)
    for dtype, tol in ((torch.float64, F64_TOL), (torch.float32, F32_TOL)):
        got = host(solver(geom, grid, 1, dtype).solve(dev(rho, dtype)))
        assert rel(got, want) <= tol, (dtype, rel(got, want))


def test_hockney_against_oracle():
    from paper_1111_4971_gb300 import PipeSolver
    grid = Grid(32, 32, 64, 0.1, 0.1, 0.05)
    rho = random_density(grid.shape, 5)
    want = pipe.hockney_fft(rho, grid)
    for dtype, tol in ((torch.float64, F64_TOL), (torch.float32, F32_TOL)):
        s = PipeSolver(None, grid, dtype=dtype, free_space=True)
        assert rel(host(s.solve(dev(rho, dtype))), want) <= tol


def test_igf_64_three_bunches():
    w = bunches.workload_igf_64()
    geom, grid = w["geom"], w["grid"]
    spectra = pipe.green_spectra(geom, grid, 1)
    s64 = solver(geom, grid, 1, torch.float64)
    s32 = solver(geom, grid, 1, torch.float32)
    for rho in w["rho"]:
        want = pipe.fft_solve(rho, geom, grid, 1, spectra=spectra)
        p64 = host(s64.solve(dev(rho, torch.float64)))
        p32 = host(s32.solve(dev(rho, torch.float32)))
        assert rel(p64, want) <= F64_TOL
        assert rel(p32, p64) <= F32_TOL
        assert rel(p32, want) <= F32_TOL


def test_adjoint_symmetry_and_inplace():
    geom, grid = GEOMS["rect32x32x64"]
    r1 = random_density(grid.shape, 1)
    r2 = random_density(grid.shape, 2)
    for dtype, tol in ((torch.float64, 1e-13), (torch.float32, 1e-6)):
        s = solver(geom, grid, 1, dtype)
        a1 = host(s.solve(dev(r1, dtype)))
        t2 = host(s.adjoint(dev(r2, dtype)))
        lhs, rhs = np.sum(a1 * r2), np.sum(r1 * t2)
        assert abs(lhs - rhs) <= tol * abs(lhs)
        assert rel(host(s.adjoint(dev(r1, dtype))), a1) <= 10 * tol
        x = dev(r1, dtype)
        s.solve(x, out=x)                                       # phi aliases rho
        assert rel(host(x), a1) <= 10 * tol


def test_solve_host_matches_device():
    geom, grid = GEOMS["rect32x32x64"]
    rho = random_density(grid.shape, 9)
    for dtype in (torch.float32, torch.float64):
        s = solver(geom, grid, 1, dtype)
        d = host(s.solve(dev(rho, dtype)))
        hin = torch.tensor(rho, dtype=dtype).pin_memory()
        hout = s.solve_host(hin)
        assert np.array_equal(hout.double().numpy(), d)


def test_solve_host_stream_matches_device_solves():
    """The overlapped host sequence gives every solve bitwise as a device solve,
    for more solves than staging buffers (the ring is reused)."""
    geom, grid = GEOMS["rect32x32x64"]
    for dtype in (torch.float32, torch.float64):
        s = solver(geom, grid, 1, dtype)
        rhos = [random_density(grid.shape, 60 + k) for k in range(5)]
        want = [host(s.solve(dev(r, dtype))) for r in rhos]
        ins = [torch.tensor(r, dtype=dtype).pin_memory() for r in rhos]
        outs = s.solve_host_stream(ins)
        for o, w in zip(outs, want):
            assert np.array_equal(o.double().numpy(), w)


def test_full_size_128x128x1024_sampled_against_direct_sum():
    w = bunches.workload_throughput_128()
    geom, grid, rho = w["geom"], w["grid"], w["rho"][0]
    s64 = solver(geom, grid, 1, torch.float64)
    s32 = solver(geom, grid, 1, torch.float32)
    p64 = host(s64.solve(dev(rho, torch.float64)))
    p32 = host(s32.solve(dev(rho, torch.float32)))
    assert rel(p32, p64) <= F32_TOL
    rng = np.random.default_rng(0)
    nodes = [(64, 64, 512), (0, 0, 0), (127, 127, 1023), (5, 100, 300)] + \
        [tuple(int(rng.integers(0, s)) for s in grid.shape) for _ in range(12)]
    want = pipe.direct_sum_at(rho, geom, grid, 1, nodes)
    got = np.array([p64[n] for n in nodes])
    scale = np.abs(p64).max()
    assert np.abs(got - want).max() <= 1e-12 * scale
    # the FP32 path in the launch configurations the bench times at the same
    # nodes: the default (the mode-space form at this size) and the padded
    # transforms (staged transverse kernel, 4-warp z CTAs)
    assert s32.plan["t_kind"] == 3
    got32 = np.array([p32[n] for n in nodes])
    assert np.abs(got32 - want).max() <= F32_TOL * scale
    s32.set_plan(z_warps=4, z_pipe=0, t_h=1, t_threads=256, t_kind=2)
    p32t = host(s32.solve(dev(rho, torch.float32)))
    assert rel(p32t, p64) <= F32_TOL
    got32t = np.array([p32t[n] for n in nodes])
    assert np.abs(got32t - want).max() <= F32_TOL * scale
