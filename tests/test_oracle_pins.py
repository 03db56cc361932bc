"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test would fail under a plausible mistake in the oracle (a dropped term,
a wrong sign, index or direction, a transposed operand, a wrong prefactor).
CPU only.
"""
import os

import numpy as np
import pytest

from inputs import bunches
from inputs.bunches import Geometry, Grid, cell_centred, random_density
from oracle import conv1d, green, pipe

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


# ---------------------------------------------------------------------------
# P1: the three solvers agree (Appendix A proof: exact in the physical block)
# ---------------------------------------------------------------------------

CASES = [
    # name, geometry, grid
    ("cell_centred", *cell_centred(2.0, 1.5, 4, 6, 8, 0.2, modes=7)),
    ("node_on_wall", Geometry(1.0, 1.0, 0.0, 0.0, 9, 9), Grid(4, 4, 6, 0.25, 0.25, 0.3)),
    ("window", Geometry(3.0, 2.0, 0.37, 0.21, 6, 5), Grid(5, 4, 6, 0.3, 0.25, 0.15)),
    ("aliased_modes", *cell_centred(1.0, 1.0, 4, 4, 4, 0.25, modes=11)),
]


@pytest.mark.parametrize("igf", [0, 1])
@pytest.mark.parametrize("name,geom,grid", CASES, ids=[c[0] for c in CASES])
def test_three_solvers_agree(name, geom, grid, igf):
    rho = random_density(grid.shape, 11, sparsity=0.3)
    p1 = pipe.direct_sum(rho, geom, grid, igf)
    p2 = pipe.naive_dft_solve(rho, geom, grid, igf)
    p3 = pipe.fft_solve(rho, geom, grid, igf)
    assert rel(p2, p1) < 1e-12
    assert rel(p3, p1) < 1e-12


def test_three_solvers_agree_16x16x32():
    w = bunches.workload_fp64_ordinary_16()
    rho = w["rho"][0]
    p1 = pipe.direct_sum(rho, w["geom"], w["grid"], 0)
    p3 = pipe.fft_solve(rho, w["geom"], w["grid"], 0)
    p2 = pipe.naive_dft_solve(rho, w["geom"], w["grid"], 0)
    assert rel(p3, p1) < 1e-12 and rel(p2, p1) < 1e-12


def test_sampled_direct_sum_matches_full_sum():
    geom, grid = cell_centred(2.0, 1.0, 6, 5, 7, 0.3, modes=8)
    rho = random_density(grid.shape, 5)
    for igf in (0, 1):
        full = pipe.direct_sum(rho, geom, grid, igf)
        nodes = [(0, 0, 0), (5, 4, 6), (2, 3, 1), (3, 0, 6)]
        got = pipe.direct_sum_at(rho, geom, grid, igf, nodes)
        want = np.array([full[n] for n in nodes])
        assert np.allclose(got, want, rtol=1e-12, atol=1e-14 * np.abs(full).max())


# ---------------------------------------------------------------------------
# Appendix A: 1-D convolution / correlation by FFT with direction control
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("J,K,extra", [(5, 3, 0), (4, 6, 2), (7, 7, 1), (1, 4, 0)])
def test_appendix_conv_and_corr(J, K, extra):
    rng = np.random.default_rng(J * 100 + K)
    r = rng.standard_normal(K)
    x = {m: rng.standard_normal() for m in range(-(K - 1), J + K)}
    N = J + K - 1 + extra
    assert np.allclose(conv1d.fft_convolution(r, x, J, N), conv1d.brute_convolution(r, x, J),
                       atol=1e-12)
    assert np.allclose(conv1d.fft_correlation(r, x, J, N), conv1d.brute_correlation(r, x, J),
                       atol=1e-12)
    # the *un*swapped directions give the convolution, not the correlation
    if K > 1:
        assert not np.allclose(conv1d.fft_convolution(r, x, J, N),
                               conv1d.brute_correlation(r, x, J), atol=1e-6)


def test_fig1_storage_layout():
    spec = {}
    offs = {}
    with open(os.path.join(GOLDEN, "fig1_layout.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            if parts[0] == "green_offset":
                offs[int(parts[1])] = int(parts[2])
            else:
                spec[parts[0]] = [int(v) for v in parts[1:]]
    n = spec["n_physical"][0]
    grid = Grid(1, 1, n, 1.0, 1.0, 1.0)
    o = pipe.conv_offsets(n, 1.0)
    assert len(o) == spec["n_stored"][0]
    for idx, off in offs.items():
        assert o[idx] == off
    padded = pipe.pad(np.ones((1, 1, n)), grid)[0, 0]
    lo, hi = spec["rho_physical_indices"]
    assert np.all(padded[lo:hi + 1] == 1.0)
    lo, hi = spec["rho_zero_indices"]
    assert np.all(padded[lo:hi + 1] == 0.0)
    assert abs(o[spec["green_unused"][0]]) == n


# ---------------------------------------------------------------------------
# P2: Eq. 7 (sine series) == Eq. 8-9 (four R terms) for any truncation
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("igf", [0, 1])
def test_sine_series_equals_four_R(igf):
    geom = Geometry(1.7, 0.9, 0.0, 0.0, 13, 9)
    rng = np.random.default_rng(3)
    n = 64
    x, xp = rng.uniform(0, geom.a, (2, n))
    y, yp = rng.uniform(0, geom.b, (2, n))
    hz = 0.05
    w = hz * rng.integers(-20, 20, n)
    g1 = green.green_sine(x, xp, y, yp, w, geom, igf, hz)
    g2 = green.green_four_R(x, xp, y, yp, w, geom, igf, hz)
    assert np.max(np.abs(g1 - g2)) <= 1e-13 * np.max(np.abs(g1))


# ---------------------------------------------------------------------------
# P3: Dirichlet walls
# ---------------------------------------------------------------------------

def test_green_vanishes_on_walls():
    geom = Geometry(2.0, 1.0, 0.0, 0.0, 20, 20)
    rng = np.random.default_rng(4)
    xp, yp = rng.uniform(0.1, 0.9, (2, 16)) * np.array([[2.0], [1.0]])
    w = rng.uniform(-1, 1, 16)
    for wall in [(0.0, None), (2.0, None), (None, 0.0), (None, 1.0)]:
        x = np.full(16, wall[0]) if wall[0] is not None else rng.uniform(0, 2, 16)
        y = np.full(16, wall[1]) if wall[1] is not None else rng.uniform(0, 1, 16)
        g = green.green_four_R(x, xp, y, yp, w, geom, 0, 0.1)
        assert np.max(np.abs(g)) < 1e-13


@pytest.mark.parametrize("igf", [0, 1])
def test_potential_vanishes_on_wall_nodes(igf):
    # node row i = 0 sits on the wall x = 0 (x0 = 0), j = 0 on y = 0
    geom = Geometry(1.0, 0.8, 0.0, 0.0, 12, 12)
    grid = Grid(8, 8, 8, 1.0 / 8, 0.8 / 8, 0.1)
    rho = np.abs(random_density(grid.shape, 9))
    phi = pipe.fft_solve(rho, geom, grid, igf)
    scale = np.abs(phi).max()
    assert np.abs(phi[0]).max() < 1e-13 * scale
    assert np.abs(phi[:, 0]).max() < 1e-13 * scale


# ---------------------------------------------------------------------------
# P4: symmetries and operator symmetry
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("igf", [0, 1])
def test_symmetries(igf):
    geom, grid = cell_centred(1.0, 1.0, 6, 6, 8, 0.15, modes=9)
    rho = random_density(grid.shape, 21)
    phi = pipe.fft_solve(rho, geom, grid, igf)
    s = np.abs(phi).max()
    # x <-> y (a = b, nx = ny)
    phiT = pipe.fft_solve(rho.transpose(1, 0, 2), geom, grid, igf)
    assert np.abs(phiT - phi.transpose(1, 0, 2)).max() < 1e-13 * s
    # x -> a - x (cell-centred: i -> nx-1-i), y -> b - y, z -> -z
    for ax in range(3):
        phir = pipe.fft_solve(np.flip(rho, ax), geom, grid, igf)
        assert np.abs(phir - np.flip(phi, ax)).max() < 1e-13 * s
    # a non-symmetric transverse geometry still has A = A^T
    g2 = Geometry(2.3, 1.1, 0.31, 0.17, 8, 7)
    gr2 = Grid(5, 6, 7, 0.33, 0.15, 0.2)
    r1, r2 = random_density(gr2.shape, 1), random_density(gr2.shape, 2)
    lhs = np.sum(pipe.fft_solve(r1, g2, gr2, igf) * r2)
    rhs = np.sum(r1 * pipe.fft_solve(r2, g2, gr2, igf))
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)
    # the literal transposed operator equals the forward one, and the brute-force transpose
    a_fft = pipe.fft_adjoint(r1, g2, gr2, igf)
    a_bf = pipe.direct_sum_adjoint(r1, g2, gr2, igf)
    a_nv = pipe.fft_adjoint(r1, g2, gr2, igf, naive=True)
    assert rel(a_fft, a_bf) < 1e-12 and rel(a_nv, a_bf) < 1e-12
    assert rel(pipe.fft_solve(r1, g2, gr2, igf), a_bf) < 1e-12


# ---------------------------------------------------------------------------
# P5: closed-form Green spectrum (node on the wall, mesh spans the pipe, M < N)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("igf", [0, 1])
def test_closed_form_green_spectrum(igf):
    nx, ny, nz = 8, 6, 5
    a, b = 1.3, 0.7
    geom = Geometry(a, b, 0.0, 0.0, 5, 4)
    grid = Grid(nx, ny, nz, a / nx, b / ny, 0.11)
    S = pipe.green_spectra(geom, grid, igf)["cc"]
    want = np.zeros_like(S)
    oz = pipe.conv_offsets(nz, grid.hz)
    r = np.arange(2 * nz)
    C = 2 * np.pi / (a * b)
    for m in range(1, geom.modes_m + 1):
        for n in range(1, geom.modes_n + 1):
            k = green.kappa(m, n, a, b)
            zp = green.z_profile(oz, k, grid.hz, igf)
            zhat = np.array([np.sum(zp * np.exp(-2j * np.pi * r * kz / (2 * nz)))
                             for kz in range(2 * nz)])
            for kx in (m, 2 * nx - m):
                for ky in (n, 2 * ny - n):
                    want[kx, ky, :] += C * nx * ny / k * zhat
    assert np.abs(S - want).max() < 1e-12 * np.abs(want).max()


def test_single_table_and_phase_identity():
    # Sec. 2: "only a single function R needs to be tabulated".  Exactly true for
    # x0 = 0 meshes spanning the pipe; for cell-centred meshes the correlation
    # tables are the convolution table shifted by one sample (a phase in k).
    for x0f, shift in [(0.0, 0), (0.5, 1)]:
        nx, ny, nz = 6, 4, 4
        geom = Geometry(1.0, 0.5, x0f / nx, x0f * 0.5 / ny, 7, 5)
        grid = Grid(nx, ny, nz, 1.0 / nx, 0.5 / ny, 0.2)
        T = pipe.green_tables(geom, grid, 1)
        F = {k: pipe.transform(v, "fff") for k, v in T.items()}
        kx = np.arange(2 * nx)[:, None, None]
        ky = np.arange(2 * ny)[None, :, None]
        ex = np.exp(1j * np.pi * shift * kx / nx)
        ey = np.exp(1j * np.pi * shift * ky / ny)
        s = np.abs(F["cc"]).max()
        assert np.abs(F["cc"].imag).max() < 1e-12 * s
        assert np.abs(F["rc"] - ex * F["cc"]).max() < 1e-12 * s
        assert np.abs(F["cr"] - ey * F["cc"]).max() < 1e-12 * s
        assert np.abs(F["rr"] - ex * ey * F["cc"]).max() < 1e-12 * s


# ---------------------------------------------------------------------------
# P6: integrated Green function
# ---------------------------------------------------------------------------

def test_igf_normalisation_and_limits():
    for kap in (0.3, 2.0, 17.0):
        for hz in (0.01, 0.1, 0.7):
            R = int(60.0 / (kap * hz)) + 2
            r = np.arange(-R, R + 1)
            s = hz * np.sum(green.gz_stable(r * hz, kap, hz))
            assert abs(s - 2.0 / kap) < 1e-12 * (2.0 / kap)
    # kappa h -> 0: g_z(w) -> e^{-kappa |w|} at fixed w
    kap, w = 3.0, 0.4
    errs = []
    for hz in (0.1, 0.05, 0.025, 0.0125):
        errs.append(abs(green.gz_stable(w, kap, hz) - np.exp(-kap * w)))
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:]))
    assert errs[-1] < 1e-3 * np.exp(-kap * w)


def test_igf_stable_matches_literal_and_high_precision():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    for kap, hz in [(1.0, 1.0), (5.0, 0.3), (2.0, 1e-2), (3.0, 1e-5)]:
        for r in (0, 1, 2, 7):
            w = r * hz
            K, H, W = mpmath.mpf(kap), mpmath.mpf(hz), mpmath.mpf(w)
            lit = (2 * H * K * (1 if r == 0 else 0) + mpmath.e ** (-K * abs(W + H))
                   - 2 * mpmath.e ** (-K * abs(W)) + mpmath.e ** (-K * abs(W - H))) / (H * K) ** 2
            st = green.gz_stable(w, kap, hz)
            assert abs(st - float(lit)) <= 1e-14 * abs(float(lit))
            if kap * hz >= 0.3:
                assert abs(green.gz_literal(w, kap, hz) - float(lit)) <= 1e-13 * abs(float(lit))


# ---------------------------------------------------------------------------
# Closed form: a single transverse mode (fixes the prefactor and the sums)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("igf", [0, 1])
def test_single_mode_closed_form(igf):
    geom, grid = cell_centred(1.6, 0.9, 8, 6, 10, 0.13, modes=5)
    x, y, z = pipe.mesh(geom, grid)
    f = np.exp(-((z - z.mean()) / 0.3) ** 2)
    rho = (np.sin(np.pi * x / geom.a)[:, None, None] * np.sin(np.pi * y / geom.b)[None, :, None]
           * f[None, None, :])
    phi = pipe.fft_solve(rho, geom, grid, igf)
    k11 = green.kappa(1, 1, geom.a, geom.b)
    zz = green.z_profile(z[:, None] - z[None, :], k11, grid.hz, igf)
    want = (2 * np.pi / k11 * np.sin(np.pi * x / geom.a)[:, None, None]
            * np.sin(np.pi * y / geom.b)[None, :, None] * (grid.hz * zz @ f)[None, None, :])
    assert rel(phi, want) < 1e-12


# ---------------------------------------------------------------------------
# P7: free-space limit as the pipe widens
# ---------------------------------------------------------------------------

def test_green_tends_to_free_space():
    errs = []
    for a in (2.0, 4.0, 8.0, 16.0):
        geom = Geometry(a, a, 0.0, 0.0, int(12 * a), int(12 * a))
        d = 0.3
        g = green.green_sine(a / 2, a / 2 + d * 0.6, a / 2, a / 2 - d * 0.8, 0.0, geom) * d
        errs.append(abs(g - 1.0))
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:]))
    assert errs[-1] < 0.05


def test_solve_tends_to_hockney():
    grid = Grid(4, 4, 6, 0.1, 0.1, 0.1)
    rho = np.zeros(grid.shape)
    rng = np.random.default_rng(8)
    rho[:, :, 2:4] = rng.uniform(0.5, 1.0, (4, 4, 2))
    free = pipe.hockney_fft(rho, grid)
    keep = [0, 5]        # z-planes at least one cell from the charge
    errs = []
    for a in (0.8, 1.6, 3.2):
        geom = bunches.windowed(Geometry(1, 1, 0, 0), grid, a, a, modes=int(20 * a))
        phi = pipe.fft_solve(rho, geom, grid, 0)
        errs.append(rel(phi[:, :, keep], free[:, :, keep]))
    # the walls' image charges contribute O(1/a): the error halves per doubling
    for e1, e2 in zip(errs, errs[1:]):
        assert 0.45 < e2 / e1 < 0.55


def test_hockney_fft_equals_direct():
    grid = Grid(4, 3, 5, 0.2, 0.3, 0.25)
    rho = random_density(grid.shape, 4)
    assert rel(pipe.hockney_fft(rho, grid), pipe.hockney_direct(rho, grid)) < 1e-12


# ---------------------------------------------------------------------------
# P8: point charge gives back the Green function
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("igf", [0, 1])
def test_point_charge(igf):
    geom, grid = cell_centred(1.0, 2.0, 6, 8, 8, 0.2, modes=10)
    i0, j0, k0 = 2, 5, 3
    rho = np.zeros(grid.shape)
    rho[i0, j0, k0] = 1.0 / pipe.h3(grid)
    phi = pipe.fft_solve(rho, geom, grid, igf)
    x, y, z = pipe.mesh(geom, grid)
    want = green.green_sine(x[:, None, None], x[i0], y[None, :, None], y[j0],
                            (z - z[k0])[None, None, :], geom, igf, grid.hz)
    assert rel(phi, want) < 1e-12


# ---------------------------------------------------------------------------
# P10: gradient of the field energy (FD in FP64)
# ---------------------------------------------------------------------------

def test_energy_gradient_fd():
    geom, grid = cell_centred(1.0, 1.0, 4, 4, 6, 0.2, modes=6)
    rho = random_density(grid.shape, 12)
    phi = pipe.fft_solve(rho, geom, grid, 1)
    grad = 0.5 * (phi + pipe.fft_adjoint(rho, geom, grid, 1))
    rng = np.random.default_rng(0)
    for _ in range(5):
        idx = tuple(int(rng.integers(0, s)) for s in grid.shape)
        e = np.zeros(grid.shape)
        e[idx] = 1e-3
        wp = pipe.field_energy(rho + e, pipe.fft_solve(rho + e, geom, grid, 1), grid)
        wm = pipe.field_energy(rho - e, pipe.fft_solve(rho - e, geom, grid, 1), grid)
        fd = (wp - wm) / 2e-3
        assert abs(fd - grad[idx]) < 1e-9 * max(1.0, abs(fd))
        assert abs(grad[idx] - phi[idx]) < 1e-12 * max(1.0, abs(phi[idx]))


# ---------------------------------------------------------------------------
# Banded reduction (Sec. 5, Eq. 17-18): two independent evaluations agree, and
# the band covering every plane is the full solve
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n_nb", [0, 1, 3])
@pytest.mark.parametrize("igf", [0, 1])
@pytest.mark.parametrize("name,geom,grid", CASES, ids=[c[0] for c in CASES])
def test_banded_solvers_agree(name, geom, grid, igf, n_nb):
    rho = random_density(grid.shape, 13, sparsity=0.3)
    p1 = pipe.direct_sum_banded(rho, geom, grid, igf, n_nb)
    p2 = pipe.banded_solve(rho, geom, grid, igf, n_nb)
    assert rel(p2, p1) < 1e-12


@pytest.mark.parametrize("igf", [0, 1])
def test_full_band_is_the_full_solve(igf):
    geom, grid = cell_centred(2.0, 1.5, 4, 6, 8, 0.2, modes=7)
    rho = random_density(grid.shape, 17)
    full = pipe.fft_solve(rho, geom, grid, igf)
    assert rel(pipe.banded_solve(rho, geom, grid, igf, grid.nz - 1), full) < 1e-12
    assert rel(pipe.direct_sum_banded(rho, geom, grid, igf, grid.nz - 1), full) < 1e-12
    # a narrower band drops the terms beyond it: the difference is exactly
    # the contribution of the source planes outside the band
    part = pipe.banded_solve(rho, geom, grid, igf, 2)
    k = 5
    near = np.zeros_like(rho)
    near[:, :, k - 2:k + 3] = rho[:, :, k - 2:k + 3]
    assert rel(part[:, :, k], pipe.fft_solve(near, geom, grid, igf)[:, :, k]) < 1e-12
    assert rel(part, full) > 1e-6


def test_banded_long_bunch_close_to_full():
    """Sec. 5: for a bunch much longer than the pipe on a coarse z mesh
    (hz = 15 a) the IGF falls off so fast that the 2-D reduction (Eq. 17)
    is within a few percent of the full solve, and one neighbour on each side
    (Eq. 18) leaves out only terms below e^{-kappa hz} ~ 1e-29."""
    geom, grid, rho = bunches.accuracy_study_case(30.0, 8, 16, modes=6)
    full = pipe.fft_solve(rho, geom, grid, 1)
    e0 = rel(pipe.banded_solve(rho, geom, grid, 1, 0), full)
    e1 = rel(pipe.banded_solve(rho, geom, grid, 1, 1), full)
    assert 1e-3 < e0 < 0.03
    assert e1 < 1e-13


# ---------------------------------------------------------------------------
# Field output E = -grad phi: exact for quadratics, second order otherwise
# ---------------------------------------------------------------------------

def test_electric_field_exact_on_quadratics_and_second_order():
    grid = Grid(7, 6, 9, 0.3, 0.2, 0.45)
    x = np.arange(grid.nx)[:, None, None] * grid.hx
    y = np.arange(grid.ny)[None, :, None] * grid.hy
    z = np.arange(grid.nz)[None, None, :] * grid.hz
    phi = 1.5 * x * x - 0.7 * x * y + 2.0 * z * z - 0.3 * y * z + x - 4.0 * y + 0.25
    E = pipe.electric_field(phi, grid)
    shape = phi.shape
    assert np.allclose(E[0], np.broadcast_to(-(3.0 * x - 0.7 * y + 1.0), shape), atol=1e-12)
    assert np.allclose(E[1], np.broadcast_to(-(-0.7 * x - 0.3 * z - 4.0), shape), atol=1e-12)
    assert np.allclose(E[2], np.broadcast_to(-(4.0 * z - 0.3 * y), shape), atol=1e-12)
    # a smooth non-polynomial potential: the error falls by 4 when h halves
    errs = []
    for n in (16, 32):
        g = Grid(n, n, n, 1.0 / n, 1.0 / n, 1.0 / n)
        t = np.arange(n) / n
        X, Y, Z = np.meshgrid(t, t, t, indexing="ij")
        E = pipe.electric_field(np.sin(2 * X) * np.cos(Y) * np.exp(Z), g)
        errs.append(np.abs(E[0] + 2 * np.cos(2 * X) * np.cos(Y) * np.exp(Z)).max())
    assert 3.0 < errs[0] / errs[1] < 5.0
