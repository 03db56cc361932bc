"""Seeded synthetic charge densities shaped like the paper's beams (Sec. 4).

The paper's numerical example (Sec. 4) uses a 3-D Gaussian bunch with
transverse rms sizes 0.15a, 0.15b and three bunch lengths, cut to zero outside
the 3-sigma ellipsoid, inside a rectangular pipe (0,a) x (0,b).  These
generators build such densities (and a uniform ellipsoid, and macroparticle
samples) on a mesh with nodes

    x_i = x0 + i*hx,  y_j = y0 + j*hy,  z_k = k*hz.

Everything here is FP64 and deterministic for a given seed.  Nothing here
touches the solver's arithmetic.
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np


@dataclass(frozen=True)
class Geometry:
    """Pipe cross-section (0,a) x (0,b), mesh origin (x0, y0), mode truncation."""

    a: float
    b: float
    x0: float
    y0: float
    modes_m: int = 20
    modes_n: int = 20


@dataclass(frozen=True)
class Grid:
    """Physical mesh nx x ny x nz with spacings hx, hy, hz."""

    nx: int
    ny: int
    nz: int
    hx: float
    hy: float
    hz: float

    @property
    def shape(self):
        return (self.nx, self.ny, self.nz)


def cell_centred(a: float, b: float, nx: int, ny: int, nz: int, hz: float, modes: int = 20):
    """Mesh spanning the whole pipe with nodes at cell centres (x0 = hx/2)."""
    hx, hy = a / nx, b / ny
    return Geometry(a, b, hx / 2, hy / 2, modes, modes), Grid(nx, ny, nz, hx, hy, hz)


def mesh_axes(geom: Geometry, grid: Grid):
    x = geom.x0 + grid.hx * np.arange(grid.nx)
    y = geom.y0 + grid.hy * np.arange(grid.ny)
    z = grid.hz * np.arange(grid.nz)
    return x, y, z


def _inside_pipe(geom, x, y):
    return (x > 0.0) & (x < geom.a) & (y > 0.0) & (y < geom.b)


def gaussian_bunch(geom: Geometry, grid: Grid, center, sigma, cutoff: float = 3.0,
                   total_charge: float | None = 1.0) -> np.ndarray:
    """Gaussian sampled at the nodes, zero outside the cutoff ellipsoid and the pipe.

    ``total_charge`` normalises hx*hy*hz*sum(rho); None leaves the peak at 1.
    """
    x, y, z = mesh_axes(geom, grid)
    X, Y, Z = np.meshgrid(x, y, z, indexing="ij")
    q = ((X - center[0]) / sigma[0]) ** 2 + ((Y - center[1]) / sigma[1]) ** 2 \
        + ((Z - center[2]) / sigma[2]) ** 2
    rho = np.exp(-0.5 * q)
    rho[q > cutoff * cutoff] = 0.0
    rho[~_inside_pipe(geom, X, Y)] = 0.0
    if total_charge is not None:
        s = rho.sum() * grid.hx * grid.hy * grid.hz
        rho *= total_charge / s
    return rho


def uniform_ellipsoid(geom: Geometry, grid: Grid, center, semi_axes,
                      total_charge: float | None = 1.0) -> np.ndarray:
    x, y, z = mesh_axes(geom, grid)
    X, Y, Z = np.meshgrid(x, y, z, indexing="ij")
    q = ((X - center[0]) / semi_axes[0]) ** 2 + ((Y - center[1]) / semi_axes[1]) ** 2 \
        + ((Z - center[2]) / semi_axes[2]) ** 2
    rho = (q <= 1.0).astype(np.float64)
    rho[~_inside_pipe(geom, X, Y)] = 0.0
    if total_charge is not None:
        s = rho.sum() * grid.hx * grid.hy * grid.hz
        rho *= total_charge / s
    return rho


def random_density(shape, seed: int, sparsity: float = 0.0) -> np.ndarray:
    """Uniform(-1, 1) values; a fraction ``sparsity`` of them set to zero."""
    rng = np.random.default_rng(seed)
    rho = rng.uniform(-1.0, 1.0, size=shape)
    if sparsity > 0:
        rho[rng.uniform(size=shape) < sparsity] = 0.0
    return rho


def particle_normals(n: int, seed: int, cutoff: float = 3.0) -> np.ndarray:
    """n standard-normal 3-vectors, redrawn while outside the cutoff sphere."""
    rng = np.random.default_rng(seed)
    out = rng.standard_normal((n, 3))
    bad = (out * out).sum(1) > cutoff * cutoff
    while bad.any():
        out[bad] = rng.standard_normal((int(bad.sum()), 3))
        bad = (out * out).sum(1) > cutoff * cutoff
    return out


# ---------------------------------------------------------------------------
# The five workloads.  Each returns plain data: geometry, grid, Green kind and
# one or more FP64 densities.
# ---------------------------------------------------------------------------

def workload_fp64_ordinary_16():
    """16x16x32 in a square pipe a=b=2 (half-width 1), hx=hy=2/16, hz=0.1.

    Ordinary point Green function, M=20; on-axis Gaussian sigma=(0.2,0.2,0.6)
    normalised to unit charge.
    """
    geom, grid = cell_centred(2.0, 2.0, 16, 16, 32, 0.1)
    zc = 0.5 * (grid.nz - 1) * grid.hz
    rho = gaussian_bunch(geom, grid, (1.0, 1.0, zc), (0.2, 0.2, 0.6))
    return dict(name="pipe16x16x32_ordinary", geom=geom, grid=grid, igf=0, rho=[rho])


def workload_igf_64(seed: int = 2):
    """64x64x256 IGF in a rectangular pipe a=2, b=1 (a/b=2), Lz=8a, M=20.

    Three seeded bunches: a Gaussian with sigma/a drawn in [0.05, 0.4] and
    sigma_z=a; a uniform ellipsoid (0.35a, 0.35b, 2.5a); an off-axis Gaussian
    (0.06a, 0.06b, a) displaced by +0.3a in x.
    """
    a, b = 2.0, 1.0
    nz = 256
    geom, grid = cell_centred(a, b, 64, 64, nz, 8 * a / nz)
    rng = np.random.default_rng(seed)
    s = rng.uniform(0.05, 0.4)
    zc = 0.5 * (nz - 1) * grid.hz
    c = (a / 2, b / 2, zc)
    rhos = [
        gaussian_bunch(geom, grid, c, (s * a, s * b, a)),
        uniform_ellipsoid(geom, grid, c, (0.35 * a, 0.35 * b, 2.5 * a)),
        gaussian_bunch(geom, grid, (a / 2 + 0.3 * a, b / 2, zc), (0.06 * a, 0.06 * b, a)),
    ]
    return dict(name="pipe64x64x256_igf_ab2", geom=geom, grid=grid, igf=1, rho=rhos,
                sigma_frac=s)


def workload_throughput_128():
    """128x128x1024 IGF, a=b=1, sigma_perp=0.15, sigma_z=3 (ratio 20), Lz=8 sigma_z."""
    nz = 1024
    geom, grid = cell_centred(1.0, 1.0, 128, 128, nz, 24.0 / nz)
    zc = 0.5 * (nz - 1) * grid.hz
    rho = gaussian_bunch(geom, grid, (0.5, 0.5, zc), (0.15, 0.15, 3.0))
    return dict(name="pipe128x128x1024_igf", geom=geom, grid=grid, igf=1, rho=[rho])


BATCH_GRIDS = ((32, 32, 64), (64, 64, 128), (64, 64, 256), (128, 128, 512))


def workload_batched_96(seed: int = 4, count: int = 96, with_rho: bool = True):
    """96 independent IGF solves on mixed grids and pipe aspect ratios a/b in [1,3]."""
    rng = np.random.default_rng(seed)
    items = []
    for _ in range(count):
        nx, ny, nz = BATCH_GRIDS[int(rng.integers(0, len(BATCH_GRIDS)))]
        b = 1.0
        a = float(rng.uniform(1.0, 3.0)) * b
        s = float(rng.uniform(0.05, 0.3))
        sz = 2 * a
        geom, grid = cell_centred(a, b, nx, ny, nz, 8 * sz / nz)
        zc = 0.5 * (nz - 1) * grid.hz
        rho = gaussian_bunch(geom, grid, (a / 2, b / 2, zc), (s * a, s * b, sz)) if with_rho else None
        items.append(dict(geom=geom, grid=grid, igf=1, rho=rho))
    return items


def workload_differentiable_128(seed: int = 5, n_particles: int = 1 << 20):
    """128x128x512, a=b=1, Lz=12.8; 2^20 macroparticles x = mu + sigma*xi."""
    nz = 512
    geom, grid = cell_centred(1.0, 1.0, 128, 128, nz, 12.8 / nz)
    zc = 0.5 * (nz - 1) * grid.hz
    return dict(name="pipe128x128x512_cic", geom=geom, grid=grid, igf=1,
                mu=np.array([0.5, 0.5, zc]), sigma=np.array([0.15, 0.15, 2.0]),
                xi=particle_normals(n_particles, seed), charge=1.0 / n_particles)


def windowed(geom: Geometry, grid: Grid, a: float, b: float, modes: int | None = None):
    """Same mesh placed centrally inside a larger pipe (a transverse window)."""
    x0 = 0.5 * (a - (grid.nx - 1) * grid.hx)
    y0 = 0.5 * (b - (grid.ny - 1) * grid.hy)
    m = geom.modes_m if modes is None else modes
    return replace(geom, a=a, b=b, x0=x0, y0=y0, modes_m=m, modes_n=m)


def accuracy_study_case(sigma_z: float, n: int, nz: int, modes: int = 20):
    """Accuracy-study bunch (Sec. 4, Figs. 2-4): square pipe a = b = 1, wall-node
    mesh (x0 = y0 = 0, n*h = a, so node n/2 lies on the axis), Gaussian with
    sigma_x = sigma_y = 0.15 a and the given sigma_z, centred on the axis at
    z = Lz/2 with Lz = 8 sigma_z; nodes z_k = k*Lz/nz, so a coarse node k is the
    fine node k*(nz_fine/nz).  Unit total charge."""
    geom = Geometry(1.0, 1.0, 0.0, 0.0, modes, modes)
    lz = 8.0 * sigma_z
    grid = Grid(n, n, nz, 1.0 / n, 1.0 / n, lz / nz)
    rho = gaussian_bunch(geom, grid, (0.5, 0.5, 0.5 * lz), (0.15, 0.15, sigma_z))
    return geom, grid, rho
