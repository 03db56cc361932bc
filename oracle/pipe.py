"""The discretised pipe Poisson problem, solved three independent ways (FP64).

Problem (Eq. 1 discretised as Eq. 4, with the pipe Green function of Eq. 7):

    phi_ijk = hx hy hz  sum_{i'j'k'} rho_{i'j'k'} G(x_i, x_i', y_j, y_j', z_k - z_k')

on the mesh x_i = x0 + i hx, y_j = y0 + j hy, z_k = k hz (node placement and
origin are not stated in the paper; the mesh origin is a parameter).

O1  ``direct_sum``        the triple sum above, G from the sine series Eq. 7.
O2  ``naive_dft_solve``   Eq. 10 literally: zero-padded rho, one forward
                          transform, four Green tables transformed with the
                          printed directions, four products, four final
                          transforms with the printed directions, summed,
                          cropped and scaled.  Transforms are dense DFT
                          matrices applied per axis.
O3  ``fft_solve``         the same with scipy.fft.

The banded reduction of Sec. 5 (Eq. 17-18: only source planes within n_nb of
the output plane) has its own pair: ``direct_sum_banded`` (O1 restricted to
the band) and ``banded_solve`` (2-D transforms per z-offset).

Conventions (Sec. 1 below Eq. 5, Eq. A.4): the forward transform f is
sum_n a_n e^{-2 pi i nk/N}, the backward transform b is sum_n a_n e^{+2 pi i nk/N};
a *final* transform carries 1/N per dimension (Eq. A.4), whatever its
direction (Eq. A.9).

Doubled-grid tables (Fig. 1 right; Eq. A.2-A.3).  On an axis with N physical
points the padded length is 2N.
  convolution (x - x'):  offset p*h for p <= N, (p - 2N)*h for p > N; slot p = N
                         is never used by the physical block and holds the
                         formula's value there.
  correlation (x + x'):  offset 2*x0 + p*h for p = 0..2N-1 (the sum index
                         i + i' runs over 0..2N-2, Eq. A.9 with the index range
                         of a correlation; slot 2N-1 is unused and holds the
                         formula's value).
z is always a convolution (G depends on z - z').
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft

from . import green

# (sign, x kind, y kind, Green transform directions, final transform directions)
# exactly the four terms of Eq. 10.
TERMS = (
    (+1.0, "c", "c", "fff", "bbb"),
    (-1.0, "c", "r", "fbf", "bfb"),
    (-1.0, "r", "c", "bff", "fbb"),
    (+1.0, "r", "r", "bbf", "ffb"),
)


def h3(grid):
    return grid.hx * grid.hy * grid.hz


def mesh(geom, grid):
    x = geom.x0 + grid.hx * np.arange(grid.nx)
    y = geom.y0 + grid.hy * np.arange(grid.ny)
    z = grid.hz * np.arange(grid.nz)
    return x, y, z


# ---------------------------------------------------------------------------
# O1: brute-force sum (Eq. 4 with Eq. 7)
# ---------------------------------------------------------------------------

def direct_sum_banded(rho, geom, grid, igf, n_nb):
    """Eq. 18 by brute force: the sum of O1 with the source planes restricted
    to |k - k'| <= n_nb (n_nb = 0 is Eq. 17, one 2-D sum per plane)."""
    rho = np.asarray(rho, dtype=np.float64)
    G4 = _pair_green(geom, grid, igf)
    nz = grid.nz
    phi = np.empty(rho.shape)
    for k in range(nz):
        kp = np.arange(max(0, k - n_nb), min(nz, k + n_nb + 1))
        sl = G4[..., k - kp + nz - 1]
        phi[:, :, k] = np.einsum("ikjlq,klq->ij", sl, rho[:, :, kp])
    return h3(grid) * phi


def banded_solve(rho, geom, grid, igf, n_nb, workers=None):
    """Eq. 18 with transforms: for every output plane k, the sum over
    d = -n_nb..n_nb of the 2-D mixed convolution/correlation (the x, y part of
    Eq. 10, on the doubled transverse grid) of source plane k - d with the R
    tables at z-offset d*hz.  Source planes outside 0..nz-1 are zero."""
    nx, ny, nz = grid.shape
    T = green_tables(geom, grid, igf)                  # z offsets d at slot d mod 2nz
    P = np.zeros((2 * nx, 2 * ny, nz))
    P[:nx, :ny, :] = rho
    P_hat = transform(P, "ff", workers=workers)        # x and y only
    acc = np.zeros(P_hat.shape, dtype=np.complex128)
    for d in range(-n_nb, n_nb + 1):
        S = np.zeros_like(P_hat)
        lo, hi = max(0, d), min(nz, nz + d)            # planes k with 0 <= k - d < nz
        S[:, :, lo:hi] = P_hat[:, :, lo - d:hi - d]
        for sign, kx, ky, gdir, fdir in TERMS:
            spec = transform(T[kx + ky][:, :, d % (2 * nz)], gdir[:2], workers=workers)
            acc += sign * transform(S * spec[:, :, None], fdir[:2], final=True, workers=workers)
    return h3(grid) * acc[:nx, :ny, :].real


def _pair_green(geom, grid, igf):
    """G4[i, i', j, j', d] = G(x_i, x_i', y_j, y_j', (d - nz + 1) hz), Eq. 7.

    The sine series is summed with tensor contractions over the mode indices
    (a plain evaluation of the double sum; nothing is dropped).
    """
    x, y, _ = mesh(geom, grid)
    m, n, kap = green.mode_grid(geom)
    sx = np.sin(m * np.pi * x[None, :] / geom.a)          # (M, nx)
    sy = np.sin(n.T * np.pi * y[None, :] / geom.b)        # (N, ny)
    d = np.arange(-(grid.nz - 1), grid.nz) * grid.hz       # (D,)
    Z = green.z_profile(d[None, None, :], kap[:, :, None], grid.hz, igf) / kap[:, :, None]
    Px = np.einsum("mi,mk->mik", sx, sx)
    Py = np.einsum("nj,nl->njl", sy, sy)
    tmp = np.einsum("njl,mnd->mjld", Py, Z)
    return green.prefactor_G(geom) * np.einsum("mik,mjld->ikjld", Px, tmp)


def direct_sum(rho, geom, grid, igf=False):
    """O1: phi = h^3 sum rho G, the O(N^6) sum of Eq. 4 with the pipe G of Eq. 7."""
    rho = np.asarray(rho, dtype=np.float64)
    G4 = _pair_green(geom, grid, igf)
    nz = grid.nz
    phi = np.empty(rho.shape)
    kp = np.arange(nz)
    for k in range(nz):
        sl = G4[..., k - kp + nz - 1]                       # (i, i', j, j', k')
        phi[:, :, k] = np.einsum("ikjlq,klq->ij", sl, rho)
    return h3(grid) * phi


def direct_sum_adjoint(dphi, geom, grid, igf=False):
    """Transpose of O1: drho_{i'j'k'} = h^3 sum_{ijk} dphi_{ijk} G(x_i,x_i',y_j,y_j',z_k-z_k')."""
    dphi = np.asarray(dphi, dtype=np.float64)
    G4 = _pair_green(geom, grid, igf)
    nz = grid.nz
    out = np.empty(dphi.shape)
    k = np.arange(nz)
    for kp in range(nz):
        sl = G4[..., k - kp + nz - 1]                       # (i, i', j, j', k)
        out[:, :, kp] = np.einsum("ikjlq,ijq->kl", sl, dphi)
    return h3(grid) * out


def direct_sum_at(rho, geom, grid, igf, nodes):
    """Exact O1 values phi_ijk at the listed mesh nodes [(i, j, k), ...].

    Same sum as ``direct_sum``; the sums over sources are taken inside the
    mode sum (G of Eq. 7 is a sum of separable terms), so that single outputs
    of a large mesh cost O(M N nx ny nz) instead of a full solve.
    """
    rho = np.asarray(rho, dtype=np.float64)
    x, y, z = mesh(geom, grid)
    m, n, kap = green.mode_grid(geom)
    sx = np.sin(m * np.pi * x[None, :] / geom.a)            # (M, nx)
    sy = np.sin(n.T * np.pi * y[None, :] / geom.b)          # (N, ny)
    # projections rho~[m, n, k'] = sum_{i'j'} sin sin rho
    t = np.tensordot(sx, rho, axes=([1], [0]))              # (M, ny, nz)
    proj = np.einsum("nj,mjk->mnk", sy, t)                  # (M, N, nz)
    out = []
    for (i, j, k) in nodes:
        w = z[k] - z                                        # (nz,)
        Zk = green.z_profile(w[None, None, :], kap[:, :, None], grid.hz, igf)
        s = np.sum(sx[:, i][:, None] * sy[:, j][None, :] / kap * np.sum(Zk * proj, axis=2))
        out.append(green.prefactor_G(geom) * h3(grid) * s)
    return np.array(out)


# ---------------------------------------------------------------------------
# Doubled-grid tables (Fig. 1, Eq. A.2-A.3)
# ---------------------------------------------------------------------------

def conv_offsets(n, h):
    p = np.arange(2 * n)
    return np.where(p <= n, p, p - 2 * n) * h


def corr_offsets(n, h, origin):
    return 2.0 * origin + np.arange(2 * n) * h


def pad(rho, grid):
    """Zero-padded density on the doubled grid, physical block in the corner (Eq. A.2)."""
    out = np.zeros((2 * grid.nx, 2 * grid.ny, 2 * grid.nz))
    out[:grid.nx, :grid.ny, :grid.nz] = rho
    return out


def green_tables(geom, grid, igf):
    """The four R tables T_{xy} on the doubled grid, x,y in {c(onv), r(corr)}.

    T_xy[p, q, r] = R(ox(p), oy(q), oz(r)) with R from Eq. 9 (or R_int, Eq. 16)
    and the offsets defined in the module docstring.  The mode sum is
    evaluated with tensor contractions.
    """
    m, n, kap = green.mode_grid(geom)
    ox = {"c": conv_offsets(grid.nx, grid.hx), "r": corr_offsets(grid.nx, grid.hx, geom.x0)}
    oy = {"c": conv_offsets(grid.ny, grid.hy), "r": corr_offsets(grid.ny, grid.hy, geom.y0)}
    oz = conv_offsets(grid.nz, grid.hz)
    Z = green.z_profile(oz[None, None, :], kap[:, :, None], grid.hz, igf) / kap[:, :, None]
    C = green.prefactor_R(geom)
    out = {}
    for kx in "cr":
        cx = np.cos(m * np.pi * ox[kx][None, :] / geom.a)      # (M, 2nx)
        U = np.tensordot(cx, Z, axes=([0], [0]))               # (2nx, N, 2nz)
        for ky in "cr":
            cy = np.cos(n.T * np.pi * oy[ky][None, :] / geom.b)  # (N, 2ny)
            T = np.einsum("pnr,nq->pqr", U, cy, optimize=True)
            out[kx + ky] = C * T
    return out


def free_space_table(grid, self_value=None):
    """Free-space 1/r on the doubled grid with convolution offsets in x, y, z (Eq. 5).

    The self term G(0,0,0) is not given by the paper; it defaults to
    1/min(hx, hy, hz).
    """
    if self_value is None:
        self_value = 1.0 / min(grid.hx, grid.hy, grid.hz)
    ox = conv_offsets(grid.nx, grid.hx)[:, None, None]
    oy = conv_offsets(grid.ny, grid.hy)[None, :, None]
    oz = conv_offsets(grid.nz, grid.hz)[None, None, :]
    return green.green_free(ox, oy, oz, self_value)


# ---------------------------------------------------------------------------
# Direction-controlled transforms (Sec. 1 below Eq. 5, Sec. 5, Eq. A.4, Eq. A.9)
# ---------------------------------------------------------------------------

def dft_matrix(n, direction):
    k = np.arange(n)
    sign = -1.0 if direction == "f" else 1.0
    return np.exp(sign * 2j * np.pi * np.outer(k, k) / n)


def transform(a, dirs, naive=False, final=False, workers=None):
    """Apply a 1-D transform along each axis with its own direction.

    ``dirs`` is a string like 'fbf'; 'f' = e^{-}, 'b' = e^{+}.  ``final`` divides
    by N along every axis (Eq. A.4).
    """
    out = np.asarray(a, dtype=np.complex128)
    for axis, d in enumerate(dirs):
        n = out.shape[axis]
        if naive:
            out = np.moveaxis(np.tensordot(dft_matrix(n, d), out, axes=([1], [axis])), 0, axis)
        elif d == "f":
            out = sfft.fft(out, axis=axis, workers=workers)
        else:
            out = sfft.ifft(out, axis=axis, workers=workers) * n
        if final:
            out = out / n
    return out


def green_spectra(geom, grid, igf, naive=False, workers=None):
    """The four transformed tables of Eq. 10: F^fff T_cc, F^fbf T_cr, F^bff T_rc, F^bbf T_rr."""
    T = green_tables(geom, grid, igf)
    return {kx + ky: transform(T[kx + ky], gdir, naive=naive, workers=workers)
            for (_, kx, ky, gdir, _) in TERMS}


def _four_term_solve(rho, geom, grid, spectra, naive, workers):
    rho_hat = transform(pad(rho, grid), "fff", naive=naive, workers=workers)
    acc = np.zeros(rho_hat.shape, dtype=np.complex128)
    for sign, kx, ky, _, fdir in TERMS:
        acc += sign * transform(rho_hat * spectra[kx + ky], fdir, naive=naive,
                                final=True, workers=workers)
    return h3(grid) * acc[:grid.nx, :grid.ny, :grid.nz].real


def naive_dft_solve(rho, geom, grid, igf=False):
    """O2: Eq. 10 with every transform a dense DFT matrix (small grids only)."""
    spectra = green_spectra(geom, grid, igf, naive=True)
    return _four_term_solve(rho, geom, grid, spectra, True, None)


def fft_solve(rho, geom, grid, igf=False, spectra=None, workers=None):
    """O3: Eq. 10 with scipy.fft.  ``spectra`` may be precomputed (Sec. 5: the
    Green function is transformed once and reused)."""
    if spectra is None:
        spectra = green_spectra(geom, grid, igf, workers=workers)
    return _four_term_solve(rho, geom, grid, spectra, False, workers)


def fft_adjoint(dphi, geom, grid, igf=False, spectra=None, naive=False, workers=None):
    """Transpose of Eq. 10 (A^T = crop F_fff D F_final pad for each term).

    Each term is applied in reverse: the zero-padded input goes through the
    term's *final* transform (with its 1/N), is multiplied by the same Green
    spectrum, and then through the forward transform F^fff; crop, real part.
    """
    if spectra is None:
        spectra = green_spectra(geom, grid, igf, naive=naive, workers=workers)
    u = pad(dphi, grid)
    acc = np.zeros(u.shape, dtype=np.complex128)
    for sign, kx, ky, _, fdir in TERMS:
        v = transform(u, fdir, naive=naive, final=True, workers=workers) * spectra[kx + ky]
        acc += sign * transform(v, "fff", naive=naive, workers=workers)
    return h3(grid) * acc[:grid.nx, :grid.ny, :grid.nz].real


def green_spectrum_octant(geom, grid, igf, scaled=True):
    """Real octant of F^fff T_cc, indices [0..nx] x [0..ny] x [0..nz] (FP64).

    For meshes spanning the whole pipe this one array determines all four
    spectra of Eq. 10 (the correlation tables are the convolution table
    shifted by 2*x0/h samples).  ``scaled`` multiplies by h^3/(8 nx ny nz),
    the overall factor of Eq. 10 with the 1/N of the final transforms.
    """
    T = green_tables(geom, grid, igf)["cc"]
    S = transform(T, "fff")
    oct_ = S[:grid.nx + 1, :grid.ny + 1, :grid.nz + 1]
    if scaled:
        oct_ = oct_ * (h3(grid) / (8.0 * grid.nx * grid.ny * grid.nz))
    return oct_


# ---------------------------------------------------------------------------
# Free-space Hockney comparison (Eq. 2-5)
# ---------------------------------------------------------------------------

def hockney_direct(rho, grid, self_value=None):
    """phi = h^3 sum rho G_free(x_i - x_i', ...) by brute force (Eq. 4 with Eq. 3)."""
    if self_value is None:
        self_value = 1.0 / min(grid.hx, grid.hy, grid.hz)
    nx, ny, nz = grid.shape
    dx = (np.arange(nx)[:, None] - np.arange(nx)[None, :]) * grid.hx
    dy = (np.arange(ny)[:, None] - np.arange(ny)[None, :]) * grid.hy
    dz = (np.arange(nz)[:, None] - np.arange(nz)[None, :]) * grid.hz
    G = green.green_free(dx[:, :, None, None, None, None], dy[None, None, :, :, None, None],
                         dz[None, None, None, None, :, :], self_value)
    return h3(grid) * np.einsum("ikjlqr,klr->ijq", G, np.asarray(rho, dtype=np.float64))


def hockney_fft(rho, grid, self_value=None, workers=None):
    """Eq. 5: phi = h^3 F^bbb{(F^fff rho)(F^fff G)} on the doubled grid, cropped."""
    Gh = transform(free_space_table(grid, self_value), "fff", workers=workers)
    rh = transform(pad(rho, grid), "fff", workers=workers)
    out = transform(rh * Gh, "bbb", final=True, workers=workers)
    return h3(grid) * out[:grid.nx, :grid.ny, :grid.nz].real


def hockney_spectrum_octant(grid, self_value=None, scaled=True):
    S = transform(free_space_table(grid, self_value), "fff")
    oct_ = S[:grid.nx + 1, :grid.ny + 1, :grid.nz + 1]
    if scaled:
        oct_ = oct_ * (h3(grid) / (8.0 * grid.nx * grid.ny * grid.nz))
    return oct_


def electric_field(phi, grid):
    """E = -grad phi on the mesh (the field a particle-in-cell code gathers).

    The paper gives no discrete gradient; the reading taken is second-order
    central differences inside the mesh and second-order one-sided
    differences on its faces, i.e. numpy.gradient with edge_order=2 (exact
    for potentials quadratic in each coordinate).  Returns E[3][nx][ny][nz].
    """
    g = np.gradient(np.asarray(phi, dtype=np.float64), grid.hx, grid.hy, grid.hz, edge_order=2)
    return -np.stack(g)


def field_energy(rho, phi, grid):
    """W = 1/2 sum rho phi (the objective of the differentiable workload)."""
    return 0.5 * float(np.sum(np.asarray(rho) * np.asarray(phi)))
