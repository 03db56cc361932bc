"""Green functions of the open rectangular pipe (Sec. 1-3), FP64.

Readings of the paper taken here (each listed in the design notes):

* Prefactor (Eq. 7, Eq. 9, Eq. 16).  The paper prints 1/(2 pi a b) for both the
  sine series G and the cosine series R.  Those two cannot both hold: the
  product-to-sum identity sin A sin B = [cos(A-B) - cos(A+B)]/2, used twice,
  gives R = G_prefactor / 4.  The normalisation that makes G -> 1/r near the
  source (the free-space Green function of Eq. 3, i.e. laplacian G = -4 pi
  delta) is G = (8 pi/(a b)) sum ..., hence R = (2 pi/(a b)) sum ....  We use
  those, so that the potential is phi = h^3 sum rho G with G ~ 1/r; a caller
  wanting SI units applies 1/(4 pi eps0).
* Truncation.  The series are summed over m = 1..M, n = 1..N (M = N = 20 in
  Sec. 4); the truncated series *is* the Green function.
* IGF evaluation (Eq. 15).  ``gz_literal`` evaluates the printed formula;
  ``gz_stable`` is an exact rewrite without cancellation:
      |w| >= h:  g = 4 sinh^2(kappa h/2) e^{-kappa |w|} / (kappa h)^2
      w  = 0  :  g = 2 (kappa h - 1 + e^{-kappa h}) / (kappa h)^2
  with a Taylor series of (x - 1 + e^{-x})/x^2 for x < 0.1.  The IGF is only
  evaluated at mesh offsets w = r*hz.
"""
from __future__ import annotations

import numpy as np


def kappa(m, n, a, b):
    """kappa_mn with kappa^2 = (m pi/a)^2 + (n pi/b)^2 (Sec. 2, below Eq. 7)."""
    return np.pi * np.sqrt((np.asarray(m, dtype=np.float64) / a) ** 2
                           + (np.asarray(n, dtype=np.float64) / b) ** 2)


def mode_grid(geom):
    """(m, n, kappa_mn) on the truncated mode set, shapes (M,1), (1,N), (M,N)."""
    m = np.arange(1, geom.modes_m + 1, dtype=np.float64)[:, None]
    n = np.arange(1, geom.modes_n + 1, dtype=np.float64)[None, :]
    return m, n, kappa(m, n, geom.a, geom.b)


def prefactor_R(geom):
    """Cosine-series prefactor 2 pi/(a b) (reading of Eq. 9, see module doc)."""
    return 2.0 * np.pi / (geom.a * geom.b)


def prefactor_G(geom):
    """Sine-series prefactor 8 pi/(a b) (reading of Eq. 7, see module doc)."""
    return 8.0 * np.pi / (geom.a * geom.b)


def gz_literal(w, kap, hz):
    """Longitudinal IGF exactly as printed in Eq. 15."""
    w, kap = np.broadcast_arrays(np.asarray(w, dtype=np.float64),
                                 np.asarray(kap, dtype=np.float64))
    delta = (w == 0.0).astype(np.float64)
    num = (2.0 * hz * kap * delta + np.exp(-kap * np.abs(w + hz))
           - 2.0 * np.exp(-kap * np.abs(w)) + np.exp(-kap * np.abs(w - hz)))
    return num / (hz * kap) ** 2


def _xm1pe_over_x2(x):
    """(x - 1 + exp(-x)) / x^2 without cancellation (series below 0.1)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    small = x < 0.1
    xs = x[small]
    # sum_{j>=0} (-x)^j / (j+2)!
    term = np.full_like(xs, 0.5)
    acc = term.copy()
    for j in range(1, 16):
        term = term * (-xs) / (j + 2)
        acc = acc + term
    out[small] = acc
    xl = x[~small]
    out[~small] = (xl - 1.0 + np.exp(-xl)) / (xl * xl)
    return out


def gz_stable(w, kap, hz):
    """Eq. 15 rewritten without cancellation (same values at mesh offsets)."""
    w, kap = np.broadcast_arrays(np.asarray(w, dtype=np.float64),
                                 np.asarray(kap, dtype=np.float64))
    x = kap * hz
    aw = np.abs(w)
    on_source = aw < 0.5 * hz
    s = np.sinh(0.5 * x)
    far = 4.0 * s * s * np.exp(-kap * aw) / (x * x)
    near = 2.0 * _xm1pe_over_x2(x)
    return np.where(on_source, near, far)


def z_profile(w, kap, hz, igf):
    """Longitudinal factor of the mode series: e^{-kappa|w|} (Eq. 9) or g_z (Eq. 16)."""
    if igf:
        return gz_stable(w, kap, hz)
    return np.exp(-np.asarray(kap) * np.abs(np.asarray(w, dtype=np.float64)))


def green_sine(x, xp, y, yp, w, geom, igf=False, hz=None):
    """Pipe Green function as the double sine series, Eq. 7 (prefactor 8 pi/(ab)).

    ``w = z - z'``.  With ``igf`` the longitudinal factor is g_z(w) (Eq. 15,
    integrated in z only, Sec. 3).  Arguments broadcast.
    """
    x, xp, y, yp, w = np.broadcast_arrays(*[np.asarray(v, dtype=np.float64)
                                             for v in (x, xp, y, yp, w)])
    acc = np.zeros(x.shape)
    for m in range(1, geom.modes_m + 1):
        sx = np.sin(m * np.pi * x / geom.a) * np.sin(m * np.pi * xp / geom.a)
        for n in range(1, geom.modes_n + 1):
            k = kappa(m, n, geom.a, geom.b)
            sy = np.sin(n * np.pi * y / geom.b) * np.sin(n * np.pi * yp / geom.b)
            acc += sx * sy * z_profile(w, k, hz, igf) / k
    return prefactor_G(geom) * acc


def R_function(u, v, w, geom, igf=False, hz=None):
    """R(u,v,w) of Eq. 9 (ordinary) or R_int of Eq. 16 (igf), prefactor 2 pi/(ab)."""
    u, v, w = np.broadcast_arrays(*[np.asarray(t, dtype=np.float64) for t in (u, v, w)])
    acc = np.zeros(u.shape)
    for m in range(1, geom.modes_m + 1):
        cu = np.cos(m * np.pi * u / geom.a)
        for n in range(1, geom.modes_n + 1):
            k = kappa(m, n, geom.a, geom.b)
            acc += cu * np.cos(n * np.pi * v / geom.b) * z_profile(w, k, hz, igf) / k
    return prefactor_R(geom) * acc


def green_four_R(x, xp, y, yp, w, geom, igf=False, hz=None):
    """Eq. 8: G = R(x-x',y-y') - R(x-x',y+y') - R(x+x',y-y') + R(x+x',y+y')."""
    return (R_function(x - xp, y - yp, w, geom, igf, hz)
            - R_function(x - xp, y + yp, w, geom, igf, hz)
            - R_function(x + xp, y - yp, w, geom, igf, hz)
            + R_function(x + xp, y + yp, w, geom, igf, hz))


def green_free(u, v, w, self_value=None):
    """Free-space Green function 1/sqrt(u^2+v^2+w^2) (Eq. 3).

    The value at the origin is not given by the paper; ``self_value`` supplies
    it (the Hockney comparison uses 1/min(hx,hy,hz)).
    """
    u, v, w = np.broadcast_arrays(*[np.asarray(t, dtype=np.float64) for t in (u, v, w)])
    r = np.sqrt(u * u + v * v + w * w)
    out = np.empty(r.shape)
    zero = r == 0.0
    out[~zero] = 1.0 / r[~zero]
    out[zero] = np.nan if self_value is None else self_value
    return out
