"""1-D FFT-based convolution and correlation (Appendix A), FP64.

``brute_convolution``  p_j = sum_{k<K} r_k x_{j-k},  j < J   (Eq. A.1)
``brute_correlation``  p_j = sum_{k<K} r_k x_{j+k},  j < J   (Eq. A.9)
``fft_convolution``    zero-padded r, periodic Green sequence xi (Eq. A.2-A.3),
                       then Eq. A.4 with W = e^{-2 pi i/N}.
``fft_correlation``    Eq. A.4 with W^{-jk} -> W^{jk} and W^{mk} -> W^{-mk}
                       (the direction swap stated after Eq. A.8).

The Green sequence ``x`` is given as a dict {offset: value}.  For the
convolution the offsets span -(K-1)..J-1; for the correlation they span
0..J+K-2 (the index j+k of Eq. A.9 runs over that range).
"""
from __future__ import annotations

import numpy as np


def brute_convolution(r, x, J):
    K = len(r)
    return np.array([sum(r[k] * x[j - k] for k in range(K)) for j in range(J)])


def brute_correlation(r, x, J):
    K = len(r)
    return np.array([sum(r[k] * x[j + k] for k in range(K)) for j in range(J)])


def _W(N):
    return np.exp(-2j * np.pi / N)


def fft_convolution(r, x, J, N):
    K = len(r)
    assert N >= J + K - 1
    rho = np.zeros(N, dtype=np.complex128)
    rho[:K] = r
    xi = np.zeros(N, dtype=np.complex128)
    for m in range(-(K - 1), J):
        xi[m % N] = x[m]
    W = _W(N)
    k = np.arange(N)
    R = np.array([np.sum(rho * W ** (np.arange(N) * kk)) for kk in k])
    X = np.array([np.sum(xi * W ** (np.arange(N) * kk)) for kk in k])
    phi = np.array([np.sum(W ** (-j * k) * R * X) / N for j in range(N)])
    return phi[:J]


def fft_correlation(r, x, J, N):
    K = len(r)
    assert N >= J + K - 1
    rho = np.zeros(N, dtype=np.complex128)
    rho[:K] = r
    xi = np.zeros(N, dtype=np.complex128)
    for m in range(0, J + K - 1):
        xi[m] = x[m]
    W = _W(N)
    k = np.arange(N)
    R = np.array([np.sum(rho * W ** (np.arange(N) * kk)) for kk in k])
    X = np.array([np.sum(xi * W ** (-np.arange(N) * kk)) for kk in k])
    phi = np.array([np.sum(W ** (j * k) * R * X) / N for j in range(N)])
    return phi[:J]
