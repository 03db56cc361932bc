"""CPU checks of the identities the GPU kernels are built on, in plain numpy.

The CUDA kernels never compute the padded transforms of Eq. 10 literally:
they rely on a few exact rewrites (Appendix A's zero padding, the
direction swap for correlations, real-to-complex packing).  These tests state
each rewrite next to its literal form and check them on random data, so that
a sign or index slip in the reasoning behind a kernel shows up on the CPU.
They share no code with the kernels or with the oracle.
"""
import numpy as np
import pytest


def group_shape(L):
    """(G, E): lanes per group and elements per lane of an L-point group FFT."""
    G = 4 if L <= 32 else 8 if L <= 128 else 16 if L <= 512 else 32
    return G, L // G


@pytest.mark.parametrize("L", [16, 32, 64, 128, 256, 512, 1024])
def test_mirror_slot_map_of_the_cyclic_layout(L):
    """Lane t of a group holds q = t + G e.  The mirror L - q (mod L) of slot e
    is slot E-1-e of lane (G - t) mod G, except in lane 0, whose slots e and
    (E - e) mod E are each other's mirrors (slot 0 is q = 0 and slot E/2 is
    q = L/2, each its own).  For the odd frequencies of a split transform the
    mirror L-1-q of slot e is slot E-1-e of lane G-1-t."""
    G, E = group_shape(L)
    for t in range(G):
        for e in range(E):
            q = t + G * e
            if t == 0:
                tm, em = 0, (E - e) % E
            else:
                tm, em = G - t, E - 1 - e
            assert tm + G * em == (L - q) % L
            # odd half
            assert (G - 1 - t) + G * (E - 1 - e) == L - 1 - q
    # the pairs handled by a lane's slots j < E/2 cover every frequency once
    covered = []
    for t in range(G):
        for j in range(E // 2):
            q = t + G * j
            covered += [q, (L - q) % L] if t or j else [0]
        if t == 0:
            covered.append(L // 2)
    assert sorted(covered) == list(range(L))


@pytest.mark.parametrize("N", [16, 32, 128])
@pytest.mark.parametrize("adjoint", [False, True])
def test_npoint_line_transform_and_its_pairs(N, adjoint):
    """The image combination of a cell-centred line (shift s = 1),
    U(q) = Y(q) - w^{-q} Y(-q) with Y the 2N-point transform of the
    zero-padded line and w = exp(-+ i pi/N), equals V(q) - w^{-q} V(N-q) with V
    the N-point transform of v_n = x_{2n} (2n < N), -x_{2N-1-2n} (otherwise);
    U(N) = 2 V(0).  The mirror member of a pair takes w^{-(N-q)} =
    -conj(w^{-q}), so one lane computes both U(q) and U(N-q)."""
    rng = np.random.default_rng(N + adjoint)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    sgn = 1 if adjoint else -1                       # forward e^{-}, adjoint e^{+}
    def dft(a, M):
        k = np.arange(M)
        return np.exp(sgn * 2j * np.pi * np.outer(k, k) / M) @ a
    Y = dft(np.concatenate([x, np.zeros(N)]), 2 * N)
    w = np.exp(sgn * 1j * np.pi / N)                 # w_{2N}
    wm = lambda q: w ** (-q)                         # the phase w^{-q} of the kernels
    U = np.array([Y[q] - wm(q) * Y[(-q) % (2 * N)] for q in range(1, N + 1)])
    n = np.arange(N)
    v = np.where(2 * n < N, x[np.minimum(2 * n, N - 1)], -x[np.clip(2 * N - 1 - 2 * n, 0, N - 1)])
    V = dft(v, N)
    for q in range(1, N):
        assert abs(U[q - 1] - (V[q] - wm(q) * V[N - q])) < 1e-10 * np.abs(Y).max()
        # the pair member N - q from the same two values
        assert abs(U[N - q - 1] - (V[N - q] + np.conj(wm(q)) * V[q])) < 1e-10 * np.abs(Y).max()
    assert abs(U[N - 1] - 2 * V[0]) < 1e-10 * np.abs(Y).max()
    assert np.allclose(wm(N - np.arange(N)), -np.conj(wm(np.arange(N))))


@pytest.mark.parametrize("N", [16, 64])
@pytest.mark.parametrize("adjoint", [False, True])
def test_npoint_inverse_line_and_its_pairs(N, adjoint):
    """A spectrum with P(-q) = -w^q P(q) (what the even Green table leaves)
    has as its 2N-point inverse transform a sequence whose even samples are
    the N-point inverse transform of V'(q) = P(q) + w^{-q} P(N-q),
    V'(0) = P(N), and whose odd samples 2n+1 are minus the even sample
    2(N-1-n); in pairs V'(N-q) = P(N-q) - conj(w^{-q}) P(q)."""
    rng = np.random.default_rng(3 * N + adjoint)
    sgn = 1 if adjoint else -1
    binv = -sgn                                      # the inverse direction
    w = np.exp(sgn * 1j * np.pi / N)
    P = np.zeros(2 * N, complex)
    P[1:N + 1] = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    for q in range(1, N):
        P[2 * N - q] = -(w ** q) * P[q]
    k = np.arange(2 * N)
    y = np.exp(binv * 2j * np.pi * np.outer(k, k) / (2 * N)) @ P
    Vp = np.array([P[N] if q == 0 else P[q] + w ** (-q) * P[N - q] for q in range(N)])
    kk = np.arange(N)
    even = np.exp(binv * 2j * np.pi * np.outer(kk, kk) / N) @ Vp
    scale = np.abs(y).max()
    assert np.abs(y[0::2] - even).max() < 1e-10 * scale
    assert np.abs(y[1::2] + even[::-1]).max() < 1e-10 * scale
    for q in range(1, N):
        assert abs(Vp[N - q] - (P[N - q] - np.conj(w ** (-q)) * P[q])) < 1e-10 * scale


@pytest.mark.parametrize("nz", [32, 256, 1024])
def test_real_to_complex_pairs_of_the_padded_z_transform(nz):
    """Appendix A's zero-padded 2nz-point transform of a real column, from the
    nz-point transform Z of the packed column z_m = rho_{2m} + i rho_{2m+1}
    (m < nz/2; the padded half is zero):
    X(k) = (Z(k) + conj Z(nz-k) - i w^k (Z(k) - conj Z(nz-k))) / 2, w = w_{2nz};
    X(nz - k) takes the same pair swapped and w^{nz-k} = -conj(w^k), and
    X(nz) = Re Z(0) - Im Z(0)."""
    rng = np.random.default_rng(nz)
    rho = rng.standard_normal(nz)
    X = np.fft.fft(np.concatenate([rho, np.zeros(nz)]))[: nz + 1]
    z = np.zeros(nz, complex)
    z[: nz // 2] = rho[0::2] + 1j * rho[1::2]
    Z = np.fft.fft(z)
    w = np.exp(-1j * np.pi / nz)
    def r2c(zk, zm, wk):
        s, d = zk + np.conj(zm), zk - np.conj(zm)
        return (s - 1j * wk * d) / 2
    scale = np.abs(X).max()
    for k in range(nz // 2 + 1):
        zk, zm = Z[k % nz], Z[(nz - k) % nz]
        assert abs(X[k] - r2c(zk, zm, w ** k)) < 1e-11 * scale
        assert abs(X[nz - k] - r2c(zm, zk, -np.conj(w ** k))) < 1e-11 * scale
    assert abs(X[nz] - (Z[0].real - Z[0].imag)) < 1e-11 * scale


@pytest.mark.parametrize("nz", [32, 256, 1024])
def test_mode_z_convolution_by_spectral_pairs(nz):
    """The z convolution of one mode column as the warp kernel forms it, against
    its plain definition psi[k] = sum_{k' < nz} K(|k - k'|) rho[k'] (K real).

    Z is the nz-point DFT of the packed column z_m = rho_{2m} + i rho_{2m+1}
    (m < nz/2, zero beyond: Appendix A's padding), g the 2nz-point DFT of the
    doubled table K(0..nz), K(nz-1..1) divided by 2nz (real and even).  For each
    pair (k, nz - k), k <= nz/2, with X as in the test above,
      Y(k) = g(k) X(k),  Y(nz - k) = g(nz - k) X(nz - k),
      s = Y(k) + conj Y(nz - k),  t = conj(w^k) (Y(k) - conj Y(nz - k)),
      U(k) = s + i t,  U(nz - k) = conj(s) + i conj(t),
    and the unnormalised inverse p_m = sum_k U(k) e^{2 pi i k m / nz} gives
    psi_{2m} + i psi_{2m+1} = p_m for m < nz/2."""
    rng = np.random.default_rng(7 + nz)
    rho = rng.standard_normal(nz)
    K = rng.standard_normal(nz + 1)
    d = np.abs(np.arange(nz)[:, None] - np.arange(nz)[None, :])
    psi = (K[d] * rho[None, :]).sum(axis=1)
    G = np.fft.fft(np.concatenate([K, K[nz - 1:0:-1]]))
    assert np.abs(G.imag).max() < 1e-9 * np.abs(G).max()
    g = G.real / (2 * nz)
    z = np.zeros(nz, complex)
    z[: nz // 2] = rho[0::2] + 1j * rho[1::2]
    Z = np.fft.fft(z)
    w = np.exp(-1j * np.pi / nz)

    def unpack(x, xm, wk):
        c = np.conj(xm)
        return ((x + c) - 1j * wk * (x - c)) / 2

    U = np.zeros(nz, complex)
    for k in range(nz // 2 + 1):
        zk, zm, wk = Z[k % nz], Z[(nz - k) % nz], w ** k
        yk = g[k] * unpack(zk, zm, wk)
        ym = g[nz - k] * unpack(zm, zk, -np.conj(wk))
        s, t = yk + np.conj(ym), np.conj(wk) * (yk - np.conj(ym))
        U[k % nz] = s + 1j * t
        if 0 < k < nz // 2:
            U[nz - k] = np.conj(s) + 1j * np.conj(t)
    p = np.fft.ifft(U) * nz
    got = np.empty(nz)
    got[0::2], got[1::2] = p[: nz // 2].real, p[: nz // 2].imag
    assert np.abs(got - psi).max() < 1e-10 * np.abs(psi).max()
