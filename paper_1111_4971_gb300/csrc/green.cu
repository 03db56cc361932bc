// Setup kernels, all FP64: twiddle tables, tabulation of the pipe Green
// function R / R_int (Sec. 2 Eq. 9, Sec. 3 Eq. 15-16) and of the free-space
// 1/r (Eq. 3) on the doubled grid, and their forward transforms.
//
// Layout of the tabulated tables: octant [r][q][p], p = 0..nx, q = 0..ny,
// r = 0..nz, holding R(p*hx, q*hy, r*hz).  The doubled-grid convolution table
// (Fig. 1, Appendix A Eq. A.3) is the even extension of this octant (R is even
// in each argument), and for a mesh that spans the pipe it is also the
// correlation table up to a shift of 2*x0/hx samples.  The forward transform
// of an even real table is real and even, so the transform of the whole
// doubled table reduces to a weighted cosine transform (DCT-I) along each axis
// of the octant:
//     That(k) = T(0) + (-1)^k T(n) + 2 sum_{p=1}^{n-1} T(p) cos(pi p k / n).
#include <cuda_runtime.h>

#include "fft_common.cuh"
#include "green_kernels.cuh"

namespace pp {

// tw[k1*G + t] = e^{-2 pi i t k1 / L}  (k1 < L/G, t < G);  w2[j] = e^{-2 pi i j / n2}
template <typename V>
__global__ void tables_kernel(V* tw, V* w2, int L, int G, int n2) {
  using R = typename real_of<V>::type;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < L) {
    const int k1 = idx / G, t = idx % G;
    const long m = (long(t) * k1) % L;
    double s, c;
    sincospi(2.0 * double(m) / double(L), &s, &c);
    tw[idx] = mk<V>(R(c), R(-s));
  }
  if (idx < n2) {
    double s, c;
    sincospi(2.0 * double(idx) / double(n2), &s, &c);
    w2[idx] = mk<V>(R(c), R(-s));
  }
}

template <typename V>
void launch_tables(V* tw, V* w2, int L, int G, int n2, cudaStream_t st) {
  const int n = L > n2 ? L : n2;
  tables_kernel<V><<<(n + 255) / 256, 256, 0, st>>>(tw, w2, L, G, n2);
}
template void launch_tables<float2>(float2*, float2*, int, int, int, cudaStream_t);
template void launch_tables<double2>(double2*, double2*, int, int, int, cudaStream_t);

// cos(m pi p h / a), m = 1..M, p = 0..n  -> tab[(m-1)*(n+1) + p]
__global__ void cos_table_kernel(double* tab, int M, int n, double h, double a) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * (n + 1)) return;
  const int m = idx / (n + 1) + 1, p = idx % (n + 1);
  tab[idx] = cospi(double(m) * double(p) * h / a);
}

// (x - 1 + e^{-x}) / x^2 without cancellation (Taylor series below 0.1)
__device__ double xm1pe_over_x2(double x) {
  if (x < 0.1) {
    double term = 0.5, acc = 0.5;
#pragma unroll 1
    for (int j = 1; j < 16; ++j) {
      term *= -x / double(j + 2);
      acc += term;
    }
    return acc;
  }
  return (x + expm1(-x)) / (x * x);
}

// Z[(m-1)*N + (n-1)][r] = kappa_mn^{-1} * Z_mn(r*hz), r = 0..nz, where Z is
// e^{-kappa |w|} (Eq. 9) or the longitudinal IGF g_z(w) (Eq. 15, evaluated in
// its cancellation-free form: 4 sinh^2(kappa h/2) e^{-kappa|w|}/(kappa h)^2 for
// |w| >= h, 2 (kappa h - 1 + e^{-kappa h})/(kappa h)^2 at w = 0).
__global__ void z_profile_kernel(double* Z, int M, int N, int nz, double hz, double a, double b,
                                 int igf) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * N * (nz + 1)) return;
  const int r = idx % (nz + 1);
  const int mn = idx / (nz + 1);
  const int m = mn / N + 1, n = mn % N + 1;
  const double km = double(m) / a, kn = double(n) / b;
  const double kap = M_PI * sqrt(km * km + kn * kn);
  const double w = double(r) * hz;
  double z;
  if (!igf) {
    z = exp(-kap * w);
  } else {
    const double x = kap * hz;
    if (r == 0) {
      z = 2.0 * xm1pe_over_x2(x);
    } else {
      const double s = sinh(0.5 * x);
      z = 4.0 * s * s * exp(-kap * w) / (x * x);
    }
  }
  Z[idx] = z / kap;
}

// U[m][q][r] = sum_n cy[n][q] Z[m][n][r]
__global__ void contract_n_kernel(double* U, const double* cy, const double* Z, int M, int N,
                                  int ny, int nz) {
  const long idx = long(blockIdx.x) * blockDim.x + threadIdx.x;
  const long total = long(M) * (ny + 1) * (nz + 1);
  if (idx >= total) return;
  const int r = int(idx % (nz + 1));
  const int q = int((idx / (nz + 1)) % (ny + 1));
  const int m = int(idx / (long(nz + 1) * (ny + 1)));
  double acc = 0.0;
#pragma unroll 4
  for (int n = 0; n < N; ++n) acc += cy[n * (ny + 1) + q] * Z[(long(m) * N + n) * (nz + 1) + r];
  U[idx] = acc;
}

// T[r][q][p] = C * sum_m cx[m][p] U[m][q][r]
__global__ void contract_m_kernel(double* T, const double* cx, const double* U, int M, int nx,
                                  int ny, int nz, double C) {
  const long idx = long(blockIdx.x) * blockDim.x + threadIdx.x;
  const long total = long(nx + 1) * (ny + 1) * (nz + 1);
  if (idx >= total) return;
  const int p = int(idx % (nx + 1));
  const int q = int((idx / (nx + 1)) % (ny + 1));
  const int r = int(idx / (long(nx + 1) * (ny + 1)));
  double acc = 0.0;
#pragma unroll 4
  for (int m = 0; m < M; ++m)
    acc += cx[m * (nx + 1) + p] * U[(long(m) * (ny + 1) + q) * (nz + 1) + r];
  T[idx] = C * acc;
}

// free space: T[r][q][p] = 1/sqrt((p hx)^2 + (q hy)^2 + (r hz)^2), T[0][0][0] = self
__global__ void free_octant_kernel(double* T, int nx, int ny, int nz, double hx, double hy,
                                   double hz, double self) {
  const long idx = long(blockIdx.x) * blockDim.x + threadIdx.x;
  const long total = long(nx + 1) * (ny + 1) * (nz + 1);
  if (idx >= total) return;
  const int p = int(idx % (nx + 1));
  const int q = int((idx / (nx + 1)) % (ny + 1));
  const int r = int(idx / (long(nx + 1) * (ny + 1)));
  const double u = p * hx, v = q * hy, w = r * hz;
  T[idx] = (p == 0 && q == 0 && r == 0) ? self : rsqrt(u * u + v * v + w * w);
}

__global__ void cos_pi_table_kernel(double* c, int n) {   // c[j] = cos(pi j / n), j < 2n
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < 2 * n) c[j] = cospi(double(j) / double(n));
}

// Weighted cosine transform along one axis, batched:
//   out[b*bs + k*ks + l*ls] = sum_{p=0}^{n} w_p cos(pi p k/n) in[b*bs + p*ks + l*ls]
// w_0 = w_n = 1, otherwise 2; k = 0..n, l < nl, b < nb.  64x64 output tiles,
// 16-deep slices of p in shared memory, 4x4 outputs per thread.
__global__ void __launch_bounds__(256) dct1_axis_kernel(const double* __restrict__ in,
                                                        double* __restrict__ out, int n, int nl,
                                                        long ks, long ls, long bs,
                                                        const double* __restrict__ cosn) {
  __shared__ double Ws[16][65];
  __shared__ double Xs[16][65];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int k0 = blockIdx.y * 64, l0 = blockIdx.x * 64;
  const long boff = long(blockIdx.z) * bs;
  double acc[4][4] = {};
  const bool p_fast = (ks == 1);
  for (int p0 = 0; p0 <= n; p0 += 16) {
    for (int idx = threadIdx.x; idx < 16 * 64; idx += 256) {
      int pp, ll;
      if (p_fast) { pp = idx % 16; ll = idx / 16; } else { pp = idx / 64; ll = idx % 64; }
      const int p = p0 + pp, l = l0 + ll;
      Xs[pp][ll] = (p <= n && l < nl) ? in[boff + p * ks + l * ls] : 0.0;
      const int kk = idx % 64, pq = idx / 64;
      const int pk = p0 + pq, k = k0 + kk;
      double wv = 0.0;
      if (pk <= n && k <= n) {
        const double wp = (pk == 0 || pk == n) ? 1.0 : 2.0;
        wv = wp * cosn[(long(pk) * k) % (2 * n)];
      }
      Ws[pq][kk] = wv;
    }
    __syncthreads();
#pragma unroll
    for (int pp = 0; pp < 16; ++pp) {
      double av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = Ws[pp][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Xs[pp][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int k = k0 + ty + 16 * i;
    if (k > n) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int l = l0 + tx + 16 * j;
      if (l < nl) out[boff + k * ks + l * ls] = acc[i][j];
    }
  }
}

__global__ void finalize_kernel(const double* T, double* g64, float* g32, long total, double scale) {
  const long idx = long(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const double v = T[idx] * scale;
  g64[idx] = v;
  g32[idx] = float(v);
}

static inline unsigned nblk(long total, int bs) { return unsigned((total + bs - 1) / bs); }

// Forward transform of an even real octant table T (in place through `tmp`):
// DCT-I along x (p), then y (q), then z (r).  Result in T.
static cudaError_t octant_transform(double* T, double* tmp, double* cosbuf, int nx, int ny, int nz,
                                    cudaStream_t st, bool transform_z = true) {
  const long sx = 1, sy = nx + 1, sz = long(nx + 1) * (ny + 1);
  // x axis: lines = q (stride sy), batches = r (stride sz)
  cos_pi_table_kernel<<<nblk(2 * nx, 256), 256, 0, st>>>(cosbuf, nx);
  {
    dim3 grid(nblk(ny + 1, 64), nblk(nx + 1, 64), nz + 1);
    dct1_axis_kernel<<<grid, 256, 0, st>>>(T, tmp, nx, ny + 1, sx, sy, sz, cosbuf);
  }
  // y axis: lines = p (stride 1), batches = r
  cos_pi_table_kernel<<<nblk(2 * ny, 256), 256, 0, st>>>(cosbuf, ny);
  {
    dim3 grid(nblk(nx + 1, 64), nblk(ny + 1, 64), nz + 1);
    dct1_axis_kernel<<<grid, 256, 0, st>>>(tmp, T, ny, nx + 1, sy, 1, sz, cosbuf);
  }
  if (!transform_z) return cudaGetLastError();               // result in T
  // z axis: lines = (q, p) flattened (stride 1), one batch
  cos_pi_table_kernel<<<nblk(2 * nz, 256), 256, 0, st>>>(cosbuf, nz);
  {
    dim3 grid(nblk(sz, 64), nblk(nz + 1, 64), 1);
    dct1_axis_kernel<<<grid, 256, 0, st>>>(T, tmp, nz, int(sz), sz, 1, 0, cosbuf);
  }
  return cudaMemcpyAsync(T, tmp, sizeof(double) * sz * (nz + 1), cudaMemcpyDeviceToDevice, st);
}

cudaError_t build_pipe_spectrum_from_modes(const GreenSpec& s, double* g64, float* g32, cudaStream_t st,
                                           bool transform_z);
__global__ void z_dct_kernel(double* Zh, const double* Z, int MN, int nz, const double* cosn);

// The octant's x-y transform straight from the modes.  The table is
// T[r][q][p] = C sum_mn cos(pi m p / nx) cos(pi n q / ny) Z_mn(r) (a mesh that
// spans the pipe: nx hx = a), and the weighted DCT-I of cos(pi m p / n) over
// p = 0..n is n delta(k - m'), m' the alias of m in [0, n] (m mod 2n, or
// 2n - (m mod 2n) above n), 2n delta at the end points k = 0 and k = n.  So
//   T^[r][ky][kx] = C sum over the modes m aliasing to kx and n aliasing to ky
//                   of dx dy Zs[m][n][r],
// Zs the z profiles (banded tables) or their DCT-I along z (full solve).
// Candidates for k: m = k + 2nj (j >= 0) and m = 2nj - k (j >= 1; the same
// modes again when k = 0 or n).
__global__ void octant_from_modes_kernel(double* T, const double* Zs, int M, int N, int nx, int ny, int nz,
                                         double C) {
  const long idx = long(blockIdx.x) * blockDim.x + threadIdx.x;
  const long total = long(nx + 1) * (ny + 1) * (nz + 1);
  if (idx >= total) return;
  const int p = int(idx % (nx + 1));
  const int q = int((idx / (nx + 1)) % (ny + 1));
  const int r = int(idx / (long(nx + 1) * (ny + 1)));
  const double dx = (p == 0 || p == nx) ? 2.0 * nx : double(nx);
  const double dy = (q == 0 || q == ny) ? 2.0 * ny : double(ny);
  double acc = 0.0;
#pragma unroll 1
  for (int fm = 0; fm < 2; ++fm) {
    if (fm == 1 && (p == 0 || p == nx)) break;
#pragma unroll 1
    for (int m = fm == 0 ? p : 2 * nx - p; m <= M; m += 2 * nx) {
      if (m < 1) continue;
#pragma unroll 1
      for (int fn = 0; fn < 2; ++fn) {
        if (fn == 1 && (q == 0 || q == ny)) break;
#pragma unroll 1
        for (int n = fn == 0 ? q : 2 * ny - q; n <= N; n += 2 * ny) {
          if (n < 1) continue;
          acc += Zs[(long(m - 1) * N + (n - 1)) * (nz + 1) + r];
        }
      }
    }
  }
  T[idx] = C * dx * dy * acc;
}

cudaError_t build_pipe_spectrum(const GreenSpec& s, double* g64, float* g32, cudaStream_t st,
                                bool transform_z) {
  if (s.modes_m <= 64 && s.modes_n <= 64) return build_pipe_spectrum_from_modes(s, g64, g32, st, transform_z);
  const int nx = s.nx, ny = s.ny, nz = s.nz, M = s.modes_m, N = s.modes_n;
  const long oct = long(nx + 1) * (ny + 1) * (nz + 1);
  double *cx = nullptr, *cy = nullptr, *Z = nullptr, *U = nullptr, *T = nullptr, *tmp = nullptr,
         *cosbuf = nullptr;
  cudaError_t err = cudaSuccess;
  const size_t szU = sizeof(double) * size_t(M) * (ny + 1) * (nz + 1);
  if ((err = cudaMalloc(&cx, sizeof(double) * M * (nx + 1))) != cudaSuccess) goto done;
  if ((err = cudaMalloc(&cy, sizeof(double) * N * (ny + 1))) != cudaSuccess) goto done;
  if ((err = cudaMalloc(&Z, sizeof(double) * size_t(M) * N * (nz + 1))) != cudaSuccess) goto done;
  if ((err = cudaMalloc(&U, szU)) != cudaSuccess) goto done;
  if ((err = cudaMalloc(&T, sizeof(double) * oct)) != cudaSuccess) goto done;
  if ((err = cudaMalloc(&tmp, sizeof(double) * oct)) != cudaSuccess) goto done;
  if ((err = cudaMalloc(&cosbuf, sizeof(double) * 2 * (nz > nx ? (nz > ny ? nz : ny) : (nx > ny ? nx : ny))))
      != cudaSuccess) goto done;
  cos_table_kernel<<<nblk(M * (nx + 1), 256), 256, 0, st>>>(cx, M, nx, s.hx, s.a);
  cos_table_kernel<<<nblk(N * (ny + 1), 256), 256, 0, st>>>(cy, N, ny, s.hy, s.b);
  z_profile_kernel<<<nblk(long(M) * N * (nz + 1), 256), 256, 0, st>>>(Z, M, N, nz, s.hz, s.a, s.b,
                                                                     s.igf);
  contract_n_kernel<<<nblk(long(M) * (ny + 1) * (nz + 1), 256), 256, 0, st>>>(U, cy, Z, M, N, ny, nz);
  contract_m_kernel<<<nblk(oct, 256), 256, 0, st>>>(T, cx, U, M, nx, ny, nz,
                                                    2.0 * M_PI / (s.a * s.b));
  if ((err = cudaGetLastError()) != cudaSuccess) goto done;
  if ((err = octant_transform(T, tmp, cosbuf, nx, ny, nz, st, transform_z)) != cudaSuccess) goto done;
  finalize_kernel<<<nblk(oct, 256), 256, 0, st>>>(T, g64, g32, oct, s.scale);
  if ((err = cudaGetLastError()) != cudaSuccess) goto done;
  err = cudaStreamSynchronize(st);
done:
  cudaFree(cx); cudaFree(cy); cudaFree(Z); cudaFree(U); cudaFree(T); cudaFree(tmp); cudaFree(cosbuf);
  return err;
}

// build_pipe_spectrum for up to 64 modes per axis: z profiles, their DCT-I
// along z per mode (full solve), the octant gathered from the modes, scaled.
cudaError_t build_pipe_spectrum_from_modes(const GreenSpec& s, double* g64, float* g32, cudaStream_t st,
                                           bool transform_z) {
  const int nx = s.nx, ny = s.ny, nz = s.nz, M = s.modes_m, N = s.modes_n;
  const long oct = long(nx + 1) * (ny + 1) * (nz + 1);
  double *Z = nullptr, *Zh = nullptr, *T = nullptr, *cosn = nullptr;
  cudaError_t err = cudaSuccess;
  if ((err = cudaMalloc(&Z, sizeof(double) * size_t(M) * N * (nz + 1))) != cudaSuccess) goto done;
  if ((err = cudaMalloc(&T, sizeof(double) * oct)) != cudaSuccess) goto done;
  z_profile_kernel<<<nblk(long(M) * N * (nz + 1), 256), 256, 0, st>>>(Z, M, N, nz, s.hz, s.a, s.b, s.igf);
  if (transform_z) {
    if ((err = cudaMalloc(&Zh, sizeof(double) * size_t(M) * N * (nz + 1))) != cudaSuccess) goto done;
    if ((err = cudaMalloc(&cosn, sizeof(double) * 2 * nz)) != cudaSuccess) goto done;
    cos_pi_table_kernel<<<nblk(2 * nz, 256), 256, 0, st>>>(cosn, nz);
    z_dct_kernel<<<nblk(long(M) * N * (nz + 1), 256), 256, 0, st>>>(Zh, Z, M * N, nz, cosn);
  }
  octant_from_modes_kernel<<<nblk(oct, 256), 256, 0, st>>>(T, transform_z ? Zh : Z, M, N, nx, ny, nz,
                                                           2.0 * M_PI / (s.a * s.b));
  finalize_kernel<<<nblk(oct, 256), 256, 0, st>>>(T, g64, g32, oct, s.scale);
  if ((err = cudaGetLastError()) != cudaSuccess) goto done;
  err = cudaStreamSynchronize(st);
done:
  cudaFree(Z); cudaFree(Zh); cudaFree(T); cudaFree(cosn);
  return err;
}

cudaError_t build_free_spectrum(const GreenSpec& s, double self_value, double* g64, float* g32,
                                cudaStream_t st) {
  const int nx = s.nx, ny = s.ny, nz = s.nz;
  const long oct = long(nx + 1) * (ny + 1) * (nz + 1);
  double *T = nullptr, *tmp = nullptr, *cosbuf = nullptr;
  cudaError_t err = cudaSuccess;
  const int nmax = nz > nx ? (nz > ny ? nz : ny) : (nx > ny ? nx : ny);
  if ((err = cudaMalloc(&T, sizeof(double) * oct)) != cudaSuccess) goto done;
  if ((err = cudaMalloc(&tmp, sizeof(double) * oct)) != cudaSuccess) goto done;
  if ((err = cudaMalloc(&cosbuf, sizeof(double) * 2 * nmax)) != cudaSuccess) goto done;
  free_octant_kernel<<<nblk(oct, 256), 256, 0, st>>>(T, nx, ny, nz, s.hx, s.hy, s.hz, self_value);
  if ((err = cudaGetLastError()) != cudaSuccess) goto done;
  if ((err = octant_transform(T, tmp, cosbuf, nx, ny, nz, st)) != cudaSuccess) goto done;
  finalize_kernel<<<nblk(oct, 256), 256, 0, st>>>(T, g64, g32, oct, s.scale);
  if ((err = cudaGetLastError()) != cudaSuccess) goto done;
  err = cudaStreamSynchronize(st);
done:
  cudaFree(T); cudaFree(tmp); cudaFree(cosbuf);
  return err;
}

// ---------------------------------------------------------------------------
// General meshes (a transverse window, Sec. 5: the mesh need not span the pipe
// nor sit at integer correlation shifts).  The four tables of Eq. 10 on the
// doubled grid,
//     T_xy(p, q, r) = C sum_mn c^x_m(p) c^y_n(q) Z_mn(r),   x, y in {conv, corr},
// with c^conv_m(p) = cos(m pi o(p) / a), o(p) = p h (p <= n), (p - 2n) h (p > n),
// c^corr_m(p) = cos(m pi (2 x0 + p h) / a), p = 0..2n-1, and the z profile Z_mn
// (even in r), are separable per mode, so their forward transforms are
//     T^_xy(kx, ky, kz) = C sum_m C^x_m(kx) sum_n C^y_n(ky) Z^_mn(kz)
// with C^ the 2n-point forward DFTs of the cosine factors and Z^ the DCT-I of
// the z profile.  All FP64; stored [t][kz][ky][kx] complex (t = cc, cr, rc,
// rr), scaled like the octant.
// ---------------------------------------------------------------------------

// out[m][k] = sum_p c_m(p) e^{-2 pi i p k / (2n)}, c from offsets (conv or corr)
__global__ void cos_factor_dft_kernel(double2* out, int M, int n, double h, double a, double origin,
                                      int corr) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int L = 2 * n;
  if (idx >= M * L) return;
  const int m = idx / L + 1, k = idx % L;
  double re = 0.0, im = 0.0;
  for (int p = 0; p < L; ++p) {
    const double o = corr ? 2.0 * origin + double(p) * h : double(p <= n ? p : p - L) * h;
    const double c = cospi(double(m) * o / a);
    double sn, cs;
    sincospi(2.0 * double((long(p) * k) % L) / double(L), &sn, &cs);
    re += c * cs;
    im -= c * sn;
  }
  out[idx] = make_double2(re, im);
}

// Zh[mn][kz] = Z(0) + (-1)^kz Z(nz) + 2 sum_{r=1}^{nz-1} Z(r) cos(pi r kz / nz)
__global__ void z_dct_kernel(double* Zh, const double* Z, int MN, int nz, const double* cosn) {
  const long idx = long(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= long(MN) * (nz + 1)) return;
  const int kz = int(idx % (nz + 1));
  const double* z = Z + (idx / (nz + 1)) * (nz + 1);
  double acc = z[0] + ((kz & 1) ? -z[nz] : z[nz]);
  for (int r = 1; r < nz; ++r) acc += 2.0 * z[r] * cosn[(long(r) * kz) % (2 * nz)];
  Zh[idx] = acc;
}

// W[m][ky][kz] = sum_n Cy[n][ky] Zh[m][n][kz]
__global__ void general_contract_n_kernel(double2* W, const double2* Cy, const double* Zh, int M, int N,
                                          int L, int nz) {
  const long idx = long(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= long(M) * L * (nz + 1)) return;
  const int kz = int(idx % (nz + 1));
  const int ky = int((idx / (nz + 1)) % L);
  const int m = int(idx / (long(nz + 1) * L));
  double re = 0.0, im = 0.0;
  for (int n = 0; n < N; ++n) {
    const double2 c = Cy[n * L + ky];
    const double z = Zh[(long(m) * N + n) * (nz + 1) + kz];
    re += c.x * z;
    im += c.y * z;
  }
  W[idx] = make_double2(re, im);
}

// T[kz][ky][kx] = C sum_m Cx[m][kx] W[m][ky][kz]  (complex product), FP64 and FP32 copies
__global__ void general_contract_m_kernel(double2* T64, float2* T32, const double2* Cx, const double2* W, int M,
                                          int Lx, int Ly, int nz, double C) {
  const long idx = long(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= long(nz + 1) * Ly * Lx) return;
  const int kx = int(idx % Lx);
  const int ky = int((idx / Lx) % Ly);
  const int kz = int(idx / (long(Lx) * Ly));
  double re = 0.0, im = 0.0;
  for (int m = 0; m < M; ++m) {
    const double2 c = Cx[m * Lx + kx];
    const double2 w = W[(long(m) * Ly + ky) * (nz + 1) + kz];
    re += c.x * w.x - c.y * w.y;
    im += c.x * w.y + c.y * w.x;
  }
  T64[idx] = make_double2(C * re, C * im);
  T32[idx] = make_float2(float(C * re), float(C * im));
}

cudaError_t build_general_spectra(const GreenSpec& s, double x0, double y0, double2* t64, float2* t32,
                                  cudaStream_t st) {
  const int nx = s.nx, ny = s.ny, nz = s.nz, M = s.modes_m, N = s.modes_n;
  const int Lx = 2 * nx, Ly = 2 * ny;
  const long plane = long(nz + 1) * Ly * Lx;
  double2 *cx[2] = {nullptr, nullptr}, *cy[2] = {nullptr, nullptr}, *W[2] = {nullptr, nullptr};
  double *Z = nullptr, *Zh = nullptr, *cosn = nullptr;
  cudaError_t err = cudaSuccess;
  for (int k = 0; k < 2; ++k) {
    if ((err = cudaMalloc(&cx[k], sizeof(double2) * M * Lx)) != cudaSuccess) goto done;
    if ((err = cudaMalloc(&cy[k], sizeof(double2) * N * Ly)) != cudaSuccess) goto done;
    if ((err = cudaMalloc(&W[k], sizeof(double2) * size_t(M) * Ly * (nz + 1))) != cudaSuccess) goto done;
  }
  if ((err = cudaMalloc(&Z, sizeof(double) * size_t(M) * N * (nz + 1))) != cudaSuccess) goto done;
  if ((err = cudaMalloc(&Zh, sizeof(double) * size_t(M) * N * (nz + 1))) != cudaSuccess) goto done;
  if ((err = cudaMalloc(&cosn, sizeof(double) * 2 * nz)) != cudaSuccess) goto done;
  for (int k = 0; k < 2; ++k) {                     // k = 0 convolution, 1 correlation
    cos_factor_dft_kernel<<<nblk(long(M) * Lx, 256), 256, 0, st>>>(cx[k], M, nx, s.hx, s.a, x0, k);
    cos_factor_dft_kernel<<<nblk(long(N) * Ly, 256), 256, 0, st>>>(cy[k], N, ny, s.hy, s.b, y0, k);
  }
  z_profile_kernel<<<nblk(long(M) * N * (nz + 1), 256), 256, 0, st>>>(Z, M, N, nz, s.hz, s.a, s.b, s.igf);
  cos_pi_table_kernel<<<nblk(2 * nz, 256), 256, 0, st>>>(cosn, nz);
  z_dct_kernel<<<nblk(long(M) * N * (nz + 1), 256), 256, 0, st>>>(Zh, Z, M * N, nz, cosn);
  for (int k = 0; k < 2; ++k)
    general_contract_n_kernel<<<nblk(long(M) * Ly * (nz + 1), 256), 256, 0, st>>>(W[k], cy[k], Zh, M, N, Ly, nz);
  // t = 2 * (x kind) + (y kind): cc, cr, rc, rr
  for (int t = 0; t < 4; ++t)
    general_contract_m_kernel<<<nblk(plane, 256), 256, 0, st>>>(t64 + t * plane, t32 + t * plane, cx[t >> 1],
                                                                W[t & 1], M, Lx, Ly, nz,
                                                                2.0 * M_PI / (s.a * s.b) * s.scale);
  if ((err = cudaGetLastError()) != cudaSuccess) goto done;
  err = cudaStreamSynchronize(st);
done:
  for (int k = 0; k < 2; ++k) { cudaFree(cx[k]); cudaFree(cy[k]); cudaFree(W[k]); }
  cudaFree(Z); cudaFree(Zh); cudaFree(cosn);
  return err;
}


// ---------------------------------------------------------------------------
// Tables of the mode-space solve (modes_impl.cuh), all FP64 with FP32 copies:
//   sx[i][s] = sin(m pi x_i / a), m = s + 1 (zero for m > Mx), i < nx, s < mxp
//   sy[j][s] = sin(n pi y_j / b) for the mode n of slot s (mode_of_slot), j < nyk
//   gz[c][kz], c = s_x * myp + s_y: the DCT-I of the doubled z table of
//       K_mn(d) = hx hy hz (8 pi / ab) kappa_mn^{-1} f_mn(d hz)
//   (f the e^{-kappa |w|} of Eq. 9 or the IGF g_z of Eq. 15), divided by 2nz.
// ---------------------------------------------------------------------------
__global__ void mode_sine_kernel(double* t64, float* t32, int rows, int slots, int nmodes, int fold,
                                 double origin, double h, double len) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * slots) return;
  const int r = idx / slots, s = idx % slots;
  const int mode = !fold ? s + 1 : (s < slots / 2 ? 2 * s + 1 : 2 * (s - slots / 2) + 2);
  const double v = mode <= nmodes ? sinpi(double(mode) * (origin + double(r) * h) / len) : 0.0;
  t64[idx] = v;
  t32[idx] = float(v);
}

__global__ void mode_gz_kernel(double* g64, float* g32, const double* Zh, int M, int N, int mxp, int myp,
                               int fold, int nz, double C) {
  const long idx = long(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= long(mxp) * myp * (nz + 1)) return;
  const int kz = int(idx % (nz + 1));
  const int c = int(idx / (nz + 1));
  const int m = c / myp + 1, s = c % myp;
  const int n = !fold ? s + 1 : (s < myp / 2 ? 2 * s + 1 : 2 * (s - myp / 2) + 2);
  const double v = (m <= M && n <= N) ? C * Zh[(long(m - 1) * N + (n - 1)) * (nz + 1) + kz] : 0.0;
  g64[idx] = v;
  g32[idx] = float(v);
}

// kb[c][d] = hx hy hz (8 pi / ab) kappa^{-1} f_mn(d hz), d = 0..nb, c = (m-1) myp + slot(n):
// the real-space z kernel of the banded operator in the mode slots
__global__ void mode_kb_kernel(double* k64, float* k32, const double* Z, int M, int N, int mxp, int myp,
                               int fold, int nb, double C) {
  const long idx = long(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= long(mxp) * myp * (nb + 1)) return;
  const int d = int(idx % (nb + 1));
  const int c = int(idx / (nb + 1));
  const int m = c / myp + 1, s = c % myp;
  const int n = !fold ? s + 1 : (s < myp / 2 ? 2 * s + 1 : 2 * (s - myp / 2) + 2);
  const double v = (m <= M && n <= N) ? C * Z[(long(m - 1) * N + (n - 1)) * (nb + 1) + d] : 0.0;
  k64[idx] = v;
  k32[idx] = float(v);
}

cudaError_t build_mode_band(const GreenSpec& s, int mxp, int myp, int fold, int nb, double* kb64, float* kb32,
                            cudaStream_t st) {
  const int M = s.modes_m, N = s.modes_n;
  double* Z = nullptr;
  cudaError_t err = cudaMalloc(&Z, sizeof(double) * size_t(M) * N * (nb + 1));
  if (err != cudaSuccess) return err;
  z_profile_kernel<<<nblk(long(M) * N * (nb + 1), 256), 256, 0, st>>>(Z, M, N, nb, s.hz, s.a, s.b, s.igf);
  mode_kb_kernel<<<nblk(long(mxp) * myp * (nb + 1), 256), 256, 0, st>>>(
      kb64, kb32, Z, M, N, mxp, myp, fold, nb, s.hx * s.hy * s.hz * 8.0 * M_PI / (s.a * s.b));
  if ((err = cudaGetLastError()) == cudaSuccess) err = cudaStreamSynchronize(st);
  cudaFree(Z);
  return err;
}

cudaError_t build_mode_tables(const GreenSpec& s, double x0, double y0, int mxp, int myp, int fold,
                              double* sx64, float* sx32, double* sy64, float* sy32, double* gz64,
                              float* gz32, cudaStream_t st) {
  const int M = s.modes_m, N = s.modes_n, nz = s.nz;
  const int nyk = fold ? s.ny / 2 : s.ny;
  double *Z = nullptr, *Zh = nullptr, *cosn = nullptr;
  cudaError_t err = cudaSuccess;
  if ((err = cudaMalloc(&Z, sizeof(double) * size_t(M) * N * (nz + 1))) != cudaSuccess) goto done;
  if ((err = cudaMalloc(&Zh, sizeof(double) * size_t(M) * N * (nz + 1))) != cudaSuccess) goto done;
  if ((err = cudaMalloc(&cosn, sizeof(double) * 2 * nz)) != cudaSuccess) goto done;
  mode_sine_kernel<<<nblk(long(s.nx) * mxp, 256), 256, 0, st>>>(sx64, sx32, s.nx, mxp, M, 0, x0, s.hx, s.a);
  mode_sine_kernel<<<nblk(long(nyk) * myp, 256), 256, 0, st>>>(sy64, sy32, nyk, myp, N, fold, y0, s.hy, s.b);
  z_profile_kernel<<<nblk(long(M) * N * (nz + 1), 256), 256, 0, st>>>(Z, M, N, nz, s.hz, s.a, s.b, s.igf);
  cos_pi_table_kernel<<<nblk(2 * nz, 256), 256, 0, st>>>(cosn, nz);
  z_dct_kernel<<<nblk(long(M) * N * (nz + 1), 256), 256, 0, st>>>(Zh, Z, M * N, nz, cosn);
  mode_gz_kernel<<<nblk(long(mxp) * myp * (nz + 1), 256), 256, 0, st>>>(
      gz64, gz32, Zh, M, N, mxp, myp, fold, nz, s.hx * s.hy * s.hz * 8.0 * M_PI / (s.a * s.b) / (2.0 * nz));
  if ((err = cudaGetLastError()) != cudaSuccess) goto done;
  err = cudaStreamSynchronize(st);
done:
  cudaFree(Z); cudaFree(Zh); cudaFree(cosn);
  return err;
}

}  // namespace pp
