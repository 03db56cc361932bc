// Cloud-in-cell charge deposit and its adjoint with respect to the particle
// positions, on the solver's mesh x_i = x0 + i hx, y_j = y0 + j hy, z_k = k hz.
// Trilinear weights w = wx(x) wy(y) wz(z) with wx = 1 - |x - x_i|/hx on the two
// nodes bracketing x; nodes outside 0..n-1 are dropped.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/pipe_poisson.h"
#include "handle.cuh"

namespace {

struct Mesh {
  int nx, ny, nz;
  double x0, y0, hx, hy, hz;
};

template <typename T>
__device__ __forceinline__ void axis_weights(T x, T x0, T h, int n, int* i0, T* w0, T* w1, T* dw) {
  const T f = (x - x0) / h;
  const T fl = floor(f);
  *i0 = int(fl);
  const T d = f - fl;
  *w0 = T(1) - d;
  *w1 = d;
  *dw = T(1) / h;           // d w1/dx = +1/h, d w0/dx = -1/h
}

template <typename T>
__global__ void cic_deposit_kernel(const T* __restrict__ xyz, long n, T qh, T* rho, Mesh m) {
  const long p = long(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= n) return;
  int i0, j0, k0;
  T wx[2], wy[2], wz[2], d;
  axis_weights<T>(xyz[3 * p + 0], T(m.x0), T(m.hx), m.nx, &i0, &wx[0], &wx[1], &d);
  axis_weights<T>(xyz[3 * p + 1], T(m.y0), T(m.hy), m.ny, &j0, &wy[0], &wy[1], &d);
  axis_weights<T>(xyz[3 * p + 2], T(0), T(m.hz), m.nz, &k0, &wz[0], &wz[1], &d);
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const int i = i0 + a;
    if (i < 0 || i >= m.nx) continue;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int j = j0 + b;
      if (j < 0 || j >= m.ny) continue;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int k = k0 + c;
        if (k < 0 || k >= m.nz) continue;
        atomicAdd(&rho[(size_t(i) * m.ny + j) * m.nz + k], qh * wx[a] * wy[b] * wz[c]);
      }
    }
  }
}

template <typename T>
__global__ void cic_gather_grad_kernel(const T* __restrict__ xyz, long n, T qh,
                                       const T* __restrict__ g, T* __restrict__ out, Mesh m) {
  const long p = long(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= n) return;
  int i0, j0, k0;
  T wx[2], wy[2], wz[2], dx, dy, dz;
  axis_weights<T>(xyz[3 * p + 0], T(m.x0), T(m.hx), m.nx, &i0, &wx[0], &wx[1], &dx);
  axis_weights<T>(xyz[3 * p + 1], T(m.y0), T(m.hy), m.ny, &j0, &wy[0], &wy[1], &dy);
  axis_weights<T>(xyz[3 * p + 2], T(0), T(m.hz), m.nz, &k0, &wz[0], &wz[1], &dz);
  const T sx[2] = {-dx, dx}, sy[2] = {-dy, dy}, sz[2] = {-dz, dz};
  T gx = 0, gy = 0, gz = 0;
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const int i = i0 + a;
    if (i < 0 || i >= m.nx) continue;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int j = j0 + b;
      if (j < 0 || j >= m.ny) continue;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int k = k0 + c;
        if (k < 0 || k >= m.nz) continue;
        const T v = g[(size_t(i) * m.ny + j) * m.nz + k];
        gx += v * sx[a] * wy[b] * wz[c];
        gy += v * wx[a] * sy[b] * wz[c];
        gz += v * wx[a] * wy[b] * sz[c];
      }
    }
  }
  out[3 * p + 0] = qh * gx;
  out[3 * p + 1] = qh * gy;
  out[3 * p + 2] = qh * gz;
}

Mesh mesh_of(const pipe_handle* h) {
  Mesh m;
  m.nx = h->grid.nx; m.ny = h->grid.ny; m.nz = h->grid.nz;
  m.x0 = h->geom.x0; m.y0 = h->geom.y0;
  m.hx = h->grid.hx; m.hy = h->grid.hy; m.hz = h->grid.hz;
  return m;
}

}  // namespace

extern "C" int pipe_cic_deposit(pipe_handle* h, const void* xyz, int64_t n, double q, void* rho,
                                void* stream) {
  if (!h || !xyz || !rho || n < 0) return PIPE_EINVAL;
  if (n == 0) return PIPE_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const Mesh m = mesh_of(h);
  const double qh = q / (m.hx * m.hy * m.hz);
  const unsigned blocks = unsigned((n + 255) / 256);
  if (h->grid.dtype == PIPE_F64)
    cic_deposit_kernel<double><<<blocks, 256, 0, st>>>(static_cast<const double*>(xyz), n, qh,
                                                        static_cast<double*>(rho), m);
  else
    cic_deposit_kernel<float><<<blocks, 256, 0, st>>>(static_cast<const float*>(xyz), n, float(qh),
                                                       static_cast<float*>(rho), m);
  return cudaGetLastError() == cudaSuccess ? PIPE_OK : PIPE_ECUDA;
}

extern "C" int pipe_cic_gather_grad(pipe_handle* h, const void* xyz, int64_t n, double q,
                                    const void* grad_rho, void* grad_xyz, void* stream) {
  if (!h || !xyz || !grad_rho || !grad_xyz || n < 0) return PIPE_EINVAL;
  if (n == 0) return PIPE_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const Mesh m = mesh_of(h);
  const double qh = q / (m.hx * m.hy * m.hz);
  const unsigned blocks = unsigned((n + 255) / 256);
  if (h->grid.dtype == PIPE_F64)
    cic_gather_grad_kernel<double><<<blocks, 256, 0, st>>>(
        static_cast<const double*>(xyz), n, qh, static_cast<const double*>(grad_rho),
        static_cast<double*>(grad_xyz), m);
  else
    cic_gather_grad_kernel<float><<<blocks, 256, 0, st>>>(
        static_cast<const float*>(xyz), n, float(qh), static_cast<const float*>(grad_rho),
        static_cast<float*>(grad_xyz), m);
  return cudaGetLastError() == cudaSuccess ? PIPE_OK : PIPE_ECUDA;
}
