// Electric field E = -grad phi on the mesh, the quantity a particle-in-cell
// step gathers after the solve.  The paper gives no discrete gradient; the
// one used is second-order central differences inside the mesh and
// second-order one-sided differences on its faces:
//     f'(0)   ~ (-3 f0 + 4 f1 - f2) / 2h,
//     f'(k)   ~ (f_{k+1} - f_{k-1}) / 2h,
//     f'(n-1) ~ (3 f_{n-1} - 4 f_{n-2} + f_{n-3}) / 2h.
// One thread per node, z (contiguous) fastest, so every stencil read of a
// warp is a contiguous run: phi is read from HBM about once (the neighbouring
// columns come from L2) and the three components are written once.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/pipe_poisson.h"
#include "handle.cuh"

namespace {

template <typename T>
__device__ __forceinline__ T d1(const T* f, long s, int k, int n, T inv2h) {
  if (k == 0) return (T(-3) * f[0] + T(4) * f[s] - f[2 * s]) * inv2h;
  if (k == n - 1) return (T(3) * f[0] - T(4) * f[-s] + f[-2 * s]) * inv2h;
  return (f[s] - f[-s]) * inv2h;
}

template <typename T>
__global__ void __launch_bounds__(256) field_kernel(const T* __restrict__ phi, T* __restrict__ E, int nx, int ny,
                                                    int nz, T ix, T iy, T iz) {
  const long nodes = long(nx) * ny * nz;
  const long idx = long(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= nodes) return;
  const int k = int(idx % nz);
  const int j = int((idx / nz) % ny);
  const int i = int(idx / (long(nz) * ny));
  const T* f = phi + idx;
  E[idx] = -d1(f, long(ny) * nz, i, nx, ix);
  E[nodes + idx] = -d1(f, long(nz), j, ny, iy);
  E[2 * nodes + idx] = -d1(f, 1L, k, nz, iz);
}

}  // namespace

extern "C" int pipe_electric_field(pipe_handle* h, const void* phi, void* E, void* stream) {
  if (!h || !phi || !E) return PIPE_EINVAL;
  if ((reinterpret_cast<uintptr_t>(phi) | reinterpret_cast<uintptr_t>(E)) % 16) return PIPE_EINVAL;
  const pipe_grid& g = h->grid;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return PIPE_ECUDA;
  if (prev != h->device && cudaSetDevice(h->device) != cudaSuccess) return PIPE_ECUDA;
  const long nodes = long(g.nx) * g.ny * g.nz;
  const unsigned blocks = unsigned((nodes + 255) / 256);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (g.dtype == PIPE_F64)
    field_kernel<double><<<blocks, 256, 0, st>>>(static_cast<const double*>(phi), static_cast<double*>(E), g.nx,
                                                 g.ny, g.nz, 0.5 / g.hx, 0.5 / g.hy, 0.5 / g.hz);
  else
    field_kernel<float><<<blocks, 256, 0, st>>>(static_cast<const float*>(phi), static_cast<float*>(E), g.nx, g.ny,
                                                g.nz, float(0.5 / g.hx), float(0.5 / g.hy), float(0.5 / g.hz));
  const cudaError_t e = cudaGetLastError();
  if (prev != h->device) cudaSetDevice(prev);
  return e == cudaSuccess ? PIPE_OK : PIPE_ECUDA;
}
