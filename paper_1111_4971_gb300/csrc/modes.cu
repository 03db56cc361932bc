// Kernels and host launchers of the mode-space solve (the method and the
// device routines are described in modes_impl.cuh).
#include <type_traits>

#include "modes.cuh"
#include "modes_impl.cuh"

namespace pp {

template <typename T, int MYP, bool FY>
__global__ void __launch_bounds__(128) mode_project_kernel(ModeArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  mode_project<T, MYP, FY>(a, smem_raw);
}

template <typename T, int MYP, bool FY>
__global__ void __launch_bounds__(128) mode_back_kernel(ModeArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  mode_back<T, MYP, FY>(a, smem_raw);
}

template <typename T>
__global__ void __launch_bounds__(256) mode_z_kernel(ModeArgs<T> a, int groups) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  mode_z<T>(a, groups, smem_raw);
}

// Banded z stage (Sec. 5, Eq. 17-18 in mode space): psi[c][k] =
// sum_{|d| <= nb, 0 <= k-d < nz} K_c(|d|) rhot[c][k-d], rhot the groups' partial
// projections summed.  One CTA per column: the column (zero-padded by nb on
// both sides) and its taps in shared memory, taps summed from d = -nb up.
constexpr int kBandThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kBandThreads) mode_band_kernel(ModeArgs<T> a, int groups) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* win = reinterpret_cast<T*>(smem_raw);           // [nz + 2 nb]: win[nb + k] = rhot[k]
  T* taps = win + a.nz + 2 * a.nb;                   // [nb + 1]
  const int c = int(blockIdx.x);
  for (int i = int(threadIdx.x); i < a.nb; i += kBandThreads) win[i] = win[a.nb + a.nz + i] = T(0);
  // the column summed over the groups (in group order, from zero), 16 bytes a
  // load, every group's load of a piece in flight together (nz is a power of
  // two >= 32, so the pieces tile it and stay 16-byte aligned)
  using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  constexpr int EV = 16 / sizeof(T);
  for (int q = int(threadIdx.x); q < a.nz / EV; q += kBandThreads) {
    T v[EV];
#pragma unroll
    for (int e = 0; e < EV; ++e) v[e] = T(0);
#pragma unroll 4
    for (int s = 0; s < groups; ++s) {
      const V p = __ldg(reinterpret_cast<const V*>(a.part + (size_t(s) * a.mc + c) * a.nz) + q);
      const T* pe = reinterpret_cast<const T*>(&p);
#pragma unroll
      for (int e = 0; e < EV; ++e) v[e] += pe[e];
    }
#pragma unroll
    for (int e = 0; e < EV; ++e) win[a.nb + q * EV + e] = v[e];
  }
  for (int d = int(threadIdx.x); d <= a.nb; d += kBandThreads) taps[d] = a.kb[size_t(c) * (a.nb + 1) + d];
  __syncthreads();
  for (int k = int(threadIdx.x); k < a.nz; k += kBandThreads) {
    const T* w = win + k + a.nb;                     // w[-d] = rhot[k - d]
    T acc = T(0);
    for (int d = -a.nb; d <= a.nb; ++d) acc += taps[d < 0 ? -d : d] * w[-d];
    a.psi[size_t(c) * a.nz + k] = acc;
  }
}

namespace {

template <typename T>
cudaError_t launch_band(const ModeArgs<T>& a, cudaStream_t st) {
  const int xblocks = a.nx / ModeShape<T>::XB;
  const size_t smem = sizeof(T) * (size_t(a.nz) + 3 * size_t(a.nb) + 1);
  void (*kern)(ModeArgs<T>, int) = mode_band_kernel<T>;
  if (smem > 48 * 1024) {
    if (smem > kMaxSmem) return cudaErrorInvalidConfiguration;
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
  }
  kern<<<unsigned(a.mc), kBandThreads, smem, st>>>(a, xblocks / mode_cluster(xblocks));
  return cudaGetLastError();
}

template <typename K>
cudaError_t set_smem(K kern, size_t smem) {
  if (smem > kMaxSmem) return cudaErrorInvalidConfiguration;
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
}

template <typename T, int MYP, bool FY>
cudaError_t launch_pb(int which, const ModeArgs<T>& a, cudaStream_t st) {
  using S = ModeShape<T>;
  const int xblocks = a.nx / S::XB;
  const dim3 grid(unsigned(a.nz / S::ZC), unsigned(xblocks));
  cudaError_t e;
  if (which == 0) {
    const size_t smem = mode_proj_smem<T>(a.ny, a.mxp, MYP, FY);
    void (*kern)(ModeArgs<T>) = mode_project_kernel<T, MYP, FY>;
    if ((e = set_smem(kern, smem)) != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(S::THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = unsigned(mode_cluster(xblocks));
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
  }
  const size_t smem = mode_back_smem<T>(a.ny, a.mx, a.mxp, MYP, FY);
  void (*kern)(ModeArgs<T>) = mode_back_kernel<T, MYP, FY>;
  if ((e = set_smem(kern, smem)) != cudaSuccess) return e;
  kern<<<grid, S::THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename T, int MYP>
cudaError_t launch_pb2(int which, bool fy, const ModeArgs<T>& a, cudaStream_t st) {
  return fy ? launch_pb<T, MYP, true>(which, a, st) : launch_pb<T, MYP, false>(which, a, st);
}

// 256 threads per CTA, L/4 per column (L = nz in 32..1024)
template <typename T>
cudaError_t launch_zc(const ModeArgs<T>& a, cudaStream_t st) {
  const int xblocks = a.nx / ModeShape<T>::XB;
  if constexpr (sizeof(T) == 4) return launch_mode_z_warp(a, xblocks / mode_cluster(xblocks), st);
  const int per = 1024 / a.nz;                       // columns per CTA
  const size_t smem = sizeof(C2<T>) * (size_t(per) * 2 * a.nz + 3 * size_t(a.nz));
  void (*kern)(ModeArgs<T>, int) = mode_z_kernel<T>;
  cudaError_t e;
  if ((e = set_smem(kern, smem)) != cudaSuccess) return e;
  kern<<<(a.mc + per - 1) / per, 256, smem, st>>>(a, xblocks / mode_cluster(xblocks));
  return cudaGetLastError();
}

}  // namespace

#ifndef PP_M_TYPE
#define PP_M_TYPE float
#endif

template <>
cudaError_t launch_mode_stage<PP_M_TYPE>(int stage, int myp, bool fy, const ModeArgs<PP_M_TYPE>& a,
                                         cudaStream_t st) {
  using T = PP_M_TYPE;
  if (stage == 1) {
    if (a.nz < 32 || a.nz > 1024 || (a.nz & (a.nz - 1))) return cudaErrorInvalidValue;
    if (a.nb >= 0) return launch_band<T>(a, st);
    return launch_zc<T>(a, st);
  }
  const int which = stage == 0 ? 0 : 1;
  switch (myp) {
    case 8: return launch_pb2<T, 8>(which, fy, a, st);
    case 12: return launch_pb2<T, 12>(which, fy, a, st);
    case 16: return launch_pb2<T, 16>(which, fy, a, st);
    case 20: return launch_pb2<T, 20>(which, fy, a, st);
    case 24: return launch_pb2<T, 24>(which, fy, a, st);
    case 32: return launch_pb2<T, 32>(which, fy, a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pp
