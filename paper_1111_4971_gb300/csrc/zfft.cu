// z-axis transform kernels and their host launchers; the device routines
// (and the description of the transforms) are in zfft_impl.cuh.
#include "zfft_impl.cuh"

namespace pp {

// CTAs of the single-tile z kernels resident per SM (their register cap:
// 128 per thread at 4 and 8 warps per CTA)
template <int WARPS>
constexpr int z_ctas_per_sm() { return WARPS <= 4 ? 4 : (WARPS <= 8 ? 2 : 1); }

// The tile that a CTA of the next wave will take: this tile plus the number
// of CTAs resident at once (SMs x CTAs per SM), blocks being issued in order.
template <int WARPS>
__device__ __forceinline__ int next_wave_tile() {
  unsigned nsm;
  asm("mov.u32 %0, %%nsmid;" : "=r"(nsm));
  return int(blockIdx.x) + int(nsm) * z_ctas_per_sm<WARPS>();
}

template <typename T, int NZ, int WARPS, bool CONJ, bool H16>
__global__ void __launch_bounds__(32 * WARPS, z_ctas_per_sm<WARPS>()) zfwd_kernel(SolveArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (threadIdx.x == 0) {
    // its input columns (contiguous, whole 16-byte units) into L2
    using Cfg = ZCfg<T, NZ, WARPS>;
    const int ncols = a.nx * a.ny, c0 = next_wave_tile<WARPS>() * Cfg::COLS;
    if (c0 < ncols) {
      const int c1 = c0 + Cfg::COLS < ncols ? c0 + Cfg::COLS : ncols;
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(a.rho + size_t(c0) * NZ),
                   "r"(unsigned(sizeof(T) * size_t(c1 - c0) * NZ))
                   : "memory");
    }
  }
  zfwd_tile<T, NZ, WARPS, CONJ, H16>(a, blockIdx.x, smem_raw);
}

template <typename T, int NZ, int WARPS, bool CONJ, bool H16>
__global__ void __launch_bounds__(32 * WARPS, z_ctas_per_sm<WARPS>()) zinv_kernel(SolveArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  zinv_tile<T, NZ, WARPS, CONJ, H16>(a, blockIdx.x, smem_raw);
}

// pipelined variants: a grid of at most (SMs x resident CTAs), each CTA
// walking tiles blockIdx.x, blockIdx.x + gridDim.x, ...
template <typename T, int NZ, int WARPS, bool CONJ>
__global__ void __launch_bounds__(32 * WARPS, 1) zfwd_pipe_kernel(SolveArgs<T> a, int ntiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int count = (ntiles - int(blockIdx.x) + int(gridDim.x) - 1) / int(gridDim.x);
  zfwd_tiles_pipe<T, NZ, WARPS, CONJ>(a, blockIdx.x, gridDim.x, count, smem_raw);
}

template <typename T, int NZ, int WARPS, bool CONJ>
__global__ void __launch_bounds__(32 * WARPS, 1) zinv_pipe_kernel(SolveArgs<T> a, int ntiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int count = (ntiles - int(blockIdx.x) + int(gridDim.x) - 1) / int(gridDim.x);
  zinv_tiles_pipe<T, NZ, WARPS, CONJ>(a, blockIdx.x, gridDim.x, count, smem_raw);
}

template <typename T, int NZ, int W, bool C>
static cudaError_t zlaunch_pipe(bool forward, const SolveArgs<T>& a, cudaStream_t st) {
  using Cfg = ZCfg<T, NZ, W>;
  if constexpr (Cfg::fwd_pipe_smem() > kMaxSmem || Cfg::inv_pipe_smem() > kMaxSmem) {
    return cudaErrorInvalidConfiguration;
  } else {
    const size_t smem = forward ? Cfg::fwd_pipe_smem() : Cfg::inv_pipe_smem();
    void (*kern)(SolveArgs<T>, int) = forward ? zfwd_pipe_kernel<T, NZ, W, C> : zinv_pipe_kernel<T, NZ, W, C>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Cfg::THREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int ntiles = (a.nx * a.ny + Cfg::COLS - 1) / Cfg::COLS;
    const int grid = ntiles < sms * per_sm ? ntiles : sms * per_sm;
    kern<<<grid, Cfg::THREADS, smem, st>>>(a, ntiles);
    return cudaGetLastError();
  }
}

template <typename T, int NZ, int W, bool C>
static cudaError_t zlaunch(bool forward, const SolveArgs<T>& a, cudaStream_t st) {
  using Cfg = ZCfg<T, NZ, W>;
  const size_t smem = Cfg::smem_bytes();
  if (smem > kMaxSmem) return cudaErrorInvalidConfiguration;
  void (*kern)(SolveArgs<T>) = forward ? zfwd_kernel<T, NZ, W, C> : zinv_kernel<T, NZ, W, C>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
  }
  const int ncols = a.nx * a.ny;
  kern<<<(ncols + Cfg::COLS - 1) / Cfg::COLS, Cfg::THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename T, int NZ, int W>
static cudaError_t zlaunch2(bool forward, int pipe, bool conj, const SolveArgs<T>& a, cudaStream_t st) {
  if (pipe)
    return conj ? zlaunch_pipe<T, NZ, W, true>(forward, a, st) : zlaunch_pipe<T, NZ, W, false>(forward, a, st);
  return conj ? zlaunch<T, NZ, W, true>(forward, a, st) : zlaunch<T, NZ, W, false>(forward, a, st);
}

#define PP_Z_INST(T, NZ, W)                                                  \
  template __global__ void zfwd_kernel<T, NZ, W, false>(SolveArgs<T>);       \
  template __global__ void zfwd_kernel<T, NZ, W, true>(SolveArgs<T>);        \
  template __global__ void zinv_kernel<T, NZ, W, false>(SolveArgs<T>);       \
  template __global__ void zinv_kernel<T, NZ, W, true>(SolveArgs<T>);

#ifndef PP_Z_TYPE
#define PP_Z_TYPE float
#endif
PP_Z_INST(PP_Z_TYPE, 32, 8)
PP_Z_INST(PP_Z_TYPE, 64, 8)
PP_Z_INST(PP_Z_TYPE, 128, 8)
PP_Z_INST(PP_Z_TYPE, 256, 8)
PP_Z_INST(PP_Z_TYPE, 512, 4)
PP_Z_INST(PP_Z_TYPE, 512, 8)
PP_Z_INST(PP_Z_TYPE, 512, 16)
PP_Z_INST(PP_Z_TYPE, 1024, 4)
PP_Z_INST(PP_Z_TYPE, 1024, 8)
PP_Z_INST(PP_Z_TYPE, 1024, 16)

template <>
cudaError_t launch_z<PP_Z_TYPE>(bool forward, int warps, int pipe, bool conj, const SolveArgs<PP_Z_TYPE>& a,
                                cudaStream_t st) {
  using T = PP_Z_TYPE;
  // 4 and 16 warps per CTA where a column fills a warp (nz >= 512), else 8
  const bool w16 = (warps == 16), w4 = (warps == 4);
  switch (a.nz) {
    case 32: return zlaunch2<T, 32, 8>(forward, pipe, conj, a, st);
    case 64: return zlaunch2<T, 64, 8>(forward, pipe, conj, a, st);
    case 128: return zlaunch2<T, 128, 8>(forward, pipe, conj, a, st);
    case 256: return zlaunch2<T, 256, 8>(forward, pipe, conj, a, st);
    case 512: return w16 ? zlaunch2<T, 512, 16>(forward, pipe, conj, a, st)
                    : w4 ? zlaunch2<T, 512, 4>(forward, pipe, conj, a, st)
                         : zlaunch2<T, 512, 8>(forward, pipe, conj, a, st);
    case 1024: return w16 ? zlaunch2<T, 1024, 16>(forward, pipe, conj, a, st)
                     : w4 ? zlaunch2<T, 1024, 4>(forward, pipe, conj, a, st)
                          : zlaunch2<T, 1024, 8>(forward, pipe, conj, a, st);
    default: return cudaErrorInvalidValue;
  }
}

#if !defined(PP_Z_F64_UNIT)
// complex-FP16 spectra (FP32 arithmetic): single-tile kernels only
template <int NZ, int W, bool C>
static cudaError_t zlaunch16(bool forward, const SolveArgs<float>& a, cudaStream_t st) {
  using Cfg = ZCfg<float, NZ, W>;
  const size_t smem = Cfg::smem_bytes() + sizeof(float) * W;      // + the tile-max scratch
  if (smem > kMaxSmem) return cudaErrorInvalidConfiguration;
  void (*kern)(SolveArgs<float>) = forward ? zfwd_kernel<float, NZ, W, C, true> : zinv_kernel<float, NZ, W, C, true>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
  }
  const int ncols = a.nx * a.ny;
  kern<<<(ncols + Cfg::COLS - 1) / Cfg::COLS, Cfg::THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

template <int NZ, int W>
static cudaError_t zlaunch16c(bool forward, bool conj, const SolveArgs<float>& a, cudaStream_t st) {
  return conj ? zlaunch16<NZ, W, true>(forward, a, st) : zlaunch16<NZ, W, false>(forward, a, st);
}

cudaError_t launch_z_c16(bool forward, int warps, bool conj, const SolveArgs<float>& a, cudaStream_t st) {
  const bool w16 = (warps == 16);
  switch (a.nz) {
    case 32: return zlaunch16c<32, 8>(forward, conj, a, st);
    case 64: return zlaunch16c<64, 8>(forward, conj, a, st);
    case 128: return zlaunch16c<128, 8>(forward, conj, a, st);
    case 256: return zlaunch16c<256, 8>(forward, conj, a, st);
    case 512: return w16 ? zlaunch16c<512, 16>(forward, conj, a, st) : zlaunch16c<512, 8>(forward, conj, a, st);
    case 1024: return w16 ? zlaunch16c<1024, 16>(forward, conj, a, st) : zlaunch16c<1024, 8>(forward, conj, a, st);
    default: return cudaErrorInvalidValue;
  }
}

int z_tile_cols(int nz, int warps) {
  const bool w16 = (warps == 16);
  switch (nz) {
    case 32: return ZCfg<float, 32, 8>::COLS;
    case 64: return ZCfg<float, 64, 8>::COLS;
    case 128: return ZCfg<float, 128, 8>::COLS;
    case 256: return ZCfg<float, 256, 8>::COLS;
    case 512: return w16 ? ZCfg<float, 512, 16>::COLS : ZCfg<float, 512, 8>::COLS;
    case 1024: return w16 ? ZCfg<float, 1024, 16>::COLS : ZCfg<float, 1024, 8>::COLS;
    default: return 0;
  }
}
#endif

}  // namespace pp
