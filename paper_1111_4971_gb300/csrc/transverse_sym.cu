// Pipe-operator transverse stage: kernel and host launcher.  The device
// routine and the description of the method are in tsym_impl.cuh.
#include "tdst_impl.cuh"
#include "tsym_impl.cuh"

namespace pp {

// MINB = 2 caps registers so that two CTAs share an SM (where their shared
// memory also fits)
template <typename T, int N, int HB, int THREADS, bool ADJ, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) transverse_sym_kernel(SolveArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  tsym_plane<T, N, HB, THREADS, ADJ>(a, blockIdx.x / HB, smem_raw);
}

template <typename T, int N, int HB, int THREADS, bool ADJ, int MINB = 1>
static cudaError_t tslaunch(const SolveArgs<T>& a, cudaStream_t st) {
  using Cfg = TSymCfg<T, N, HB, THREADS>;
  if constexpr (Cfg::smem_bytes() > kMaxSmem || N / HB < 2 || (N < 128 && HB != 1)) {
    return cudaErrorInvalidConfiguration;
  } else {
    const size_t smem = Cfg::smem_bytes();
    void (*kern)(SolveArgs<T>) = transverse_sym_kernel<T, N, HB, THREADS, ADJ, MINB>;
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(HB * (a.nz + 1)), 1, 1);
    cfg.blockDim = dim3(THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = HB;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
  }
}

// the cyclic-layout variant: one CTA of 512 threads per plane
template <typename T, int N, bool ADJ>
__global__ void __launch_bounds__(512, 1) transverse_cyc_kernel(SolveArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  tsym_cyc_plane<T, N, 512, ADJ>(a, blockIdx.x, smem_raw);
}

template <typename T, int N, bool ADJ>
static cudaError_t tclaunch(const SolveArgs<T>& a, cudaStream_t st) {
  using Cfg = TCycCfg<T, N, 512>;
  if constexpr (Cfg::smem_bytes() > kMaxSmem) {
    return cudaErrorInvalidConfiguration;
  } else {
    const size_t smem = Cfg::smem_bytes();
    void (*kern)(SolveArgs<T>) = transverse_cyc_kernel<T, N, ADJ>;
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      if (e != cudaSuccess) return e;
    }
    kern<<<a.nz + 1, 512, smem, st>>>(a);
    return cudaGetLastError();
  }
}

// the N-point routine for cell-centred meshes: one CTA per kz plane
template <typename T, int N, int THREADS, bool ADJ, bool H16 = false, bool GB = false>
__global__ void __launch_bounds__(THREADS, 1) transverse_dst_kernel(SolveArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  tdst_plane<T, N, THREADS, ADJ, H16, GB>(a, blockIdx.x, smem_raw);
}

// planes that do not fit in shared memory go through the global scratch a.tbuf
template <typename T, int N, int THREADS, bool ADJ, bool H16 = false>
static cudaError_t tdlaunch(const SolveArgs<T>& a, cudaStream_t st) {
  constexpr bool GB = TDstCfg<T, N, THREADS, false>::smem_bytes() > kMaxSmem;
  using Cfg = TDstCfg<T, N, THREADS, GB>;
  if constexpr (Cfg::smem_bytes() > kMaxSmem || (GB && H16)) {
    return cudaErrorInvalidConfiguration;
  } else {
    if (GB && !a.tbuf) return cudaErrorInvalidConfiguration;
    const size_t smem = Cfg::smem_bytes();
    void (*kern)(SolveArgs<T>) = transverse_dst_kernel<T, N, THREADS, ADJ, H16, GB>;
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      if (e != cudaSuccess) return e;
    }
    kern<<<a.nz + 1, THREADS, smem, st>>>(a);
    return cudaGetLastError();
  }
}

// the staged persistent form of the N-point routine: one CTA per SM (as many
// as fit), each looping over planes with its rows copied in ahead by TMA
template <typename T, int N, int THREADS, bool ADJ>
__global__ void __launch_bounds__(THREADS, 1) transverse_dsts_kernel(SolveArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  tdst_persistent<T, N, THREADS, ADJ>(a, smem_raw);
}

template <typename T, int N, int THREADS, bool ADJ>
static cudaError_t tdslaunch(const SolveArgs<T>& a, cudaStream_t st) {
  using Cfg = TDstCfg<T, N, THREADS, false, true>;
  if constexpr (Cfg::smem_bytes() > kMaxSmem) {
    return cudaErrorInvalidConfiguration;
  } else {
    const size_t smem = Cfg::smem_bytes();
    void (*kern)(SolveArgs<T>) = transverse_dsts_kernel<T, N, THREADS, ADJ>;
    cudaError_t e;
    if (smem > 48 * 1024) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      if (e != cudaSuccess) return e;
    }
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, smem)) != cudaSuccess) return e;
    if (per_sm < 1 || sms < 1) return cudaErrorInvalidConfiguration;
    const int grid = a.nz + 1 < sms * per_sm ? a.nz + 1 : sms * per_sm;
    kern<<<grid, THREADS, smem, st>>>(a);
    return cudaGetLastError();
  }
}

template <typename T, int N>
static cudaError_t tdslaunch2(bool adjoint, int hb, int threads, const SolveArgs<T>& a, cudaStream_t st) {
  if (hb != 1 || a.sx != 1 || a.sy != 1) return cudaErrorInvalidValue;
  switch (threads) {
    case 128: return adjoint ? tdslaunch<T, N, 128, true>(a, st) : tdslaunch<T, N, 128, false>(a, st);
    case 256: return adjoint ? tdslaunch<T, N, 256, true>(a, st) : tdslaunch<T, N, 256, false>(a, st);
    case 512: return adjoint ? tdslaunch<T, N, 512, true>(a, st) : tdslaunch<T, N, 512, false>(a, st);
    default: return cudaErrorInvalidConfiguration;
  }
}

template <typename T, int N>
static cudaError_t tdlaunch2(bool adjoint, int hb, int threads, const SolveArgs<T>& a, cudaStream_t st) {
  if (hb != 1 || a.sx != 1 || a.sy != 1) return cudaErrorInvalidValue;
  switch (threads) {
    case 128: return adjoint ? tdlaunch<T, N, 128, true>(a, st) : tdlaunch<T, N, 128, false>(a, st);
    case 256: return adjoint ? tdlaunch<T, N, 256, true>(a, st) : tdlaunch<T, N, 256, false>(a, st);
    case 512: return adjoint ? tdlaunch<T, N, 512, true>(a, st) : tdlaunch<T, N, 512, false>(a, st);
    default: return cudaErrorInvalidConfiguration;
  }
}

template <typename T, int N>
static cudaError_t tslaunch2(bool adjoint, int hb, int threads, const SolveArgs<T>& a, cudaStream_t st) {
  if (hb == 1 && threads == 512)            // cyclic-layout variant, 16 warps
    return adjoint ? tclaunch<T, N, true>(a, st) : tclaunch<T, N, false>(a, st);
#define PP_TS_CASE(HH, TT)                                                           \
  if (hb == HH && threads == TT)                                                     \
    return adjoint ? tslaunch<T, N, HH, TT, true>(a, st) : tslaunch<T, N, HH, TT, false>(a, st);
  PP_TS_CASE(1, 128)
  PP_TS_CASE(1, 256)
  PP_TS_CASE(2, 128)
  PP_TS_CASE(2, 256)
  PP_TS_CASE(4, 128)
#undef PP_TS_CASE
  if (hb == 4 && threads == 256)          // 112 KB of shared memory: two CTAs per SM
    return adjoint ? tslaunch<T, N, 4, 256, true, 2>(a, st) : tslaunch<T, N, 4, 256, false, 2>(a, st);
  return cudaErrorInvalidConfiguration;
}

#ifndef PP_TS_TYPE
#define PP_TS_TYPE float
#endif

template <>
cudaError_t launch_transverse_sym<PP_TS_TYPE>(bool adjoint, int kind, int hb, int threads,
                                              const SolveArgs<PP_TS_TYPE>& a, cudaStream_t st) {
  using T = PP_TS_TYPE;
  if (a.nx != a.ny || !a.images) return cudaErrorInvalidValue;
  if (kind == 1) {
    switch (a.nx) {
      case 16: return tdlaunch2<T, 16>(adjoint, hb, threads, a, st);
      case 32: return tdlaunch2<T, 32>(adjoint, hb, threads, a, st);
      case 64: return tdlaunch2<T, 64>(adjoint, hb, threads, a, st);
      case 128: return tdlaunch2<T, 128>(adjoint, hb, threads, a, st);
      default: return cudaErrorInvalidValue;
    }
  }
  if (kind == 2) {
    switch (a.nx) {
      case 16: return tdslaunch2<T, 16>(adjoint, hb, threads, a, st);
      case 32: return tdslaunch2<T, 32>(adjoint, hb, threads, a, st);
      case 64: return tdslaunch2<T, 64>(adjoint, hb, threads, a, st);
      case 128: return tdslaunch2<T, 128>(adjoint, hb, threads, a, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (a.nx) {
    case 16: return tslaunch2<T, 16>(adjoint, hb, threads, a, st);
    case 32: return tslaunch2<T, 32>(adjoint, hb, threads, a, st);
    case 64: return tslaunch2<T, 64>(adjoint, hb, threads, a, st);
    case 128: return tslaunch2<T, 128>(adjoint, hb, threads, a, st);
    default: return cudaErrorInvalidValue;
  }
}

#if !defined(PP_TS_F64_UNIT)
template <int N>
static cudaError_t tdlaunch16(bool adjoint, int threads, const SolveArgs<float>& a, cudaStream_t st) {
  switch (threads) {
    case 128: return adjoint ? tdlaunch<float, N, 128, true, true>(a, st) : tdlaunch<float, N, 128, false, true>(a, st);
    case 256: return adjoint ? tdlaunch<float, N, 256, true, true>(a, st) : tdlaunch<float, N, 256, false, true>(a, st);
    case 512: return adjoint ? tdlaunch<float, N, 512, true, true>(a, st) : tdlaunch<float, N, 512, false, true>(a, st);
    default: return cudaErrorInvalidConfiguration;
  }
}

cudaError_t launch_transverse_c16(bool adjoint, int threads, const SolveArgs<float>& a, cudaStream_t st) {
  if (a.nx != a.ny || !a.images || a.sx != 1 || a.sy != 1 || a.zcols <= 0) return cudaErrorInvalidValue;
  switch (a.nx) {
    case 16: return tdlaunch16<16>(adjoint, threads, a, st);
    case 32: return tdlaunch16<32>(adjoint, threads, a, st);
    case 64: return tdlaunch16<64>(adjoint, threads, a, st);
    case 128: return tdlaunch16<128>(adjoint, threads, a, st);
    default: return cudaErrorInvalidValue;
  }
}
#endif

}  // namespace pp
