// z-axis transforms of the pipe Poisson solve (Sec. 2 Eq. 10, Appendix A).
//
// Forward (zfwd_kernel): for every (i,j) column, the 2*nz-point real DFT of the
// zero-padded column (Eq. A.2; the padded half is never read):
//     X(kz) = sum_{k<nz} rho_ijk e^{-2 pi i k kz/(2 nz)},   kz = 0..nz
// Packing z_m = rho_{2m} + i rho_{2m+1} (m < nz/2) turns it into an nz-point
// complex DFT whose input is half zero; that one splits into two nz/2-point
// FFTs (even and odd kz of Z, the odd one on the input twisted by w_nz^m).
// X follows from Z(k) and conj Z(nz-k).  Output is written kz-plane major,
// work[kz][i*ny + j], through a shared-memory staging tile so that every
// store is a contiguous run of COLS columns.
//
// Inverse (zinv_kernel): the transpose of the above for a Hermitian half
// spectrum: rebuild Z from X(k), X(nz-k), two nz/2-point inverse FFTs, keep
// only the physical outputs k < nz (the discarded half is never computed).
// Unnormalised (the 1/(2 nz) lives in the Green spectrum).
//
// CONJ gives the transforms of the opposite direction, used by the adjoint:
// for real data the e^{+} transform is the conjugate of the e^{-} one.
#include "solver.cuh"

namespace pp {

// asynchronous global -> shared copy of one complex element (8 or 16 bytes)
template <typename V>
__device__ __forceinline__ void cp_async_elem(V* dst, const V* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  if constexpr (sizeof(V) == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

template <typename T, int NZ, int WARPS, bool CONJ>
__global__ void __launch_bounds__(32 * WARPS) zfwd_kernel(SolveArgs<T> a) {
  using Cfg = ZCfg<T, NZ, WARPS>;
  using V = C2<T>;
  constexpr int L = Cfg::L, G = Cfg::G, E = Cfg::E;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* sbase = reinterpret_cast<V*>(smem_raw);
  V* stage = sbase;                                   // reused after the FFT

  const int ncols = a.nx * a.ny;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int t = lane % G;
  const int p = (lane / G) & 1;                       // parity of kz produced
  const int col_local = warp * Cfg::CPW + lane / Cfg::UNIT;
  const int col0 = blockIdx.x * Cfg::COLS;
  const int col = col0 + col_local;
  const bool valid = col < ncols;
  V* scratch = sbase + (threadIdx.x / G) * GroupShape<L>::SSTRIDE;

  // packed column, z_m = (rho[2m], rho[2m+1]), m = t + G e
  V v[E];
  const V* src = reinterpret_cast<const V*>(a.rho + size_t(valid ? col : 0) * NZ);
#pragma unroll
  for (int e = 0; e < E; ++e) v[e] = valid ? __ldg(&src[t + G * e]) : mk<V>(0, 0);
  if (p) {
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = cmul(v[e], __ldg(&a.w2_z[2 * (t + G * e)]));  // w_nz^m
  }
  group_fft<L, false>(v, scratch, a.tw_z, t);        // v[e] = Z(2q + p), q = t + G e
  const V z0 = v[0];
  V m[E];
  mirror_fetch<L>(v, m, t, p, lane - t);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int k = 2 * (t + G * e) + p;
    const V zc = cconj(m[e]);
    const V s = cadd(v[e], zc);
    const V d = csub(v[e], zc);
    const V wd = cmul(__ldg(&a.w2_z[k]), d);
    V x = mk<V>(T(0.5) * (s.x + wd.y), T(0.5) * (s.y - wd.x));   // (s - i w d)/2
    v[e] = CONJ ? cconj(x) : x;
  }
  // X(nz) = Re Z(0) - Im Z(0), held by lane t=0 of the even half
  const V xN = mk<V>(z0.x - z0.y, T(0));

  // staged, coalesced stores of the whole (nz+1) x COLS tile
  __syncthreads();                                    // FFT scratch becomes the staging tile
#pragma unroll
  for (int e = 0; e < E; ++e) stage[(2 * (t + G * e) + p) * Cfg::SPAD + col_local] = v[e];
  if (p == 0 && t == 0) stage[NZ * Cfg::SPAD + col_local] = CONJ ? cconj(xN) : xN;
  __syncthreads();
  for (int idx = threadIdx.x; idx < (NZ + 1) * Cfg::COLS; idx += Cfg::THREADS) {
    const int r = idx / Cfg::COLS;
    const int cc = idx % Cfg::COLS;
    if (col0 + cc < ncols) a.work[size_t(r) * ncols + col0 + cc] = stage[r * Cfg::SPAD + cc];
  }
}

template <typename T, int NZ, int WARPS, bool CONJ>
__global__ void __launch_bounds__(32 * WARPS) zinv_kernel(SolveArgs<T> a) {
  using Cfg = ZCfg<T, NZ, WARPS>;
  using V = C2<T>;
  constexpr int L = Cfg::L, G = Cfg::G, E = Cfg::E;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* sbase = reinterpret_cast<V*>(smem_raw);
  V* stage = sbase;                                   // FFT scratch reuses it afterwards

  const int ncols = a.nx * a.ny;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int t = lane % G;
  const int p = (lane / G) & 1;
  const int col_local = warp * Cfg::CPW + lane / Cfg::UNIT;
  const int col0 = blockIdx.x * Cfg::COLS;
  const int col = col0 + col_local;
  const bool valid = col < ncols;
  V* scratch = sbase + (threadIdx.x / G) * GroupShape<L>::SSTRIDE;

  // the whole (nz+1) x COLS tile in flight at once (cp.async, one element each)
  for (int idx = threadIdx.x; idx < (NZ + 1) * Cfg::COLS; idx += Cfg::THREADS) {
    const int r = idx / Cfg::COLS;
    const int cc = idx % Cfg::COLS;
    if (col0 + cc < ncols) cp_async_elem(&stage[r * Cfg::SPAD + cc], &a.work[size_t(r) * ncols + col0 + cc]);
  }
  cp_async_wait_all();
  __syncthreads();
  V v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) v[e] = stage[(2 * (t + G * e) + p) * Cfg::SPAD + col_local];
  V xN = stage[NZ * Cfg::SPAD + col_local];
  __syncthreads();                                    // staging tile becomes FFT scratch
  if (CONJ) {
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = cconj(v[e]);
    xN = cconj(xN);
  }
  // partner X(nz - k) of every k = 2q + p (q = 0 pairs with X(nz))
  V m[E];
  mirror_fetch<L>(v, m, t, p, lane - t);
  if (p == 0 && t == 0) m[0] = xN;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int k = 2 * (t + G * e) + p;
    const V xm = cconj(m[e]);
    const V s = cadd(v[e], xm);
    const V d = csub(v[e], xm);
    const V wd = cmulc<true>(d, __ldg(&a.w2_z[k]));           // w_{2nz}^{-k} d
    v[e] = mk<V>(s.x - wd.y, s.y + wd.x);                      // s + i w d
  }
  group_fft<L, true>(v, scratch, a.tw_z, t);                  // z_p(m), m = t + G e
  if (p) {
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = cmulc<true>(v[e], __ldg(&a.w2_z[2 * (t + G * e)]));
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    v[e].x += __shfl_xor_sync(0xffffffffu, v[e].x, G);
    v[e].y += __shfl_xor_sync(0xffffffffu, v[e].y, G);
  }
  if (valid) {
    V* dst = reinterpret_cast<V*>(a.phi + size_t(col) * NZ);
#pragma unroll
    for (int e2 = 0; e2 < E / 2; ++e2) {
      const int e = e2 + p * (E / 2);
      const V val = p ? v[e2 + E / 2] : v[e2];
      dst[t + G * e] = val;
    }
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
static cudaError_t zlaunch2(bool forward, bool conj, const SolveArgs<T>& a, cudaStream_t st) {
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
PP_Z_INST(PP_Z_TYPE, 512, 8)
PP_Z_INST(PP_Z_TYPE, 512, 16)
PP_Z_INST(PP_Z_TYPE, 1024, 8)
PP_Z_INST(PP_Z_TYPE, 1024, 16)

template <>
cudaError_t launch_z<PP_Z_TYPE>(bool forward, int warps, bool conj, const SolveArgs<PP_Z_TYPE>& a,
                                cudaStream_t st) {
  using T = PP_Z_TYPE;
  const bool w16 = (warps == 16);
  switch (a.nz) {
    case 32: return zlaunch2<T, 32, 8>(forward, conj, a, st);
    case 64: return zlaunch2<T, 64, 8>(forward, conj, a, st);
    case 128: return zlaunch2<T, 128, 8>(forward, conj, a, st);
    case 256: return zlaunch2<T, 256, 8>(forward, conj, a, st);
    case 512: return w16 ? zlaunch2<T, 512, 16>(forward, conj, a, st)
                         : zlaunch2<T, 512, 8>(forward, conj, a, st);
    case 1024: return w16 ? zlaunch2<T, 1024, 16>(forward, conj, a, st)
                          : zlaunch2<T, 1024, 8>(forward, conj, a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pp
