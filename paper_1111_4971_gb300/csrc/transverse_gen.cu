// Transverse stage of the pipe operator for general meshes (a transverse
// window, Sec. 5): the four-term product of Eq. 10 with the four transformed
// tables stored in full, no symmetry assumed.
//
// Per kz plane of the z half-spectrum u[i][j] (i, j < N):
//   pass 1  rows i: 2N-point forward transform along y of the zero-padded row
//           -> Y[i][ky], ky = 0..2N-1, in shared memory;
//   pass 2  column pairs (ky, -ky) together: 2N-point forward transforms
//           along x of both zero-padded columns, X_ky(kx) and X_-ky(kx), with
//           their mirrors X(-kx) from warp shuffles, then
//             Phi(kx,ky) = Tcc X_ky(kx) - Tcr X_-ky(kx) - Trc X_ky(-kx) + Trr X_-ky(-kx)
//           (tables at (kx, ky)), which is Eq. 10's four products with the
//           reflections R_t applied to the density spectrum; the inverse
//           transforms along x keep rows i < N;
//   pass 3  rows i: 2N-point inverse transform along y, keep j < N.
// The adjoint applies the transposed product, the tables taken at the
// reflected frequencies: Tcc(k) S(k) - Tcr(kx,-ky) S(kx,-ky)
// - Trc(-kx,ky) S(-kx,ky) + Trr(-kx,-ky) S(-kx,-ky), with the transform
// directions swapped.  Tables: a.green viewed as complex [4][nz+1][2N][2N]
// (cc, cr, rc, rr; kx fastest), scaled by hx hy hz / (8 nx ny nz).
#include "fft_common.cuh"
#include "solver.cuh"

namespace pp {

namespace {

template <typename T, int N, int THREADS>
struct TGenCfg {
  static constexpr int L = 2 * N;
  using S = GroupShape<L>;
  static constexpr int G = S::G, E = S::E;
  static constexpr int LD = L + 1;                 // padded row of Y
  static constexpr int GROUPS = THREADS / G;
  static constexpr size_t smem_bytes() {
    return sizeof(C2<T>) * (size_t(N) * LD + size_t(GROUPS) * S::SSTRIDE);
  }
};

template <typename V>
__device__ __forceinline__ V cmadd(V acc, V a, V b) {      // acc + a b
  return mk<V>(acc.x + (a.x * b.x - a.y * b.y), acc.y + (a.x * b.y + a.y * b.x));
}
template <typename V>
__device__ __forceinline__ V cmsub(V acc, V a, V b) {      // acc - a b
  return mk<V>(acc.x - (a.x * b.x - a.y * b.y), acc.y - (a.x * b.y + a.y * b.x));
}

template <typename T, int N, int THREADS, bool ADJ>
__global__ void __launch_bounds__(THREADS, 1) transverse_gen_kernel(SolveArgs<T> a) {
  using Cfg = TGenCfg<T, N, THREADS>;
  using V = C2<T>;
  constexpr int L = Cfg::L, G = Cfg::G, E = Cfg::E, H = E / 2, LD = Cfg::LD;
  constexpr int WARPS = THREADS / 32, GPW = 32 / G, GPC = WARPS * GPW;
  constexpr bool INV1 = ADJ, INV2 = !ADJ;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* Y = reinterpret_cast<V*>(smem_raw);
  V* scratch = Y + size_t(N) * LD + (threadIdx.x / G) * GroupShape<L>::SSTRIDE;
  const V* tw = a.tw_t2c;
  const int lane = threadIdx.x & 31;
  const int t = lane % G;
  const int line = lane / G + GPW * (threadIdx.x >> 5);
  const int kz = blockIdx.x;
  V* plane = a.work + size_t(kz) * N * N;
  const size_t tplane = size_t(L) * L;
  const V* tab = reinterpret_cast<const V*>(a.green) + size_t(kz) * tplane;
  const size_t tstride = size_t(a.nz + 1) * tplane;          // between the four tables

  // pass 1: rows along y
#pragma unroll 1
  for (int r0 = 0; r0 < N; r0 += GPC) {
    const int il = r0 + line;
    const int i = il < N ? il : 0;
    V v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = e < H ? plane[size_t(i) * N + t + G * e] : mk<V>(0, 0);
    group_fft<L, INV1>(v, scratch, tw, t);
    if (il < N) {
#pragma unroll
      for (int e = 0; e < E; ++e) Y[i * LD + t + G * e] = v[e];
    }
  }
  __syncthreads();

  // pass 2: column pairs (ky, -ky), ky = 0..N
#pragma unroll 1
  for (int c0 = 0; c0 <= N; c0 += GPC) {
    const int q = c0 + line;
    const bool act = q <= N;
    const int ka = act ? q : 0;
    const int kb = (L - ka) & (L - 1);                        // -ky
    V xa[E], xb[E], ma[E], mb[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int i = t + G * e;
      xa[e] = e < H ? Y[i * LD + ka] : mk<V>(0, 0);
      xb[e] = e < H ? Y[i * LD + kb] : mk<V>(0, 0);
    }
    group_fft<L, INV1>(xa, scratch, tw, t);
    group_fft<L, INV1>(xb, scratch, tw, t);
    mirror_fetch<L>(xa, ma, t, 0, lane - t);                  // X_ky(-kx)
    mirror_fetch<L>(xb, mb, t, 0, lane - t);                  // X_-ky(-kx)
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int kx = t + G * e;
      const int mkx = (L - kx) & (L - 1);
      V pa = mk<V>(0, 0), pb = mk<V>(0, 0);
      if (act) {
        const V* Tcc = tab;
        const V* Tcr = tab + tstride;
        const V* Trc = tab + 2 * tstride;
        const V* Trr = tab + 3 * tstride;
        if constexpr (!ADJ) {
          pa = cmul(__ldg(&Tcc[size_t(ka) * L + kx]), xa[e]);
          pa = cmsub(pa, __ldg(&Tcr[size_t(ka) * L + kx]), xb[e]);
          pa = cmsub(pa, __ldg(&Trc[size_t(ka) * L + kx]), ma[e]);
          pa = cmadd(pa, __ldg(&Trr[size_t(ka) * L + kx]), mb[e]);
          pb = cmul(__ldg(&Tcc[size_t(kb) * L + kx]), xb[e]);
          pb = cmsub(pb, __ldg(&Tcr[size_t(kb) * L + kx]), xa[e]);
          pb = cmsub(pb, __ldg(&Trc[size_t(kb) * L + kx]), mb[e]);
          pb = cmadd(pb, __ldg(&Trr[size_t(kb) * L + kx]), ma[e]);
        } else {
          pa = cmul(__ldg(&Tcc[size_t(ka) * L + kx]), xa[e]);
          pa = cmsub(pa, __ldg(&Tcr[size_t(kb) * L + kx]), xb[e]);
          pa = cmsub(pa, __ldg(&Trc[size_t(ka) * L + mkx]), ma[e]);
          pa = cmadd(pa, __ldg(&Trr[size_t(kb) * L + mkx]), mb[e]);
          pb = cmul(__ldg(&Tcc[size_t(kb) * L + kx]), xb[e]);
          pb = cmsub(pb, __ldg(&Tcr[size_t(ka) * L + kx]), xa[e]);
          pb = cmsub(pb, __ldg(&Trc[size_t(kb) * L + mkx]), mb[e]);
          pb = cmadd(pb, __ldg(&Trr[size_t(ka) * L + mkx]), ma[e]);
        }
      }
      xa[e] = pa;
      xb[e] = pb;
    }
    group_fft<L, INV2>(xa, scratch, tw, t);
    group_fft<L, INV2>(xb, scratch, tw, t);
    if (act) {
#pragma unroll
      for (int e = 0; e < H; ++e) {
        const int i = t + G * e;
        Y[i * LD + ka] = xa[e];
        if (kb != ka) Y[i * LD + kb] = xb[e];
      }
    }
  }
  __syncthreads();

  // pass 3: rows back along y, keep j < N
#pragma unroll 1
  for (int r0 = 0; r0 < N; r0 += GPC) {
    const int il = r0 + line;
    const int i = il < N ? il : 0;
    V v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = Y[i * LD + t + G * e];
    group_fft<L, INV2>(v, scratch, tw, t);
    if (il < N) {
#pragma unroll
      for (int e = 0; e < H; ++e) plane[size_t(i) * N + t + G * e] = v[e];
    }
  }
}

template <typename T, int N, int THREADS, bool ADJ>
cudaError_t tglaunch(const SolveArgs<T>& a, cudaStream_t st) {
  using Cfg = TGenCfg<T, N, THREADS>;
  if constexpr (Cfg::smem_bytes() > kMaxSmem) {
    return cudaErrorInvalidConfiguration;
  } else {
    const size_t smem = Cfg::smem_bytes();
    void (*kern)(SolveArgs<T>) = transverse_gen_kernel<T, N, THREADS, ADJ>;
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      if (e != cudaSuccess) return e;
    }
    kern<<<a.nz + 1, THREADS, smem, st>>>(a);
    return cudaGetLastError();
  }
}

template <typename T, int N>
cudaError_t tglaunch2(bool adjoint, int threads, const SolveArgs<T>& a, cudaStream_t st) {
  switch (threads) {
    case 128: return adjoint ? tglaunch<T, N, 128, true>(a, st) : tglaunch<T, N, 128, false>(a, st);
    case 256: return adjoint ? tglaunch<T, N, 256, true>(a, st) : tglaunch<T, N, 256, false>(a, st);
    case 512: return adjoint ? tglaunch<T, N, 512, true>(a, st) : tglaunch<T, N, 512, false>(a, st);
    default: return cudaErrorInvalidConfiguration;
  }
}

template <typename T>
cudaError_t launch_gen(bool adjoint, int threads, const SolveArgs<T>& a, cudaStream_t st) {
  if (a.nx != a.ny) return cudaErrorInvalidValue;
  switch (a.nx) {
    case 16: return tglaunch2<T, 16>(adjoint, threads, a, st);
    case 32: return tglaunch2<T, 32>(adjoint, threads, a, st);
    case 64: return tglaunch2<T, 64>(adjoint, threads, a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

template <>
cudaError_t launch_transverse_gen<float>(bool adjoint, int threads, const SolveArgs<float>& a, cudaStream_t st) {
  return launch_gen<float>(adjoint, threads, a, st);
}
template <>
cudaError_t launch_transverse_gen<double>(bool adjoint, int threads, const SolveArgs<double>& a,
                                          cudaStream_t st) {
  return launch_gen<double>(adjoint, threads, a, st);
}

}  // namespace pp
