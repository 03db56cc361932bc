// Transverse stage of the pipe Poisson solve: for one kz plane of the z
// half-spectrum, the forward x,y transforms of the zero-padded plane, the
// four-term Green product of Eq. 10 and the inverse x,y transforms cropped to
// the physical block -- fused, one thread-block cluster per plane.
//
// Pruned padded transforms (Appendix A padding, Eq. A.2).  A row a_j, j < n,
// zero-padded to 2n has the 2n-point DFT
//     Y(2q)   = sum_j a_j w_n^{jq}                       (n-point FFT of a)
//     Y(2q+1) = sum_j (a_j w_{2n}^{j}) w_n^{jq}          (n-point FFT of the twisted row)
// and the inverse kept on j < n is the sum of the two inverse halves, the odd
// one twisted back.  So every transform here is an n-point FFT; the zero half
// is never read and the discarded half never computed.
//
// The four terms of Eq. 10 (convolution or correlation per transverse axis,
// chosen by the direction of the transforms) are applied in the spectral
// domain of a single forward transform: a correlation in y is the product
// with rho_hat(kx, -ky) (Eq. A.9 with the final transform's direction folded
// into an index reflection).  For a mesh spanning the pipe, the correlation
// tables are the convolution table shifted by s = 2*x0/h samples, so all four
// Green spectra are one real octant g(|kx|,|ky|,kz) times phases
// e_x = e^{i pi s_x kx/n}, e_y = e^{i pi s_y ky/n}:
//     Phi = g [rho(kx,ky) - e_y rho(kx,-ky) - e_x rho(-kx,ky) + e_x e_y rho(-kx,-ky)]
//         = g (1 - e_x P_x)(1 - e_y P_y) rho.
// The adjoint (ADJ) applies the transposed chain: backward transforms of the
// padded input first, the transposed product (conjugate phases), forward
// transforms cropped last.
//
// Work split inside the cluster of 2H CTAs: CTA (py, hb) owns the y-parity
// class py (ky = 2q + py) for the rows of block hb.
//   phase 1  y transform of its rows, parity py only      -> local tile Y[q][i]
//   phase 2  column pairs (ky, -ky): x transform, product, inverse x; the
//            column segments of the other row blocks come over DSMEM
//   phase 3  half of block hb's rows: inverse y of both parity halves (one of
//            them in the partner CTA's shared memory), sum, store to HBM
#include <cooperative_groups.h>

#include "solver.cuh"

namespace cg = cooperative_groups;

namespace pp {

template <typename T, int N, int H_, int THREADS_, bool ADJ>
__global__ void __launch_bounds__(THREADS_) transverse_kernel(SolveArgs<T> a) {
  using Cfg = TCfg<T, N, H_, THREADS_>;
  using V = C2<T>;
  constexpr int G = Cfg::G, E = Cfg::E, H = Cfg::H, ROWS = Cfg::ROWS, LD = Cfg::LD;
  constexpr int WARPS = Cfg::THREADS / 32;
  constexpr bool INV1 = ADJ;     // direction of the transforms of the padded input
  constexpr bool INV2 = !ADJ;    // direction of the cropped transforms

  cg::cluster_group cluster = cg::this_cluster();
  const int rank = int(cluster.block_rank());
  const int py = rank / H;
  const int hb = rank % H;
  const int kz = blockIdx.x / Cfg::CLUSTER;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* ybuf = reinterpret_cast<V*>(smem_raw);
  V* scratch = ybuf + N * LD + (threadIdx.x / G) * GroupShape<N>::SSTRIDE;
  V* remote[2 * H];
#pragma unroll
  for (int r = 0; r < 2 * H; ++r) remote[r] = cluster.map_shared_rank(ybuf, r);

  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int t = lane % G;
  V* plane = a.work + size_t(kz) * N * N;

  // ---------------- phase 1: y transform of the padded rows, parity py ----------
  {
    constexpr int GPW = 32 / G;
    constexpr int GPC = WARPS * GPW;
    const int gw = lane / G;
#pragma unroll 1
    for (int r0 = 0; r0 < ROWS; r0 += GPC) {
      const int il = r0 + warp + WARPS * gw;
      const bool act = il < ROWS;
      const int i = hb * ROWS + (act ? il : 0);
      V v[E];
#pragma unroll
      for (int e = 0; e < E; ++e) v[e] = act ? plane[size_t(i) * N + t + G * e] : mk<V>(0, 0);
      if (py) {
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = cmulc<INV1>(v[e], __ldg(&a.w2_t[t + G * e]));
      }
      group_fft<N, INV1>(v, scratch, a.tw_t, t);
      if (act) {
#pragma unroll
        for (int e = 0; e < E; ++e) ybuf[(t + G * e) * LD + il] = v[e];
      }
    }
  }
  cluster.sync();

  // ---------------- phase 2: column pairs (ky, -ky) ----------------
  {
    constexpr int UL = 4 * G;              // lanes per column pair
    constexpr int UPW = 32 / UL;
    constexpr int UPC = (N / 2) / H;       // pairs handled by this CTA
    constexpr int UPP = WARPS * UPW;
    const int ul = lane % UL;
    const int c = ul / (2 * G);            // 0: column A, 1: column B
    const int px = (ul / G) & 1;           // kx parity computed by this group
    const int ey_sign = ADJ ? 1 : -1;      // e_y = w_{2n}^{-s ky} (forward), conjugate (adjoint)
#pragma unroll 1
    for (int u0 = 0; u0 < UPC; u0 += UPP) {
      const int ui = u0 + warp * UPW + lane / UL;
      const bool act = ui < UPC;
      const int u = hb * UPC + (act ? ui : 0);
      int qA, qB;
      bool selfpair;
      if (py == 0) {
        selfpair = (u == 0);
        qA = u;
        qB = selfpair ? N / 2 : N - u;
      } else {
        selfpair = false;
        qA = u;
        qB = N - 1 - u;
      }
      const int q = c ? qB : qA;
      const int ky = 2 * q + py;

      V v[E];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int i = t + G * e;
        const int h = i / ROWS;
        v[e] = act ? remote[py * H + h][q * LD + (i - h * ROWS)] : mk<V>(0, 0);
      }
      if (px) {
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = cmulc<INV1>(v[e], __ldg(&a.w2_t[t + G * e]));
      }
      group_fft<N, INV1>(v, scratch, a.tw_t, t);       // v[e] = X(kx = 2(t+Ge) + px, ky)

      if (a.images) {
        // (1 - e_y P_y): partner column holds -ky at the same kx
        const V ey = __ldg(&a.w2_t[((ey_sign * a.sy * ky) % (2 * N) + 2 * N) % (2 * N)]);
#pragma unroll
        for (int e = 0; e < E; ++e) {
          V o;
          o.x = __shfl_xor_sync(0xffffffffu, v[e].x, 2 * G);
          o.y = __shfl_xor_sync(0xffffffffu, v[e].y, 2 * G);
          if (selfpair) o = v[e];
          v[e] = cfms(v[e], ey, o);
        }
        // (1 - e_x P_x): mirror -kx lives in the same group
        V mm[E];
        mirror_fetch<N>(v, mm, t, px, lane - t);
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int kx = 2 * (t + G * e) + px;
          const V ex = __ldg(&a.w2_t[((ey_sign * a.sx * kx) % (2 * N) + 2 * N) % (2 * N)]);
          v[e] = cfms(v[e], ex, mm[e]);
        }
      }
      {
        const int aky = ky <= N ? ky : 2 * N - ky;
        const T* grow = a.green + (size_t(kz) * (N + 1) + aky) * (N + 1);
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int kx = 2 * (t + G * e) + px;
          const int akx = kx <= N ? kx : 2 * N - kx;
          v[e] = cscale(v[e], act ? __ldg(&grow[akx]) : T(0));
        }
      }
      group_fft<N, INV2>(v, scratch, a.tw_t, t);       // v[e] = x-inverse half px at i = t + G e
      if (px) {
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = cmulc<INV2>(v[e], __ldg(&a.w2_t[t + G * e]));
      }
#pragma unroll
      for (int e = 0; e < E; ++e) {
        v[e].x += __shfl_xor_sync(0xffffffffu, v[e].x, G);
        v[e].y += __shfl_xor_sync(0xffffffffu, v[e].y, G);
      }
      if (act) {
#pragma unroll
        for (int e2 = 0; e2 < E / 2; ++e2) {
          const int e = e2 + px * (E / 2);
          const V val = px ? v[e2 + E / 2] : v[e2];
          const int i = t + G * e;
          const int h = i / ROWS;
          remote[py * H + h][q * LD + (i - h * ROWS)] = val;
        }
      }
    }
  }
  cluster.sync();

  // ---------------- phase 3: inverse y of both parity halves, cropped ----------
  {
    constexpr int RL = 2 * G;
    constexpr int RPW = 32 / RL;
    constexpr int RPC = ROWS / 2;          // rows finished by this CTA
    constexpr int RPP = WARPS * RPW;
    const int sp = (lane / G) & 1;         // source parity
    const V* src = remote[sp * H + hb];
#pragma unroll 1
    for (int r0 = 0; r0 < RPC; r0 += RPP) {
      const int ri = r0 + warp * RPW + lane / RL;
      const bool act = ri < RPC;
      const int il = py * RPC + (act ? ri : 0);
      const int i = hb * ROWS + il;
      V v[E];
#pragma unroll
      for (int e = 0; e < E; ++e) v[e] = act ? src[(t + G * e) * LD + il] : mk<V>(0, 0);
      group_fft<N, INV2>(v, scratch, a.tw_t, t);
      if (sp) {
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = cmulc<INV2>(v[e], __ldg(&a.w2_t[t + G * e]));
      }
#pragma unroll
      for (int e = 0; e < E; ++e) {
        v[e].x += __shfl_xor_sync(0xffffffffu, v[e].x, G);
        v[e].y += __shfl_xor_sync(0xffffffffu, v[e].y, G);
      }
      if (act) {
#pragma unroll
        for (int e2 = 0; e2 < E / 2; ++e2) {
          const int e = e2 + sp * (E / 2);
          const V val = sp ? v[e2 + E / 2] : v[e2];
          plane[size_t(i) * N + t + G * e] = val;
        }
      }
    }
  }
  cluster.sync();
}

template <typename T, int N, int H, int THREADS, bool ADJ>
static cudaError_t tlaunch(const SolveArgs<T>& a, cudaStream_t st) {
  using Cfg = TCfg<T, N, H, THREADS>;
  const size_t smem = Cfg::smem_bytes();
  if constexpr (Cfg::smem_bytes() > kMaxSmem || (N / 2) / H < 1) {
    return cudaErrorInvalidConfiguration;
  } else {
    void (*kern)(SolveArgs<T>) = transverse_kernel<T, N, H, THREADS, ADJ>;
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(Cfg::CLUSTER * (a.nz + 1)), 1, 1);
    cfg.blockDim = dim3(Cfg::THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = Cfg::CLUSTER;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
  }
}

template <typename T, int N>
static cudaError_t tlaunch2(bool adjoint, int h, int threads, const SolveArgs<T>& a, cudaStream_t st) {
#define PP_T_CASE(HH, TT)                                                           \
  if (h == HH && threads == TT)                                                     \
    return adjoint ? tlaunch<T, N, HH, TT, true>(a, st) : tlaunch<T, N, HH, TT, false>(a, st);
  PP_T_CASE(1, 256)
  PP_T_CASE(1, 512)
  PP_T_CASE(2, 256)
  PP_T_CASE(2, 512)
#undef PP_T_CASE
  return cudaErrorInvalidConfiguration;
}

#ifndef PP_T_TYPE
#define PP_T_TYPE float
#endif

template <>
cudaError_t launch_transverse<PP_T_TYPE>(bool adjoint, int h, int threads,
                                         const SolveArgs<PP_T_TYPE>& a, cudaStream_t st) {
  using T = PP_T_TYPE;
  if (a.nx != a.ny) return cudaErrorInvalidValue;
  switch (a.nx) {
    case 16: return tlaunch2<T, 16>(adjoint, h, threads, a, st);
    case 32: return tlaunch2<T, 32>(adjoint, h, threads, a, st);
    case 64: return tlaunch2<T, 64>(adjoint, h, threads, a, st);
    case 128: return tlaunch2<T, 128>(adjoint, h, threads, a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pp
