// Device routine of the pipe-operator transverse stage, shared by the
// per-stage kernel (transverse_sym.cu) and the batched persistent kernel.
//
// Transverse stage of the pipe operator on a mesh spanning the pipe.
//
// For one kz plane of the z half-spectrum this computes the padded forward
// x,y transforms, the four-term product of Eq. 10 and the cropped inverse
// x,y transforms.  On a mesh with n*h = a and an integer s = 2*x0/h, the
// correlation tables are the convolution table shifted by s samples, so the
// four transformed Green tables are one real octant g(|kx|,|ky|,kz) times the
// phases e_x = e^{i pi s_x kx/n}, e_y = e^{i pi s_y ky/n}, and the product of
// Eq. 10 (correlation = product with the index-reflected spectrum, Eq. A.9)
// factorises:
//     Phi = g (1 - e_x P_x)(1 - e_y P_y) rho_hat,   (P f)(k) = f(-k).
// Consequences used here (exact identities, not approximations):
//   u = (1 - e_y P_y) Y satisfies u(-ky) = -conj(e_y(ky)) u(ky) and u(0) = 0,
//   and the x part and g do not depend on the sign of ky, so the whole product
//   is carried by the columns ky = 1..n; the inverse y transform rebuilds
//   ky > n from them.  (The same holds in x; there both halves are formed in
//   registers.)
//
// Every transform is a full 2n-point FFT of the zero-padded line (Appendix A,
// Eq. A.2): the padded half of the input is a compile-time zero in
// registers and the discarded half of the output is never stored, so the
// compiler prunes the corresponding butterflies.  Spectra use the paired
// layout of fft_common.cuh, which keeps q and -q in the same lane.
//
// One cluster of HB CTAs per plane; CTA h holds rows [h*n/HB, (h+1)*n/HB)
// of the tile u[ky][i] (ky = 1..n) in shared memory:
//   phase 1  y transform of its rows, form u(ky), store columns ky = 1..n
//   phase 2  its share of the columns: x transform, (1 - e_x P_x) g, inverse
//            x transform (column segments of other CTAs over DSMEM)
//   phase 3  its rows: rebuild the 2n-point y spectrum, inverse, crop, store
// ADJ runs the transposed chain (backward transforms first, conjugate phases).
#pragma once

#include <cooperative_groups.h>

#include "solver.cuh"

namespace cg = cooperative_groups;

namespace pp {

// tile slot of (column ky in 1..N, local row il)
template <typename Cfg>
__device__ __forceinline__ int tile_at(int ky, int il) {
  return (ky - 1) * Cfg::LD + (il ^ ((ky - 1) & Cfg::SWM));
}

// one kz plane; a cluster of HB CTAs of THREADS threads (HB = 1: one CTA)
template <typename T, int N, int HB, int THREADS, bool ADJ>
__device__ __forceinline__ void tsym_plane(const SolveArgs<T>& a, int kz, unsigned char* smem_raw) {
  using Cfg = TSymCfg<T, N, HB, THREADS>;
  using V = C2<T>;
  constexpr int L = 2 * N;
  constexpr int G = Cfg::G, E = Cfg::E, ROWS = Cfg::ROWS;
  constexpr int WARPS = THREADS / 32;
  constexpr int GPW = 32 / G;                 // groups per warp
  constexpr int GPC = WARPS * GPW;            // groups per CTA
  constexpr bool INV1 = ADJ;                  // direction of the padded forward transforms
  constexpr bool INV2 = !ADJ;                 // direction of the cropped inverse transforms
  constexpr int MASK = L - 1;

  V* ybuf = reinterpret_cast<V*>(smem_raw);                 // [N columns ky=1..N][LD]
  V* stw = ybuf + Cfg::YBUF;                                // L twiddles
  V* stwT = stw + L;                                        // the same, transposed
  V* sw2 = stwT + L;                                        // 2N phases w_{2N}^j
  V* scratch = sw2 + L + (threadIdx.x / G) * PairShape<L>::SSTRIDE;

  int h = 0;
  V* remote[HB];
  if constexpr (HB > 1) {
    cg::cluster_group cluster = cg::this_cluster();
    h = int(cluster.block_rank());
#pragma unroll
    for (int r = 0; r < HB; ++r) remote[r] = cluster.map_shared_rank(ybuf, r);
  } else {
    remote[0] = ybuf;
  }
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int t = lane % G;
  const int gw = lane / G;
  V* plane = a.work + size_t(kz) * N * N;
  const int sgn = ADJ ? 1 : -1;                             // e = w_{2N}^{sgn*s*k}

  for (int i = threadIdx.x; i < L; i += THREADS) {
    const V w = a.tw_t2[i];
    stw[i] = w;
    stwT[(i % G) * E + i / G] = w;
    sw2[i] = a.w2_t[i];
  }
  __syncthreads();

  // ------------------------------------------------------------------ phase 1
#pragma unroll 1
  for (int r0 = 0; r0 < ROWS; r0 += GPC) {
    const int il = r0 + warp + WARPS * gw;
    const bool act = il < ROWS;
    const int i = h * ROWS + (act ? il : 0);
    V v[E];
#pragma unroll
    for (int e = 0; e < E; ++e)
      v[e] = (e < E / 2 && act) ? plane[size_t(i) * N + t + G * e] : mk<V>(0, 0);
    fft_c2p<L, INV1, false>(v, scratch, stw, t);             // Y(q), paired
    apply_mirror_pairs<L>(v, t, [&](V self, V mir, int idx) {
      const int q = paired_q<L, false>(t, idx);
      return cfms(self, sw2[(sgn * a.sy * q) & MASK], mir); // u(q) = Y(q) - e_y(q) Y(-q)
    });
    if (act) {
#pragma unroll
      for (int idx = 0; idx < E; ++idx) {
        const int q = paired_q<L, false>(t, idx);
        if (q >= 1 && q <= N) ybuf[tile_at<Cfg>(q, il)] = v[idx];
      }
    }
  }
  if constexpr (HB > 1) cg::this_cluster().sync(); else __syncthreads();

  // ------------------------------------------------------------------ phase 2
  {
    constexpr int CPC = N / HB;                              // columns of this CTA
#pragma unroll 1
    for (int c0 = 0; c0 < CPC; c0 += GPC) {
      const int cl = c0 + warp + WARPS * gw;
      const bool act = cl < CPC;
      const int ky = 1 + h * CPC + (act ? cl : 0);           // 1..N
      V v[E];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        if (e < E / 2) {
          const int i = t + G * e;
          const int hh = i / ROWS;
          v[e] = act ? remote[hh][tile_at<Cfg>(ky, i - hh * ROWS)] : mk<V>(0, 0);
        } else {
          v[e] = mk<V>(0, 0);
        }
      }
      fft_c2p<L, INV1, false>(v, scratch, stw, t);           // X(kx, ky), paired
      const T* grow = a.green + (size_t(kz) * (N + 1) + ky) * (N + 1);
      apply_mirror_pairs<L>(v, t, [&](V self, V mir, int idx) {
        const int kx = paired_q<L, false>(t, idx);
        const int akx = kx <= N ? kx : L - kx;
        const T g = act ? __ldg(&grow[akx]) : T(0);
        return cscale(cfms(self, sw2[(sgn * a.sx * kx) & MASK], mir), g);   // (1 - e_x P_x) g
      });
      fft_p2c<L, INV2, false>(v, scratch, stwT, t);          // column, rows i = t + G e
      if (act) {
#pragma unroll
        for (int e = 0; e < E / 2; ++e) {
          const int i = t + G * e;
          const int hh = i / ROWS;
          remote[hh][tile_at<Cfg>(ky, i - hh * ROWS)] = v[e];
        }
      }
    }
  }
  if constexpr (HB > 1) cg::this_cluster().sync(); else __syncthreads();

  // ------------------------------------------------------------------ phase 3
#pragma unroll 1
  for (int r0 = 0; r0 < ROWS; r0 += GPC) {
    const int il = r0 + warp + WARPS * gw;
    const bool act = il < ROWS;
    const int i = h * ROWS + (act ? il : 0);
    V v[E];
#pragma unroll
    for (int idx = 0; idx < E; ++idx) {
      const int q = paired_q<L, false>(t, idx);
      const int qq = q <= N ? q : L - q;                     // 0..N
      V val = (act && qq >= 1) ? ybuf[tile_at<Cfg>(qq, il)] : mk<V>(0, 0);
      if (q > N) {                                           // Phi(-ky) = -conj(e_y(ky)) Phi(ky)
        const V ey = sw2[(sgn * a.sy * qq) & MASK];
        val = mk<V>(-(val.x * ey.x + val.y * ey.y), -(val.y * ey.x - val.x * ey.y));
      }
      v[idx] = val;
    }
    fft_p2c<L, INV2, false>(v, scratch, stwT, t);
    if (act) {
#pragma unroll
      for (int e = 0; e < E / 2; ++e) plane[size_t(i) * N + t + G * e] = v[e];
    }
  }
  if constexpr (HB > 1) cg::this_cluster().sync();
}

// ---------------------------------------------------------------------------
// The same plane with the cyclic-layout group FFT (16-lane groups for 2n =
// 256, E = 16 values per lane) and the mirrors fetched by shuffles: about 10 %
// more instructions than the paired layout, but about half the registers, so
// a 512-thread CTA (16 warps) fits one SM.  HB = 1 only.
// ---------------------------------------------------------------------------
template <typename T, int N, int THREADS>
struct TCycCfg {
  static constexpr int L = 2 * N;
  using S = GroupShape<L>;
  static constexpr int G = S::G;
  static constexpr int E = S::E;
  static constexpr int ROWS = N;
  static constexpr int LD = N;
  static constexpr int SWM = (N < 16 ? N : 16) - 1;
  static constexpr int YBUF = N * LD;
  static constexpr int GROUPS = THREADS / G;
  static constexpr size_t smem_bytes() {
    return sizeof(C2<T>) * (size_t(YBUF) + size_t(L) + size_t(GROUPS) * S::SSTRIDE);
  }
};

template <typename T, int N, int THREADS, bool ADJ>
__device__ __forceinline__ void tsym_cyc_plane(const SolveArgs<T>& a, int kz, unsigned char* smem_raw) {
  using Cfg = TCycCfg<T, N, THREADS>;
  using V = C2<T>;
  constexpr int L = 2 * N;
  constexpr int G = Cfg::G, E = Cfg::E;
  constexpr int WARPS = THREADS / 32;
  constexpr int GPW = 32 / G;
  constexpr int GPC = WARPS * GPW;
  constexpr bool INV1 = ADJ, INV2 = !ADJ;
  constexpr int MASK = L - 1;
  V* ybuf = reinterpret_cast<V*>(smem_raw);
  V* sw2 = ybuf + Cfg::YBUF;                                   // 2N phases w_{2N}^j
  V* scratch = sw2 + L + (threadIdx.x / G) * GroupShape<L>::SSTRIDE;
  const V* tw = a.tw_t2c;     // group_fft reads its twiddles from global memory (__ldg)
  auto tile = [](int ky, int il) { return (ky - 1) * Cfg::LD + (il ^ ((ky - 1) & Cfg::SWM)); };
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int t = lane % G;
  const int gw = lane / G;
  V* plane = a.work + size_t(kz) * N * N;
  const int sgn = ADJ ? 1 : -1;

  for (int i = threadIdx.x; i < L; i += THREADS) sw2[i] = a.w2_t[i];
  __syncthreads();

  // phase 1: rows
#pragma unroll 1
  for (int r0 = 0; r0 < N; r0 += GPC) {
    const int il = r0 + warp + WARPS * gw;
    const bool act = il < N;
    const int i = act ? il : 0;
    V v[E];
#pragma unroll
    for (int e = 0; e < E; ++e)
      v[e] = (e < E / 2 && act) ? plane[size_t(i) * N + t + G * e] : mk<V>(0, 0);
    group_fft<L, INV1>(v, scratch, tw, t);                     // Y(q), q = t + G e
    V m[E];
    mirror_fetch<L>(v, m, t, 0, lane - t);                      // Y(-q)
    if (act) {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int q = t + G * e;
        if (q >= 1 && q <= N) ybuf[tile(q, il)] = cfms(v[e], sw2[(sgn * a.sy * q) & MASK], m[e]);
      }
    }
  }
  __syncthreads();

  // phase 2: columns ky = 1..N
#pragma unroll 1
  for (int c0 = 0; c0 < N; c0 += GPC) {
    const int cl = c0 + warp + WARPS * gw;
    const bool act = cl < N;
    const int ky = 1 + (act ? cl : 0);
    V v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = (e < E / 2 && act) ? ybuf[tile(ky, t + G * e)] : mk<V>(0, 0);
    group_fft<L, INV1>(v, scratch, tw, t);                     // X(kx), kx = t + G e
    V m[E];
    mirror_fetch<L>(v, m, t, 0, lane - t);                      // X(-kx)
    const T* grow = a.green + (size_t(kz) * (N + 1) + ky) * (N + 1);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int kx = t + G * e;
      const int akx = kx <= N ? kx : L - kx;
      const T g = act ? __ldg(&grow[akx]) : T(0);
      v[e] = cscale(cfms(v[e], sw2[(sgn * a.sx * kx) & MASK], m[e]), g);
    }
    group_fft<L, INV2>(v, scratch, tw, t);                     // column, rows i = t + G e
    if (act) {
#pragma unroll
      for (int e = 0; e < E / 2; ++e) ybuf[tile(ky, t + G * e)] = v[e];
    }
  }
  __syncthreads();

  // phase 3: rows
#pragma unroll 1
  for (int r0 = 0; r0 < N; r0 += GPC) {
    const int il = r0 + warp + WARPS * gw;
    const bool act = il < N;
    const int i = act ? il : 0;
    V v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int q = t + G * e;
      const int qq = q <= N ? q : L - q;
      V val = (act && qq >= 1) ? ybuf[tile(qq, i)] : mk<V>(0, 0);
      if (q > N) {
        const V ey = sw2[(sgn * a.sy * qq) & MASK];
        val = mk<V>(-(val.x * ey.x + val.y * ey.y), -(val.y * ey.x - val.x * ey.y));
      }
      v[e] = val;
    }
    group_fft<L, INV2>(v, scratch, tw, t);
    if (act) {
#pragma unroll
      for (int e = 0; e < E / 2; ++e) plane[size_t(i) * N + t + G * e] = v[e];
    }
  }
}

}  // namespace pp
