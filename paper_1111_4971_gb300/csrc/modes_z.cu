// FP32 z convolution of the mode-space solve, one warp-level FFT per mode
// column: the same steps as mode_z (modes_impl.cuh) -- the packed 2nz-point
// real transform of Appendix A (Eq. A.1-A.4) as an L = nz point complex FFT,
// the real-spectrum unpack, the product with the kernel spectrum g and the
// packed inverse -- with each column's L points held in the registers of S
// lanes (E = L / S points a lane, S = 2^floor(log2 L / 2)) instead of a CTA's
// shared memory.
//
// Four-step transform (L = S * E).  Lane b of a column holds the points
// m = b + S a (a < E).  Then, with k = k1 + E k2,
//   X(k1 + E k2) = sum_b w_S^{b k2} [ w_L^{b k1} sum_a x(b + S a) w_E^{a k1} ],
// i.e. (1) an E-point DFT over a in each lane's registers, (2) the twiddle
// w_L^{b k1}, (3) a transpose through shared memory, after which lane l takes
// the rows k1 = l + S i (i < E / S) and (4) an S-point DFT over b for each.
// The inverse is the same with conjugate twiddles.  Only the first L/2 input
// points are nonzero (the zero padding), so the first DFT skips its upper
// half; only the first L/2 outputs of the inverse are kept (psi is the first
// nz of the 2nz-point result), so the last DFT computes only those.  Between
// the two transforms the spectrum goes to shared memory in natural order and
// each lane forms, for its points k = b + S a (into a second buffer, read back
// in the layout of the inverse's input),
//   Y(k)    = g(k)     [Z(k) + conj Z(L-k) - i w^k (Z(k) - conj Z(L-k))] / 2,
//   Y(L-k)  = g(L-k)   [Z(L-k) + conj Z(k) - i w^{L-k} (Z(L-k) - conj Z(k))] / 2,
//   Z'(k)   = Y(k) + conj Y(L-k) + i w^{-k} (Y(k) - conj Y(L-k)),
// w = e^{-i pi / L}, Z(L) = Z(0).  Everything between the loads of the partial projections
// (summed over their groups) and the stores of psi is registers and one
// warp's shared memory: no block-wide barrier.
#include "modes.cuh"
#include "modes_impl.cuh"

namespace pp {

namespace {

constexpr int kZWarps = 2;                       // warps per CTA

constexpr int ilog2(int n) { return n > 1 ? 1 + ilog2(n / 2) : 0; }

template <int L>
struct ZWarpShape {
  static constexpr int LOG = ilog2(L);
  static constexpr int S = 1 << (LOG / 2);       // lanes per column
  static constexpr int E = L / S;                // points per lane (E >= S)
  static constexpr int CPW = 32 / S;             // columns per warp
  static constexpr int CB = E * (S + 1) + 1;     // complex values of a column's buffer
  // floats of the CTA's kernel spectra, rounded up to a whole number of
  // complex values
  static constexpr int GS = (kZWarps * CPW * (L + 1) + 1) / 2 * 2;
  static constexpr size_t SMEM = sizeof(float2) * (2 * size_t(L) + size_t(kZWarps) * CPW * 2 * CB) + sizeof(float) * GS;
};

// CTA `blk` of a solve: its columns blk * CPC ..
template <int L>
__device__ __forceinline__ void z_warp(const ModeArgs<float>& a, int groups, int blk) {
  using V = float2;
  using Sh = ZWarpShape<L>;
  constexpr int S = Sh::S, E = Sh::E, CPW = Sh::CPW;
  constexpr int CPC = kZWarps * CPW;             // columns per CTA
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sub = lane / S, b = lane % S;
  const int cl = warp * CPW + sub;               // column within the CTA
  const int col0 = blk * CPC;
  const int col = col0 + cl;
  const bool valid = col < a.mc;
  // shared memory: the stage-2 twiddles tw[k1][b] = w_L^{b k1}, the spectral
  // twiddles w^k (k < L), the CTA's kernel spectra g[c][k] (k <= L), then a
  // transpose buffer per column.  The tables arrive by cp.async together with
  // the columns' loads, so the kernel pays one memory latency, not one per step.
  V* tws = reinterpret_cast<V*>(smem_raw);       // [E][S]
  V* wks = tws + L;                              // [L]
  float* gs = reinterpret_cast<float*>(wks + L); // [CPC][L + 1]
  V* T = reinterpret_cast<V*>(gs + Sh::GS) + size_t(cl) * 2 * Sh::CB;   // two buffers a column
  const V* w2 = a.w2_z;                          // w2[j] = e^{-2 pi i j / (2L)}, j < 2L
  for (int i = int(threadIdx.x); i < L; i += 32 * kZWarps) {
    const int k1 = i / S, bb = i % S;
    cp_async8(tws + i, w2 + 2 * bb * k1);
  }
  for (int i = int(threadIdx.x); i < L / 2; i += 32 * kZWarps) cp_async16(wks + 2 * i, w2 + 2 * i);
  {
    const int nc = a.mc - col0 < CPC ? a.mc - col0 : CPC;
    const float* g0 = a.gz + size_t(col0) * (L + 1);
    for (int i = int(threadIdx.x); i < nc * (L + 1); i += 32 * kZWarps) cp_async4(gs + i, g0 + i);
  }
  cp_async_commit();

  // 1. the packed column z(m) = x(2m) + i x(2m+1), m = b + S a < L/2, summed
  //    over the groups of partial projections
  V v[E];
#pragma unroll
  for (int i = 0; i < E; ++i) v[i] = make_float2(0.f, 0.f);
  if (valid) {
#pragma unroll 4
    for (int s = 0; s < groups; ++s) {
      const V* src = reinterpret_cast<const V*>(a.part + (size_t(s) * a.mc + col) * L) + b;
#pragma unroll
      for (int i = 0; i < E / 2; ++i) {
        const V z = __ldg(src + S * i);
        v[i].x += z.x;
        v[i].y += z.y;
      }
    }
  }
  cp_async_wait<0>();
  __syncthreads();

  // 2. forward transform
  dft_reg<E, false>(v);                          // over a; inputs a >= E/2 are zero
#pragma unroll
  for (int k1 = 1; k1 < E; ++k1) v[k1] = cmul(v[k1], tws[k1 * S + b]);     // w_L^{b k1}
#pragma unroll
  for (int k1 = 0; k1 < E; ++k1) T[k1 * (S + 1) + b] = v[k1];
  __syncwarp();
#pragma unroll
  for (int i = 0; i < E / S; ++i) {
    V* u = v + i * S;
#pragma unroll
    for (int bb = 0; bb < S; ++bb) u[bb] = T[(b + S * i) * (S + 1) + bb];
    dft_reg<S, false>(u);                        // over b: X(k1 + E k2), k1 = b + S i
  }
  __syncwarp();
#pragma unroll
  for (int i = 0; i < E / S; ++i)
#pragma unroll
    for (int k2 = 0; k2 < S; ++k2) T[b + S * i + E * k2] = v[i * S + k2];
  __syncwarp();

  // 3. real spectrum, kernel product, packed inverse input Z'(k) into the
  //    column's second buffer, then back to registers in the layout of the
  //    inverse.  Each pair (k, L-k), k = b + S i < L/2, is formed once:
  //    with s = Y(k) + conj Y(L-k) and t = conj(w^k) (Y(k) - conj Y(L-k)),
  //    Z'(k) = s + i t and Z'(L-k) = conj(s) + i conj(t); lane b = 0 also
  //    takes the self-paired k = L/2.  (A rolled loop: the code stays small
  //    enough for the instruction cache.)
  const float* g = gs + cl * (L + 1);
  V* U = T + Sh::CB;
  auto pair = [&](int k, bool both) {
    const V zk = T[k], zm = T[(L - k) & (L - 1)];
    const V wk = wks[k];                         // w^k
    const V wm = make_float2(-wk.x, wk.y);       // w^{L-k} = -conj(w^k)
    const float gk = valid ? g[k] : 0.f, gm = valid ? g[L - k] : 0.f;
    auto unpack = [](V x, V xm, V w) {           // (x + conj xm - i w (x - conj xm)) / 2
      const V c = cconj(xm);
      const V su = cadd(x, c), df = csub(x, c);
      const V wd = cmul(w, df);
      return make_float2(0.5f * (su.x + wd.y), 0.5f * (su.y - wd.x));
    };
    const V yk = cscale(unpack(zk, zm, wk), gk);
    const V ym = cscale(unpack(zm, zk, wm), gm);
    const V c = cconj(ym);
    const V sp = cadd(yk, c), d = csub(yk, c);
    const V t = cmulc<true>(d, wk);
    U[k] = make_float2(sp.x - t.y, sp.y + t.x);
    if (both) U[L - k] = make_float2(sp.x + t.y, t.x - sp.y);
  };
#pragma unroll 2
  for (int i = 0; i < E / 2; ++i) {
    const int k = b + S * i;
    pair(k, k != 0);
  }
  if (b == 0) pair(L / 2, false);
  __syncwarp();
#pragma unroll
  for (int i = 0; i < E; ++i) v[i] = U[b + S * i];

  // 4. inverse transform; the outputs m = k1 + E k2 < L/2 (k2 < S/2) are psi
  dft_reg<E, true>(v);
#pragma unroll
  for (int k1 = 1; k1 < E; ++k1) v[k1] = cmulc<true>(v[k1], tws[k1 * S + b]);
#pragma unroll
  for (int k1 = 0; k1 < E; ++k1) T[k1 * (S + 1) + b] = v[k1];
  __syncwarp();
  V* dst = reinterpret_cast<V*>(a.psi + size_t(valid ? col : 0) * L);
#pragma unroll
  for (int i = 0; i < E / S; ++i) {
    V* u = v + i * S;
#pragma unroll
    for (int bb = 0; bb < S; ++bb) u[bb] = T[(b + S * i) * (S + 1) + bb];
    dft_reg<S, true>(u);
    if (valid) {
#pragma unroll
      for (int k2 = 0; k2 < S / 2; ++k2) dst[b + S * i + E * k2] = u[k2];
    }
  }
}

template <int L>
__global__ void __launch_bounds__(32 * kZWarps) mode_z_warp_kernel(ModeArgs<float> a, int groups) {
  z_warp<L>(a, groups, int(blockIdx.x));
}

// a group of solves of one shape: solve s takes the CTAs s * cps .. (s + 1) * cps - 1
template <int L>
__global__ void __launch_bounds__(32 * kZWarps) mode_z_warp_group_kernel(const __grid_constant__ ModeGroup g,
                                                                          int groups, int cps) {
  const int s = int(blockIdx.x) / cps;
  const ModeArgs<float> a = g.args[s];
  z_warp<L>(a, groups, int(blockIdx.x) % cps);
}

template <int L>
cudaError_t launch_zw(const ModeArgs<float>& a, int groups, const ModeGroup* g, cudaStream_t st) {
  using Sh = ZWarpShape<L>;
  const int per = kZWarps * Sh::CPW;             // columns per CTA
  const int cps = (a.mc + per - 1) / per;        // CTAs per solve
  void (*kern)(ModeArgs<float>, int) = mode_z_warp_kernel<L>;
  void (*gkern)(const ModeGroup, int, int) = mode_z_warp_group_kernel<L>;
  if (Sh::SMEM > 48 * 1024) {
    const cudaError_t e = g ? cudaFuncSetAttribute(gkern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Sh::SMEM))
                            : cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Sh::SMEM));
    if (e != cudaSuccess) return e;
  }
  if (g) gkern<<<g->n * cps, 32 * kZWarps, Sh::SMEM, st>>>(*g, groups, cps);
  else kern<<<cps, 32 * kZWarps, Sh::SMEM, st>>>(a, groups);
  return cudaGetLastError();
}

cudaError_t launch_zw_any(const ModeArgs<float>& a, int groups, const ModeGroup* g, cudaStream_t st) {
  switch (a.nz) {
    case 32: return launch_zw<32>(a, groups, g, st);
    case 64: return launch_zw<64>(a, groups, g, st);
    case 128: return launch_zw<128>(a, groups, g, st);
    case 256: return launch_zw<256>(a, groups, g, st);
    case 512: return launch_zw<512>(a, groups, g, st);
    case 1024: return launch_zw<1024>(a, groups, g, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_mode_z_warp(const ModeArgs<float>& a, int groups, cudaStream_t st) {
  return launch_zw_any(a, groups, nullptr, st);
}

cudaError_t launch_mode_z_warp_group(const ModeArgs<float>& a, int groups, const ModeGroup& g, cudaStream_t st) {
  if (g.n < 1 || g.n > kMaxModeGroup) return cudaErrorInvalidValue;
  return launch_zw_any(a, groups, &g, st);
}

}  // namespace pp
