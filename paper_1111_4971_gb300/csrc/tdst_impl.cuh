// Pipe-operator transverse stage for cell-centred meshes (x0 = hx/2,
// y0 = hy/2, mesh spanning the pipe): the same operator as tsym_impl.cuh, with
// every padded 2N-point transform replaced by an N-point one.
//
// Why this is the same operator.  Along one transverse axis the stage forms,
// from the N physical samples x_j of a line, the combination
//     U(q) = Y(q) - w^{-s q} Y(-q),   q = 1..N,
// where Y is the 2N-point transform of the zero-padded line, w = e^{-i pi/N}
// (conjugated for the adjoint) and s = 2 x0 / h is the image offset of the
// correlation terms of Eq. 10 (the reflections R_t).  For s = 1, U is the
// 2N-point transform of the antisymmetric extension z_j = x_j,
// z_{2N-1-j} = -x_j.  Splitting z into even and odd samples and using the
// antisymmetry turns the odd half into the even half reversed, so with
//     v_n = z_{2n}  (x_{2n} for 2n < N, -x_{2N-1-2n} otherwise),
//     V = N-point transform of v,
// one has U(q) = V(q) - w^{-q} V(N-q) for q = 1..N-1 and U(N) = 2 V(0).
// The inverse direction is the transpose: a spectrum with P(-q) = -w^q P(q)
// (what the Green product of Eq. 10 leaves, the table being even in q) has
// as its 2N-point inverse transform a sequence antisymmetric in the same
// sense, whose even samples are the N-point inverse transform of
//     V'(q) = P(q) + w^{-q} P(N-q),  V'(0) = P(N),
// and whose odd samples 2n+1 are minus the even sample 2(N-1-n).  Each line
// therefore costs one N-point transform plus a mirror combination of the
// pairs (q, N-q), instead of a 2N-point transform with half its inputs zero.
//
// Layout and schedule are those of the cyclic 2N-point routine: one CTA per
// kz plane, lanes of a group of G hold elements q = t + G e; pass 1 transforms
// the N rows along y into the ky = 1..N columns of a shared-memory buffer,
// pass 2 transforms each column along x, multiplies by the Green octant,
// transforms back and stores it in place, pass 3 transforms the rows back.
#pragma once

#include "fft_common.cuh"
#include "solver.cuh"

namespace pp {

// GB: the plane buffer in a global scratch plane (a.tbuf, L2-resident)
// instead of shared memory, for planes too large for it (FP64 128 x 128)
template <typename T, int N, int THREADS, bool GB = false>
struct TDstCfg {
  using S = GroupShape<N>;
  static constexpr int G = S::G;
  static constexpr int E = S::E;
  static constexpr int LD = N;
  static constexpr int SWM = (N < 16 ? N : 16) - 1;
  static constexpr int YBUF = N * LD;
  static constexpr int GROUPS = THREADS / G;
  static constexpr size_t smem_bytes() {
    return sizeof(C2<T>) * ((GB ? 0 : size_t(YBUF)) + size_t(2 * N) + size_t(GROUPS) * S::SSTRIDE);
  }
};

// a + w * b
template <typename V>
__device__ __forceinline__ V cfma_(V a, V w, V b) {
  return mk<V>(a.x + (w.x * b.x - w.y * b.y), a.y + (w.x * b.y + w.y * b.x));
}

// H16 (complex-FP16 spectra, FP32 arithmetic): the plane is read as __half2
// with the z-forward tile scales, the Green product is taken in FP16 with one
// scale per column for each operand, and the result is stored as __half2
// with one scale per row (a.tscale).
template <typename T, int N, int THREADS, bool ADJ, bool H16 = false, bool GB = false>
struct TDst {
  using Cfg = TDstCfg<T, N, THREADS, GB>;
  using V = C2<T>;
  static constexpr int G = Cfg::G, E = Cfg::E, H = E / 2;
  static constexpr int WARPS = THREADS / 32;
  static constexpr int GPW = 32 / G;
  static constexpr int GPC = WARPS * GPW;                      // lines in flight per CTA
  static constexpr bool INV1 = ADJ, INV2 = !ADJ;
  static constexpr int MASK = 2 * N - 1;
  static constexpr int SGN = ADJ ? 1 : -1;                     // w^{-q} = sw2[(SGN q) mod 2N]

  V* ybuf;
  V* sw2;                                                      // 2N phases w_{2N}^j
  V* scratch;
  const V* tw;                // N-point twiddles, read by group_fft from global memory
  int lane, t, line;

  __device__ __forceinline__ TDst(const SolveArgs<T>& a, unsigned char* smem_raw) {
    ybuf = reinterpret_cast<V*>(smem_raw);           // (GB: set per plane)
    sw2 = GB ? ybuf : ybuf + Cfg::YBUF;
    scratch = sw2 + 2 * N + (threadIdx.x / G) * GroupShape<N>::SSTRIDE;
    tw = a.tw_t;
    lane = threadIdx.x & 31;
    t = lane % G;
    line = lane / G + GPW * (threadIdx.x >> 5);                // groups of a warp: adjacent lines
  }

  // the plane buffer [ky-1][i] with row i XOR-swizzled by a function of ky
  // whose bit 0 alternates with ky and whose bits 1-3 differ over any 8
  // consecutive ky: conflict-free (two wavefronts per warp access) for the
  // row stores, the column loads / stores and both last-pass loads
  __device__ static __forceinline__ int tile(int ky, int il) {
    const int x = ky - 1;
    return x * Cfg::LD + (il ^ (((2 * x) & Cfg::SWM & ~1) | (x & 1)));
  }

  // the even/odd-split samples v_n of row il (row 0 stands in past the end)
  __device__ __forceinline__ void load_row(const V* plane, int il, V (&v)[E]) const {
    const V* row = plane + size_t(il < N ? il : 0) * N;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int n = t + G * e;
      if (e < H) {
        v[e] = row[2 * n];
      } else {
        const V x = row[2 * N - 1 - 2 * n];
        v[e] = mk<V>(-x.x, -x.y);
      }
    }
  }

  // max over the G lanes of one group (consecutive lanes)
  __device__ static __forceinline__ float group_max(float x) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
  }

  // load_row for complex-FP16 planes: values times their z-tile scale
  __device__ __forceinline__ void load_row16(const SolveArgs<T>& a, int kz, int il, V (&v)[E]) const {
    const int i = il < N ? il : 0;
    const __half2* row = reinterpret_cast<const __half2*>(a.work) + (size_t(kz) * N + i) * N;
    const float* zs = a.zscale;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int n = t + G * e;
      const int j = e < H ? 2 * n : 2 * N - 1 - 2 * n;
      const float2 f = __half22float2(row[j]);
      const float sc = __ldg(&zs[(i * N + j) / a.zcols]) * (e < H ? 1.f : -1.f);
      v[e] = mk<V>(T(f.x * sc), T(f.y * sc));
    }
  }

  // the phase table; the caller synchronises before the first plane
  __device__ __forceinline__ void load_tables(const SolveArgs<T>& a) {
    for (int i = threadIdx.x; i < 2 * N; i += THREADS) sw2[i] = a.w2_t[i];
  }

  // Plane kz in place (the phase table already loaded and synchronised).
  // Ends with the plane's stores issued; the caller synchronises before
  // another plane reuses the buffers.
  __device__ __forceinline__ void plane(const SolveArgs<T>& a, int kz) {
    V* pl = a.work + size_t(kz) * N * N;
    if constexpr (GB) ybuf = a.tbuf + size_t(kz) * N * N;
    V ph[E];                                                   // w^{-q} of this lane's slots
#pragma unroll
    for (int e = 0; e < E; ++e) ph[e] = sw2[(SGN * (t + G * e)) & MASK];
    // the group-FFT twiddles of this lane, in registers when they fit (at
    // most 256 threads), else read from the table at each transform
    constexpr bool RTW = THREADS <= 256 && !GB;
    V twr[RTW ? E : 1];
    if constexpr (RTW) {
#pragma unroll
      for (int k1 = 0; k1 < E; ++k1) twr[k1] = __ldg(&tw[k1 * G + t]);
    }
    auto fft = [&](auto inv, V (&x)[E]) {
      if constexpr (RTW) group_fft_r<N, decltype(inv)::value>(x, scratch, twr, t);
      else group_fft<N, decltype(inv)::value>(x, scratch, tw, t);
    };
    using Fwd = std::integral_constant<bool, INV1>;
    using Bwd = std::integral_constant<bool, INV2>;

    // pass 1: rows i, along y -> ybuf[ky][i], ky = 1..N
#pragma unroll 1
    for (int r0 = 0; r0 < N; r0 += GPC) {
      const int il = r0 + line;
      V v[E];
      if constexpr (H16) load_row16(a, kz, il, v);
      else load_row(pl, il, v);
      fft(Fwd{}, v);                   // V(q)
      V m[E];
      mirror_fetch<N>(v, m, t, 0, lane - t);                   // V(N-q)
      if (il < N) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int q = t + G * e;
          if (q == 0) ybuf[tile(N, il)] = mk<V>(v[e].x + v[e].x, v[e].y + v[e].y);
          else ybuf[tile(q, il)] = cfms(v[e], ph[e], m[e]);
        }
      }
    }
    __syncthreads();

    // pass 2: columns ky = 1..N, along x, Green product, back along x
#pragma unroll 1
    for (int c0 = 0; c0 < N; c0 += GPC) {
      const int cl = c0 + line;
      const bool act = cl < N;
      const int ky = 1 + (act ? cl : 0);
      V u[E];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int n = t + G * e;
        if (e < H) {
          u[e] = ybuf[tile(ky, 2 * n)];
        } else {
          const V x = ybuf[tile(ky, 2 * N - 1 - 2 * n)];
          u[e] = mk<V>(-x.x, -x.y);
        }
      }
      const T* grow = a.green + (size_t(kz) * (N + 1) + ky) * (N + 1);
      T gpre[E];                       // the Green row, read before the transform
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int kx = t + G * e;
        gpre[e] = act ? __ldg(&grow[kx == 0 ? N : kx]) : T(0);
      }
      fft(Fwd{}, u);                   // V(kx)
      V m[E];
      mirror_fetch<N>(u, m, t, 0, lane - t);
      if constexpr (!H16) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int kx = t + G * e;
          const T g = gpre[e];
          // slot 0 carries kx = N: U(N) = 2 V(0)
          const V w = (kx == 0) ? mk<V>(u[e].x + u[e].x, u[e].y + u[e].y)
                                : cfms(u[e], ph[e], m[e]);
          u[e] = cscale(w, g);                                 // P(kx)
        }
      } else {
        // complex-FP16 product: both operands scaled per column so that
        // their largest magnitude is 2^7 (the product stays below 2^14)
        float g[E];
        float mu = 0.f, mg = 0.f;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int kx = t + G * e;
          g[e] = float(gpre[e]);
          u[e] = (kx == 0) ? mk<V>(u[e].x + u[e].x, u[e].y + u[e].y)
                           : cfms(u[e], ph[e], m[e]);
          mu = fmaxf(mu, fmaxf(fabsf(float(u[e].x)), fabsf(float(u[e].y))));
          mg = fmaxf(mg, fabsf(g[e]));
        }
        mu = group_max(mu);
        mg = group_max(mg);
        const float su = mu > 0.f ? mu * (1.f / 128.f) : 1.f, sg = mg > 0.f ? mg * (1.f / 128.f) : 1.f;
        const float iu = 1.f / su, ig = 1.f / sg, back = su * sg;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const __half2 uh = __floats2half2_rn(float(u[e].x) * iu, float(u[e].y) * iu);
          const __half2 ph = __hmul2(uh, __float2half2_rn(g[e] * ig));
          const float2 pf = __half22float2(ph);
          u[e] = mk<V>(T(pf.x * back), T(pf.y * back));       // P(kx)
        }
      }
      mirror_fetch<N>(u, m, t, 0, lane - t);                   // P(N-kx)
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int q = t + G * e;
        if (q != 0) u[e] = cfma_(u[e], ph[e], m[e]);   // V'(q); V'(0) = P(N)
      }
      fft(Bwd{}, u);                   // even samples 2n of the column
      if (act) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int n = t + G * e;
          if (e < H) ybuf[tile(ky, 2 * n)] = u[e];
          else ybuf[tile(ky, 2 * N - 1 - 2 * n)] = mk<V>(-u[e].x, -u[e].y);
        }
      }
    }
    __syncthreads();

    // pass 3: rows i, back along y
#pragma unroll 1
    for (int r0 = 0; r0 < N; r0 += GPC) {
      const int il = r0 + line;
      const int i = il < N ? il : 0;
      V u[E];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int q = t + G * e;
        if (q == 0) {
          u[e] = ybuf[tile(N, i)];                             // V'(0) = P(N)
        } else {
          const V p = ybuf[tile(q, i)];
          const V pm = ybuf[tile(N - q, i)];
          u[e] = cfma_(p, ph[e], pm);
        }
      }
      fft(Bwd{}, u);
      if constexpr (H16) {
        float mx = 0.f;
#pragma unroll
        for (int e = 0; e < E; ++e) mx = fmaxf(mx, fmaxf(fabsf(float(u[e].x)), fabsf(float(u[e].y))));
        mx = group_max(mx);
        const float sc = mx > 0.f ? mx * (1.f / 16384.f) : 1.f, inv = 1.f / sc;
        if (il < N) {
          if (t == 0) a.tscale[size_t(kz) * N + i] = sc;
          __half2* out = reinterpret_cast<__half2*>(a.work) + (size_t(kz) * N + i) * N;
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int n = t + G * e;
            const float sg = e < H ? inv : -inv;
            out[e < H ? 2 * n : 2 * N - 1 - 2 * n] = __floats2half2_rn(float(u[e].x) * sg, float(u[e].y) * sg);
          }
        }
      } else if (il < N) {
        V* out = pl + size_t(i) * N;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int n = t + G * e;
          if (e < H) out[2 * n] = u[e];
          else out[2 * N - 1 - 2 * n] = mk<V>(-u[e].x, -u[e].y);
        }
      }
    }
  }
};

// one plane
template <typename T, int N, int THREADS, bool ADJ, bool H16 = false, bool GB = false>
__device__ __forceinline__ void tdst_plane(const SolveArgs<T>& a, int kz, unsigned char* smem_raw) {
  TDst<T, N, THREADS, ADJ, H16, GB> r(a, smem_raw);
  r.load_tables(a);
  __syncthreads();
  r.plane(a, kz);
}

}  // namespace pp
