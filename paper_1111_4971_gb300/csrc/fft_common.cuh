// Device-side FFT building blocks for the pipe Poisson solver (sm_103a).
//
// Everything the solver transforms is reduced to complex FFTs of a power-of-two
// length L <= 1024 computed by a *group* of G consecutive lanes of one warp,
// each lane holding E = L/G elements in registers:
//
//   lane t holds x[t + G*e], e = 0..E-1          (the "cyclic" layout)
//
// The group FFT is the four-step factorisation L = E x G:
//   A. an E-point DFT in registers over e                 (compile-time twiddles)
//   B. multiply by w_L^{t*k1}                              (table, layout [k1][t])
//   C. transpose through a padded shared-memory tile, then a G-point DFT in
//      registers for each k1 = t + G*j.
// Input and output are both in the cyclic layout, so transforms chain without
// reshuffling.  One shared-memory round trip per FFT.
//
// Conventions: forward = sum_n a_n e^{-2 pi i nk/L}; INV selects e^{+}; nothing
// is normalised (the solver folds every 1/L into the Green spectrum).
#pragma once

#include <cuda_fp16.h>

#include <cuda_runtime.h>
#include <cstdint>
#include <type_traits>

namespace pp {

// ---------------------------------------------------------------------------
// complex helpers (float2 / double2)
// ---------------------------------------------------------------------------
template <typename T> struct cplx_t;
template <> struct cplx_t<float> { using type = float2; };
template <> struct cplx_t<double> { using type = double2; };
template <typename T> using C2 = typename cplx_t<T>::type;

template <typename V> struct real_of;
template <> struct real_of<float2> { using type = float; };
template <> struct real_of<double2> { using type = double; };

template <typename V> __host__ __device__ __forceinline__ V mk(typename real_of<V>::type x,
                                                              typename real_of<V>::type y) {
  V r; r.x = x; r.y = y; return r;
}
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return mk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return mk<V>(a.x - b.x, a.y - b.y); }
// FP32: one packed instruction for both parts (sm_100 and later; each half
// rounds as the scalar add, so the results are the same bits)
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) {
  float2 d;
  asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
  float2 d;
  asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
template <typename V> __device__ __forceinline__ V cconj(V a) { return mk<V>(a.x, -a.y); }
template <typename V> __device__ __forceinline__ V cscale(V a, typename real_of<V>::type s) {
  return mk<V>(a.x * s, a.y * s);
}
// a * b
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  return mk<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b) when CONJ, else a * b
template <bool CONJ, typename V> __device__ __forceinline__ V cmulc(V a, V b) {
  if constexpr (CONJ) return mk<V>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
  else return cmul(a, b);
}
// a - w * b
template <typename V> __device__ __forceinline__ V cfms(V a, V w, V b) {
  return mk<V>(a.x - (w.x * b.x - w.y * b.y), a.y - (w.x * b.y + w.y * b.x));
}

// ---------------------------------------------------------------------------
// compile-time twiddles: cos / sin of 2 pi k / n.  Octant reduction with exact
// integer arithmetic, then Taylor series on [0, pi/4] (error < 1e-28).
// ---------------------------------------------------------------------------
constexpr double kPi = 3.141592653589793238462643383279502884;

constexpr double taylor_sin(double x) {
  double x2 = x * x, term = x, sum = x;
  for (int i = 1; i < 14; ++i) {
    term *= -x2 / double((2 * i) * (2 * i + 1));
    sum += term;
  }
  return sum;
}
constexpr double taylor_cos(double x) {
  double x2 = x * x, term = 1.0, sum = 1.0;
  for (int i = 1; i < 14; ++i) {
    term *= -x2 / double((2 * i - 1) * (2 * i));
    sum += term;
  }
  return sum;
}
// (cos, sin)(2 pi k / n) into c, s
constexpr void cossin2pi(long k, long n, double& c, double& s) {
  k %= n;
  if (k < 0) k += n;
  const long o = (8 * k) / n;                 // octant
  const double q = kPi / 4.0;
  const double phi = double(8 * k - o * n) / double(n) * q;          // in [0, pi/4)
  const double psi = double((o + 1) * n - 8 * k) / double(n) * q;    // pi/4 - phi
  switch (o) {
    case 0: c = taylor_cos(phi); s = taylor_sin(phi); break;
    case 1: c = taylor_sin(psi); s = taylor_cos(psi); break;
    case 2: c = -taylor_sin(phi); s = taylor_cos(phi); break;
    case 3: c = -taylor_cos(psi); s = taylor_sin(psi); break;
    case 4: c = -taylor_cos(phi); s = -taylor_sin(phi); break;
    case 5: c = -taylor_sin(psi); s = -taylor_cos(psi); break;
    case 6: c = taylor_sin(phi); s = -taylor_cos(phi); break;
    default: c = taylor_cos(psi); s = -taylor_sin(psi); break;
  }
}
constexpr double ccos2pi(long k, long n) { double c = 0, s = 0; cossin2pi(k, n, c, s); return c; }
constexpr double csin2pi(long k, long n) { double c = 0, s = 0; cossin2pi(k, n, c, s); return s; }

// multiply v by the compile-time twiddle e^{-+ 2 pi i K / N}
template <int N, int K, bool INV, typename V>
__device__ __forceinline__ V twiddle_const(V v) {
  using R = typename real_of<V>::type;
  constexpr int k = ((K % N) + N) % N;
  if constexpr (k == 0) {
    return v;
  } else if constexpr (4 * k == N) {          // -i (forward) / +i (inverse)
    return INV ? mk<V>(-v.y, v.x) : mk<V>(v.y, -v.x);
  } else if constexpr (2 * k == N) {
    return mk<V>(-v.x, -v.y);
  } else if constexpr (4 * k == 3 * N) {
    return INV ? mk<V>(v.y, -v.x) : mk<V>(-v.y, v.x);
  } else if constexpr (8 * k == N || 8 * k == 3 * N || 8 * k == 5 * N || 8 * k == 7 * N) {
    constexpr R r = R(0.70710678118654752440084436210484903928);
    constexpr R c = R(ccos2pi(k, N) >= 0 ? 1.0 : -1.0) * r;
    constexpr R s = R((INV ? 1.0 : -1.0) * (csin2pi(k, N) >= 0 ? 1.0 : -1.0)) * r;
    return mk<V>(v.x * c - v.y * s, v.x * s + v.y * c);
  } else {
    constexpr R c = R(ccos2pi(k, N));
    constexpr R s = R((INV ? 1.0 : -1.0) * csin2pi(k, N));
    return mk<V>(v.x * c - v.y * s, v.x * s + v.y * c);
  }
}

template <int I, int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, N>(f);
  }
}

// ---------------------------------------------------------------------------
// In-register DFT of N points on x[0..N-1], natural order in and out.
// Radix-4 decimation in time (radix-2 for an odd power of two at the top);
// every index and twiddle is a compile-time constant.
// ---------------------------------------------------------------------------
template <int N, bool INV, typename V>
__device__ __forceinline__ void dft_reg(V* x) {
  if constexpr (N == 1) {
    return;
  } else if constexpr (N == 2) {
    V a = x[0], b = x[1];
    x[0] = cadd(a, b);
    x[1] = csub(a, b);
  } else if constexpr (N == 4) {
    V s0 = cadd(x[0], x[2]), d0 = csub(x[0], x[2]);
    V s1 = cadd(x[1], x[3]), d1 = csub(x[1], x[3]);
    V d1r = twiddle_const<4, 1, INV>(d1);
    x[0] = cadd(s0, s1);
    x[2] = csub(s0, s1);
    x[1] = cadd(d0, d1r);
    x[3] = csub(d0, d1r);
  } else if constexpr ((N & 0x55555555) != 0) {      // N = 4^k: radix 4
    constexpr int Q = N / 4;
    V a[4][Q];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int i = 0; i < Q; ++i) a[r][i] = x[4 * i + r];
#pragma unroll
    for (int r = 0; r < 4; ++r) dft_reg<Q, INV>(a[r]);
    static_for<0, Q>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      V y0 = a[0][k];
      V y1 = twiddle_const<N, k, INV>(a[1][k]);
      V y2 = twiddle_const<N, 2 * k, INV>(a[2][k]);
      V y3 = twiddle_const<N, 3 * k, INV>(a[3][k]);
      V s0 = cadd(y0, y2), d0 = csub(y0, y2);
      V s1 = cadd(y1, y3), d1 = twiddle_const<4, 1, INV>(csub(y1, y3));
      x[k] = cadd(s0, s1);
      x[k + 2 * Q] = csub(s0, s1);
      x[k + Q] = cadd(d0, d1);
      x[k + 3 * Q] = csub(d0, d1);
    });
  } else {                                             // N = 2 * 4^k: one radix-2 step
    constexpr int H = N / 2;
    V e[H], o[H];
#pragma unroll
    for (int i = 0; i < H; ++i) {
      e[i] = x[2 * i];
      o[i] = x[2 * i + 1];
    }
    dft_reg<H, INV>(e);
    dft_reg<H, INV>(o);
    static_for<0, H>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      V t = twiddle_const<N, k, INV>(o[k]);
      x[k] = cadd(e[k], t);
      x[k + H] = csub(e[k], t);
    });
  }
}

// ---------------------------------------------------------------------------
// Group FFTs with the "paired" spectral layout.
//
// L = E x G; a group of G lanes, lane t.  Time-domain data use the cyclic
// layout (lane t holds n = t + G*e).  Spectral data use the paired layout:
// lane t owns U = E/(2G) pairs of rows k1 of the E x G index grid
// q = k1 + E*k2, and for each owned row all G values k2, in
// v[(2j+s)*G + k2] (pair j, member s).  Rows are paired so that the mirror
// frequency of every element the lane holds is held by the same lane:
//   EVEN pairing (mirror q -> -q mod L):    rows {u, E-u}, u = t + G j; u = 0 -> {0, E/2}
//   ODD  pairing (mirror q -> L-1-q):       rows {u, E-1-u}
// ODD also selects the odd frequencies of the 2L-point transform of the
// zero-padded sequence: X(q) = sum_n x_n w_{2L}^{n(2q+1)}.  Its twist is
// split into a compile-time factor w_{2E}^{e} and a twiddle table
// tw_odd[k1][t] = w_{2L}^{t(2k1+1)}; the even table is tw_even[k1][t] = w_L^{t k1}.
// ---------------------------------------------------------------------------
template <int L> struct PairShape {
  static_assert(L >= 16 && L <= 512 && (L & (L - 1)) == 0, "FFT length");
  static constexpr int G = (L == 16) ? 2 : (L <= 64 ? 4 : (L <= 256 ? 8 : 16));
  static constexpr int E = L / G;
  static constexpr int U = E / (2 * G);               // row pairs per lane
  static_assert(U >= 1 && E % (2 * G) == 0, "paired shape");
  // padded scratch tile, complex elements per group; groups are spaced by
  // SSTRIDE so that two groups of one half-warp fall on different banks
  static constexpr int SCRATCH = E * (G + 1);
  static constexpr int SSTRIDE = SCRATCH + 8;
};

// row of member s of pair j held by lane t
template <int L, bool ODDP>
__device__ __forceinline__ int pair_row(int t, int j, int s) {
  constexpr int G = PairShape<L>::G, E = PairShape<L>::E;
  const int u = t + G * j;
  if constexpr (ODDP) {
    return s ? (E - 1 - u) : u;
  } else {
    if (u == 0) return s ? E / 2 : 0;
    return s ? (E - u) : u;
  }
}

// frequency index q of slot idx = (2j+s)*G + k2
template <int L, bool ODDP>
__device__ __forceinline__ int paired_q(int t, int idx) {
  constexpr int G = PairShape<L>::G, E = PairShape<L>::E;
  return pair_row<L, ODDP>(t, idx / (2 * G), (idx / G) & 1) + E * (idx % G);
}

// slot of the mirror of slot idx (compile-time idx): general rule, and the
// rule of the self-paired unit u = 0 of the EVEN pairing (lane 0, pair 0)
template <int L, int IDX>
struct MirrorSlot {
  static constexpr int G = PairShape<L>::G;
  static constexpr int j = IDX / (2 * G), s = (IDX / G) & 1, k2 = IDX % G;
  static constexpr int general = (2 * j + (1 - s)) * G + (G - 1 - k2);
  static constexpr int unit0 = (s == 0) ? (2 * j) * G + ((G - k2) % G) : (2 * j + 1) * G + (G - 1 - k2);
};

// cyclic time layout -> paired spectral layout.  tw: tw_even or tw_odd per ODDP.
template <int L, bool INV, bool ODDP, typename V>
__device__ __forceinline__ void fft_c2p(V (&v)[PairShape<L>::E], V* scratch, const V* tw, int t) {
  constexpr int G = PairShape<L>::G, E = PairShape<L>::E, U = PairShape<L>::U;
  if constexpr (ODDP) {
    static_for<1, E>([&](auto ec) {
      constexpr int e = decltype(ec)::value;
      v[e] = twiddle_const<2 * E, e, INV>(v[e]);
    });
  }
  dft_reg<E, INV>(v);
#pragma unroll
  for (int k1 = (ODDP ? 0 : 1); k1 < E; ++k1) v[k1] = cmulc<INV>(v[k1], tw[k1 * G + t]);
  __syncwarp();
#pragma unroll
  for (int k1 = 0; k1 < E; ++k1) scratch[k1 * (G + 1) + t] = v[k1];
  __syncwarp();
#pragma unroll
  for (int j = 0; j < U; ++j) {
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int r = pair_row<L, ODDP>(t, j, s);
      V u[G];
#pragma unroll
      for (int tt = 0; tt < G; ++tt) u[tt] = scratch[r * (G + 1) + tt];
      dft_reg<G, INV>(u);
#pragma unroll
      for (int k2 = 0; k2 < G; ++k2) v[(2 * j + s) * G + k2] = u[k2];
    }
  }
}

// paired spectral layout -> cyclic time layout (the transpose of fft_c2p's
// index map): y_n = sum_q X(q) w_L^{qn}, times w_{2L}^{n} when ODDP.
// twT is the same twiddle table transposed, twT[n2*E + k1] = tw[k1*G + n2],
// so that lanes reading different rows k1 hit different banks.
template <int L, bool INV, bool ODDP, typename V>
__device__ __forceinline__ void fft_p2c(V (&v)[PairShape<L>::E], V* scratch, const V* twT, int t) {
  constexpr int G = PairShape<L>::G, E = PairShape<L>::E, U = PairShape<L>::U;
#pragma unroll
  for (int j = 0; j < U; ++j) {
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      dft_reg<G, INV>(&v[(2 * j + s) * G]);
      const int r = pair_row<L, ODDP>(t, j, s);
#pragma unroll
      for (int n2 = 1; n2 < G; ++n2)          // column n2 = 0 of both tables is 1
        v[(2 * j + s) * G + n2] = cmulc<INV>(v[(2 * j + s) * G + n2], twT[n2 * E + r]);
    }
  }
  __syncwarp();
#pragma unroll
  for (int j = 0; j < U; ++j)
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int r = pair_row<L, ODDP>(t, j, s);
#pragma unroll
      for (int n2 = 0; n2 < G; ++n2) scratch[r * (G + 1) + n2] = v[(2 * j + s) * G + n2];
    }
  __syncwarp();
#pragma unroll
  for (int k1 = 0; k1 < E; ++k1) v[k1] = scratch[k1 * (G + 1) + t];
  dft_reg<E, INV>(v);
  if constexpr (ODDP) {
    static_for<1, E>([&](auto nc) {
      constexpr int n1 = decltype(nc)::value;
      v[n1] = twiddle_const<2 * E, n1, INV>(v[n1]);
    });
  }
}

// v[idx] <- f(v[idx], v[mirror(idx)], idx) for every slot, EVEN pairing, in
// lane (the mirror of frequency q is -q mod L).  Pairs never cross the first
// 2G slots, so those go through a small copy (the self-paired unit of lane 0
// pairs them differently) and the rest are updated pairwise in place.
template <int L, typename V, typename F>
__device__ __forceinline__ void apply_mirror_pairs(V (&v)[PairShape<L>::E], int t, F&& f) {
  constexpr int G = PairShape<L>::G, E = PairShape<L>::E;
  const bool u0 = (t == 0);
  V mm[2 * G];
  static_for<0, 2 * G>([&](auto ic) {
    constexpr int idx = decltype(ic)::value;
    mm[idx] = u0 ? v[MirrorSlot<L, idx>::unit0] : v[MirrorSlot<L, idx>::general];
  });
  static_for<2 * G, E>([&](auto ic) {
    constexpr int idx = decltype(ic)::value;
    constexpr int g = MirrorSlot<L, idx>::general;
    if constexpr (idx < g) {
      const V a = v[idx], b = v[g];
      v[idx] = f(a, b, idx);
      v[g] = f(b, a, g);
    }
  });
  static_for<0, 2 * G>([&](auto ic) {
    constexpr int idx = decltype(ic)::value;
    v[idx] = f(v[idx], mm[idx], idx);
  });
}

// ---------------------------------------------------------------------------
// Group FFT (four-step, one shared-memory transpose).
// ---------------------------------------------------------------------------
template <int L> struct GroupShape {
  static_assert(L >= 16 && L <= 1024 && (L & (L - 1)) == 0, "FFT length");
  static constexpr int G = (L <= 32) ? 4 : (L <= 128 ? 8 : (L <= 512 ? 16 : 32));
  static constexpr int E = L / G;
  static_assert(E >= G && E % G == 0, "four-step shape");
  // padded scratch tile, complex elements per group; groups are spaced by
  // SSTRIDE so that two groups of one half-warp fall on different banks
  static constexpr int SCRATCH = E * (G + 1);
  static constexpr int SSTRIDE = SCRATCH + 8;
};

// v: E values in cyclic layout; scratch: SCRATCH complex in shared memory (per
// group); tw: L entries in GLOBAL memory (read with __ldg),
// tw[k1*G + t] = e^{-2 pi i t k1 / L}; t: lane in group.
// All lanes of the warp must call this together (it uses __syncwarp).
template <int L, bool INV, typename V>
__device__ __forceinline__ void group_fft(V (&v)[GroupShape<L>::E], V* scratch, const V* __restrict__ tw,
                                          int t) {
  constexpr int G = GroupShape<L>::G;
  constexpr int E = GroupShape<L>::E;
  dft_reg<E, INV>(v);
#pragma unroll
  for (int k1 = 1; k1 < E; ++k1) v[k1] = cmulc<INV>(v[k1], __ldg(&tw[k1 * G + t]));
  __syncwarp();
#pragma unroll
  for (int k1 = 0; k1 < E; ++k1) scratch[k1 * (G + 1) + t] = v[k1];
  __syncwarp();
#pragma unroll
  for (int j = 0; j < E / G; ++j) {
    V u[G];
    const int k1 = t + G * j;
#pragma unroll
    for (int s = 0; s < G; ++s) u[s] = scratch[k1 * (G + 1) + s];
    dft_reg<G, INV>(u);
#pragma unroll
    for (int k2 = 0; k2 < G; ++k2) v[j + (E / G) * k2] = u[k2];
  }
}

// group_fft with this lane's twiddles in registers: twr[k1] = tw[k1*G + t]
template <int L, bool INV, typename V>
__device__ __forceinline__ void group_fft_r(V (&v)[GroupShape<L>::E], V* scratch,
                                            const V (&twr)[GroupShape<L>::E], int t) {
  constexpr int G = GroupShape<L>::G;
  constexpr int E = GroupShape<L>::E;
  dft_reg<E, INV>(v);
#pragma unroll
  for (int k1 = 1; k1 < E; ++k1) v[k1] = cmulc<INV>(v[k1], twr[k1]);
  __syncwarp();
#pragma unroll
  for (int k1 = 0; k1 < E; ++k1) scratch[k1 * (G + 1) + t] = v[k1];
  __syncwarp();
#pragma unroll
  for (int j = 0; j < E / G; ++j) {
    V u[G];
    const int k1 = t + G * j;
#pragma unroll
    for (int s = 0; s < G; ++s) u[s] = scratch[k1 * (G + 1) + s];
    dft_reg<G, INV>(u);
#pragma unroll
    for (int k2 = 0; k2 < G; ++k2) v[j + (E / G) * k2] = u[k2];
  }
}

// group_fft whose twiddles w^{t k1} come from a recurrence in k1 restarted
// from the table every 8 steps (4 table reads per lane instead of E - 1)
template <int L, bool INV, typename V>
__device__ __forceinline__ void group_fft_rec(V (&v)[GroupShape<L>::E], V* scratch, const V* __restrict__ tw,
                                              int t) {
  constexpr int G = GroupShape<L>::G;
  constexpr int E = GroupShape<L>::E;
  dft_reg<E, INV>(v);
  const V w1 = __ldg(&tw[G + t]);
  V cur = w1;
#pragma unroll
  for (int k1 = 1; k1 < E; ++k1) {
    if (k1 > 1) cur = ((k1 & 7) == 0) ? __ldg(&tw[k1 * G + t]) : cmul(cur, w1);
    v[k1] = cmulc<INV>(v[k1], cur);
  }
  __syncwarp();
#pragma unroll
  for (int k1 = 0; k1 < E; ++k1) scratch[k1 * (G + 1) + t] = v[k1];
  __syncwarp();
#pragma unroll
  for (int j = 0; j < E / G; ++j) {
    V u[G];
    const int k1 = t + G * j;
#pragma unroll
    for (int s = 0; s < G; ++s) u[s] = scratch[k1 * (G + 1) + s];
    dft_reg<G, INV>(u);
#pragma unroll
    for (int k2 = 0; k2 < G; ++k2) v[j + (E / G) * k2] = u[k2];
  }
}

// Value of the *mirror* element for every e, for a length-L transform split
// into its even (P=0) or odd (P=1) outputs.  Element q = t + G*e of the half
// of parity P is paired with q' = (L - q) mod L (P=0) or L-1-q (P=1).  Returns,
// for each e, the partner's value.  base: first lane of the group.
template <int L, typename V>
__device__ __forceinline__ void mirror_fetch(const V (&v)[GroupShape<L>::E], V (&m)[GroupShape<L>::E],
                                             int t, int parity, int base) {
  constexpr int G = GroupShape<L>::G;
  constexpr int E = GroupShape<L>::E;
  const int src = base + (parity == 0 ? ((G - t) & (G - 1)) : (G - 1 - t));
  const bool zero_lane = (parity == 0) && (t == 0);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    // what this lane must SEND so that its partner receives the partner's mirror
    V send = zero_lane ? v[(E - e) % E] : v[E - 1 - e];
    m[e].x = __shfl_sync(0xffffffffu, send.x, src);
    m[e].y = __shfl_sync(0xffffffffu, send.y, src);
  }
}

}  // namespace pp
