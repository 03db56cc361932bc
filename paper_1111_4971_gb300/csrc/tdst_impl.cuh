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
// Layout and schedule are those of the cyclic 2N-point routine: lanes of a
// group of G hold elements q = t + G e; pass 1 transforms the N rows along y
// into the ky = 1..N columns of a shared-memory buffer, pass 2 transforms each
// column along x, multiplies by the Green octant, transforms back and stores
// it in place, pass 3 transforms the rows back.  The pairs (q, N-q) of the
// mirror combinations are formed by the lane holding q for the first half of
// its slots, so half of the values cross lanes.  tdst_plane runs one plane
// per CTA; tdst_persistent is the staged form, one CTA per SM looping over
// planes, its pass-1 rows arriving by TMA bulk copies.
#pragma once

#include "../../include/pipe_poisson.h"
#include "fft_common.cuh"
#include "solver.cuh"

namespace pp {

// Bulk asynchronous copies (TMA, global -> shared) completed on an mbarrier.
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// order this thread's earlier shared-memory accesses (and, after a barrier,
// the CTA's) before later asynchronous-proxy writes to shared memory
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// one arrival that also announces `bytes` of copies to complete on `bar`,
// then the copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// non-blocking test of phase `parity` of `bar` (acquire: the copied bytes are
// visible to the caller once it returns true)
__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// polls of a staged-row wait before it gives up (about 0.2 s with the back-off)
constexpr long long kStageSpinLimit = 1LL << 21;

// GB: the plane buffer in a global scratch plane (a.tbuf, L2-resident)
// instead of shared memory, for planes too large for it (FP64 128 x 128).
// STG: the staged persistent form (one CTA per SM looping over planes); the
// rows of pass 1 arrive by bulk copies in a staging buffer of SR rows, and
// the first rows of the CTA's next plane are copied in while the current
// plane is still in passes 2 and 3.
template <typename T, int N, int THREADS, bool GB = false, bool STG = false>
struct TDstCfg {
  using S = GroupShape<N>;
  static constexpr int G = S::G;
  static constexpr int E = S::E;
  static constexpr int LD = N;
  static constexpr int SWM = (N < 16 ? N : 16) - 1;
  static constexpr int YBUF = N * LD;
  static constexpr int GROUPS = THREADS / G;
  static constexpr int GPC = (THREADS / 32) * (32 / G);        // lines in flight per CTA
  static constexpr int SR = GPC < N ? GPC : N;                 // staged rows per copy
  static_assert(N % SR == 0, "staged chunks tile the plane");
  static constexpr size_t STG_OFF =
      (sizeof(C2<T>) * ((GB ? 0 : size_t(YBUF)) + size_t(2 * N) + size_t(GROUPS) * S::SSTRIDE) + 15) / 16 * 16;
  static constexpr size_t STG_BYTES = sizeof(C2<T>) * size_t(SR) * N;
  static constexpr size_t BAR_OFF = STG_OFF + STG_BYTES;
  static constexpr size_t smem_bytes() { return STG ? BAR_OFF + 16 : STG_OFF; }
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
template <typename T, int N, int THREADS, bool ADJ, bool H16 = false, bool GB = false, bool STG = false>
struct TDst {
  static_assert(!(STG && (GB || H16)), "staged rows: FP32 / FP64 planes in shared memory");
  using Cfg = TDstCfg<T, N, THREADS, GB, STG>;
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
  V* stg;                     // STG: the staged rows [SR][N]
  uint64_t* bar;              // STG: completion barrier of the staged copies
  // this lane's per-slot phases w^{-q} and, when they fit in registers (at
  // most 256 threads, plane buffer in shared memory), its group-FFT twiddles
  static constexpr bool RTW = THREADS <= 256 && !GB;
  V ph[E];
  V twr[RTW ? E : 1];
  unsigned sphase = 0;        // STG: parity of the next staged chunk
  bool sfail = false;         // STG: a wait gave up (PIPE_ETIMEOUT recorded)
  int nissued = 0;            // STG, issuing thread: bulk copies issued so far
  int lane, t, line;

  __device__ __forceinline__ TDst(const SolveArgs<T>& a, unsigned char* smem_raw) {
    ybuf = reinterpret_cast<V*>(smem_raw);           // (GB: set per plane)
    sw2 = GB ? ybuf : ybuf + Cfg::YBUF;
    scratch = sw2 + 2 * N + (threadIdx.x / G) * GroupShape<N>::SSTRIDE;
    tw = a.tw_t;
    lane = threadIdx.x & 31;
    t = lane % G;
    line = lane / G + GPW * (threadIdx.x >> 5);                // groups of a warp: adjacent lines
    stg = reinterpret_cast<V*>(smem_raw + Cfg::STG_OFF);
    bar = reinterpret_cast<uint64_t*>(smem_raw + Cfg::BAR_OFF);
  }

  // STG, one thread: copy rows r0 .. r0+SR-1 of plane kz into the staging
  // buffer (the caller has synchronised after the buffer's last reads).  No
  // copy is issued once this thread's own wait has given up, and the copy
  // that a failure-detection test asks CTA 0 to leave out is skipped.
  __device__ __forceinline__ void stage_issue(const SolveArgs<T>& a, int kz, int r0) {
    const bool drop = blockIdx.x == 0 && nissued + 1 == a.stage_drop;
    ++nissued;
    if (sfail || drop) return;
    fence_async_smem();
    bulk_load(stg, a.work + (size_t(kz) * N + r0) * N, unsigned(Cfg::STG_BYTES), bar);
  }

  // STG: wait for the next staged chunk; a wait that gives up records
  // PIPE_ETIMEOUT and later waits return at once, so the kernel always ends
  __device__ __forceinline__ void stage_wait(const SolveArgs<T>& a) {
    if (!sfail) {
      const long long limit = a.stage_polls > 0 ? a.stage_polls : kStageSpinLimit;
      long long polls = 0;
      while (!mbar_test(bar, sphase)) {
        if (++polls > limit) {
          sfail = true;
          if (a.err) atomicExch(a.err, PIPE_ETIMEOUT);
          break;
        }
        if (polls > 32) __nanosleep(64);
      }
    }
    sphase ^= 1u;
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
    load_row_at(plane + size_t(il < N ? il : 0) * N, v);
  }
  __device__ __forceinline__ void load_row_at(const V* row, V (&v)[E]) const {
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

  // Mirror pairs of an N-point spectrum in the cyclic layout (lane t holds
  // q = t + G e): the mirror N - q of slot e is slot E-1-e of lane (G-t) mod G,
  // except in lane 0, whose slots e and E-e are each other's mirrors (slot 0,
  // q = 0, and slot E/2, q = N/2, are their own).  Each lane works on the
  // pairs of its slots j < E/2, so half of the values cross lanes.
  // pair_fetch: the mirror values of the slots j < E/2.
  __device__ __forceinline__ void pair_fetch(const V (&x)[E], V (&xm)[H]) const {
    const int src = (lane - t) + ((G - t) & (G - 1));
#pragma unroll
    for (int j = 0; j < H; ++j) {
      const V snd = x[E - 1 - j];
      V r;
      r.x = __shfl_sync(0xffffffffu, snd.x, src);
      r.y = __shfl_sync(0xffffffffu, snd.y, src);
      xm[j] = t == 0 ? x[(E - j) % E] : r;
    }
  }
  // pair_return: from results at the slots j < E/2 (ra) and at their mirrors
  // (rb; lane 0: rb[0] unused, rh at its slot E/2), the cyclic layout again
  // (slot E-1-j of lane t is the mirror of slot j of lane (G-t) mod G)
  __device__ __forceinline__ void pair_return(const V (&ra)[H], const V (&rb)[H], V rh, V (&x)[E]) const {
    const int src = (lane - t) + ((G - t) & (G - 1));
#pragma unroll
    for (int j = 0; j < H; ++j) {
      x[j] = ra[j];
      V r;
      r.x = __shfl_sync(0xffffffffu, rb[j].x, src);
      r.y = __shfl_sync(0xffffffffu, rb[j].y, src);
      const V own = (j + 1 < H) ? rb[j + 1 < H ? j + 1 : 0] : rh;   // lane 0
      x[E - 1 - j] = t == 0 ? own : r;
    }
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

  // this lane's phases and twiddles (after load_tables and a barrier); they
  // serve every plane the CTA transforms
  __device__ __forceinline__ void lane_tables() {
#pragma unroll
    for (int e = 0; e < E; ++e) ph[e] = sw2[(SGN * (t + G * e)) & MASK];
    if constexpr (RTW) {
#pragma unroll
      for (int k1 = 0; k1 < E; ++k1) twr[k1] = __ldg(&tw[k1 * G + t]);
    }
  }

  // Plane kz in place (the phase table already loaded and synchronised).
  // Ends with the plane's stores issued; the caller synchronises before
  // another plane reuses the buffers.
  // STG: next >= 0 is the CTA's next plane, whose first rows are copied in
  // once this plane's pass 1 has read its last staged rows.
  __device__ __forceinline__ void plane(const SolveArgs<T>& a, int kz, int next = -1) {
    V* pl = a.work + size_t(kz) * N * N;
    if constexpr (GB) ybuf = a.tbuf + size_t(kz) * N * N;
    // the group-FFT twiddles from registers (RTW), else from the table at
    // each transform
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
      if constexpr (H16) {
        load_row16(a, kz, il, v);
      } else if constexpr (STG) {
        stage_wait(a);
        load_row_at(stg + size_t(il < N ? il - r0 : 0) * N, v);
        __syncthreads();               // every lane has read the staged rows
        if (threadIdx.x == 0) {
          if (r0 + GPC < N) stage_issue(a, kz, r0 + GPC);
          else if (next >= 0) stage_issue(a, next, 0);
        }
      } else {
        load_row(pl, il, v);
      }
      fft(Fwd{}, v);                   // V(q)
      V vm[H];
      pair_fetch(v, vm);               // V(N-q) of the slots j < E/2
      if (il < N) {
        // U(q) = V(q) - w^{-q} V(N-q), U(N-q) = V(N-q) + conj(w^{-q}) V(q)
        // (w^{-(N-q)} = -conj(w^{-q})); lane 0: U(N) = 2 V(0), and q = N/2
#pragma unroll
        for (int j = 0; j < H; ++j) {
          const int q = t + G * j;
          if (q == 0) {
            ybuf[tile(N, il)] = mk<V>(v[0].x + v[0].x, v[0].y + v[0].y);
          } else {
            ybuf[tile(q, il)] = cfms(v[j], ph[j], vm[j]);
            ybuf[tile(N - q, il)] = cfms(vm[j], mk<V>(-ph[j].x, ph[j].y), v[j]);
          }
        }
        if (t == 0) ybuf[tile(N / 2, il)] = cfms(v[H], ph[H], v[H]);
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
      if constexpr (!H16) {
        // the Green row at kx = q_j (N for q_j = 0) and N - q_j of the slots
        // j < E/2, and at N/2 (lane 0), read before the transform
        T ga[H], gb[H];
#pragma unroll
        for (int j = 0; j < H; ++j) {
          const int kx = t + G * j;
          ga[j] = act ? __ldg(&grow[kx == 0 ? N : kx]) : T(0);
          gb[j] = act ? __ldg(&grow[N - kx]) : T(0);
        }
        const T gh = act ? __ldg(&grow[N / 2]) : T(0);
        fft(Fwd{}, u);                 // V(kx)
        V um[H];
        pair_fetch(u, um);             // V(N-kx) of the slots j < E/2
        // P = g U at kx and N - kx, then V'(q) = P(q) + w^{-q} P(N-q) and
        // V'(N-q) = P(N-q) - conj(w^{-q}) P(q); lane 0: V'(0) = P(N) with
        // U(N) = 2 V(0), and the self-mirrored kx = N/2
        V ra[H], rb[H];
#pragma unroll
        for (int j = 0; j < H; ++j) {
          const int kx = t + G * j;
          const V nph = mk<V>(-ph[j].x, ph[j].y);
          if (kx == 0) {
            ra[j] = cscale(mk<V>(u[0].x + u[0].x, u[0].y + u[0].y), ga[j]);
            rb[j] = ra[j];
          } else {
            const V pa = cscale(cfms(u[j], ph[j], um[j]), ga[j]);
            const V pb = cscale(cfms(um[j], nph, u[j]), gb[j]);
            ra[j] = cfma_(pa, ph[j], pb);
            rb[j] = cfma_(pb, nph, pa);
          }
        }
        V rh = mk<V>(T(0), T(0));
        if (t == 0) {
          const V pn = cscale(cfms(u[H], ph[H], u[H]), gh);
          rh = cfma_(pn, ph[H], pn);
        }
        pair_return(ra, rb, rh, u);    // V'(q) in the cyclic layout
      } else {
        T gpre[E];                     // the Green row, read before the transform
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int kx = t + G * e;
          gpre[e] = act ? __ldg(&grow[kx == 0 ? N : kx]) : T(0);
        }
        fft(Fwd{}, u);                 // V(kx)
        V m[E];
        mirror_fetch<N>(u, m, t, 0, lane - t);
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
          const __half2 hp = __hmul2(uh, __float2half2_rn(g[e] * ig));
          const float2 pf = __half22float2(hp);
          u[e] = mk<V>(T(pf.x * back), T(pf.y * back));       // P(kx)
        }
        mirror_fetch<N>(u, m, t, 0, lane - t);                 // P(N-kx)
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int q = t + G * e;
          if (q != 0) u[e] = cfma_(u[e], ph[e], m[e]);         // V'(q); V'(0) = P(N)
        }
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
  r.lane_tables();
  r.plane(a, kz);
}

// the staged persistent form: CTA b takes planes b, b + gridDim.x, ...
template <typename T, int N, int THREADS, bool ADJ>
__device__ __forceinline__ void tdst_persistent(const SolveArgs<T>& a, unsigned char* smem_raw) {
  TDst<T, N, THREADS, ADJ, false, false, true> r(a, smem_raw);
  const int first = int(blockIdx.x);
  if (first > a.nz) return;
  if (threadIdx.x == 0) {
    mbar_init(r.bar, 1);
    r.stage_issue(a, first, 0);
  }
  r.load_tables(a);
  __syncthreads();
  r.lane_tables();
#pragma unroll 1
  for (int kz = first; kz <= a.nz; kz += int(gridDim.x)) {
    const int next = kz + int(gridDim.x) <= a.nz ? kz + int(gridDim.x) : -1;
    r.plane(a, kz, next);
    __syncthreads();                   // before the next plane reuses the buffers
  }
  // after a wait gave up a copy may still be in flight: wait for it (bounded)
  // so that it does not land after the CTA has left
  if (threadIdx.x == 0 && r.sfail) {
    const long long limit = a.stage_polls > 0 ? a.stage_polls : kStageSpinLimit;
    for (long long polls = 0; polls < limit && !mbar_test(r.bar, r.sphase); ++polls) __nanosleep(64);
  }
}

}  // namespace pp
