// Device routines of the z-axis transforms, shared by the per-stage kernels
// (zfft.cu) and the batched persistent kernel (batched.cu).
//
// z-axis transforms of the pipe Poisson solve (Sec. 2 Eq. 10, Appendix A).
//
// Forward (zfwd_tile): for every (i,j) column, the 2*nz-point real DFT of the
// zero-padded column (Eq. A.2; the padded half is never read):
//     X(kz) = sum_{k<nz} rho_ijk e^{-2 pi i k kz/(2 nz)},   kz = 0..nz
// Packing z_m = rho_{2m} + i rho_{2m+1} (m < nz/2) turns it into an nz-point
// complex DFT whose input is half zero; that one splits into two nz/2-point
// FFTs (even and odd kz of Z, the odd one on the input twisted by w_nz^m).
// X follows from Z(k) and conj Z(nz-k).  Output is written kz-plane major,
// work[kz][i*ny + j], through a shared-memory staging tile so that every
// store is a contiguous run of COLS columns.
//
// Inverse (zinv_tile): the transpose of the above for a Hermitian half
// spectrum: rebuild Z from X(k), X(nz-k), two nz/2-point inverse FFTs, keep
// only the physical outputs k < nz (the discarded half is never computed).
// Unnormalised (the 1/(2 nz) lives in the Green spectrum).
//
// CONJ gives the transforms of the opposite direction, used by the adjoint:
// for real data the e^{+} transform is the conjugate of the e^{-} one.
#pragma once

#include "solver.cuh"

namespace pp {

// asynchronous 16-byte global -> shared copy (L2 only, not cached in L1)
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

// asynchronous 4-byte global -> shared copy
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}

// largest component of a complex-FP16 slab is stored as 2^14 (headroom below
// the FP16 maximum 65504); an all-zero slab keeps scale 1
__device__ __forceinline__ float slab_scale(float mx) { return mx > 0.f ? mx * (1.f / 16384.f) : 1.f; }

// asynchronous 8-byte global -> shared copy
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
template <typename V>
__device__ __forceinline__ void cp_async_elem(V* dst, const V* src) {
  if constexpr (sizeof(V) == 16) cp_async16(dst, src);
  else cp_async8(dst, src);
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Warp-uniform phase steps of the z transforms, compile-time constants in
// constant memory (read through the constant cache, off the L1 data path).
// The phase of output k = 2(t + G e) + p factors into a per-lane part and a
// part that depends only on the unrolled index e:
//     w_{2nz}^k = w_{2nz}^{2t+p} * w_nz^{G e},
// so each lane reads one table value and takes w_nz^{G e} from here.
constexpr int kZSteps = 84;                       // sum of E over nz = 32..1024
constexpr int zstep_offset(int nz) {
  return nz == 32 ? 0 : nz == 64 ? 4 : nz == 128 ? 12 : nz == 256 ? 20 : nz == 512 ? 36 : 52;
}
template <typename T>
struct ZStepTab {
  T c[kZSteps];
  T s[kZSteps];
};
template <typename T>
constexpr ZStepTab<T> make_zsteps() {
  ZStepTab<T> z{};
  for (int nz = 32; nz <= 1024; nz *= 2) {
    const int L = nz / 2;
    const int G = (L <= 32) ? 4 : (L <= 128 ? 8 : (L <= 512 ? 16 : 32));
    for (int e = 0; e < L / G; ++e) {
      z.c[zstep_offset(nz) + e] = T(ccos2pi(long(G) * e, nz));
      z.s[zstep_offset(nz) + e] = T(-csin2pi(long(G) * e, nz));
    }
  }
  return z;
}
static __constant__ ZStepTab<float> c_zsteps_f = make_zsteps<float>();
static __constant__ ZStepTab<double> c_zsteps_d = make_zsteps<double>();
template <typename T, int NZ>
__device__ __forceinline__ C2<T> zstep(int e) {              // w_nz^{G e}
  if constexpr (sizeof(T) == 8) return mk<C2<T>>(c_zsteps_d.c[zstep_offset(NZ) + e], c_zsteps_d.s[zstep_offset(NZ) + e]);
  else return mk<C2<T>>(c_zsteps_f.c[zstep_offset(NZ) + e], c_zsteps_f.s[zstep_offset(NZ) + e]);
}

// FP32: the phase of element (t, e) as (lane base) x (constant step), and the
// group-FFT twiddles from a short recurrence -- fewer reads through L1, which
// bounds the FP32 kernels.  FP64 (bound by its arithmetic rate on this GPU):
// plain table reads, no extra multiplies.
template <typename T, int NZ>
__device__ __forceinline__ C2<T> zphase(const C2<T>* __restrict__ w2, C2<T> base, int idx, int e) {
  if constexpr (sizeof(T) == 4) return cmul(base, zstep<T, NZ>(e));
  else return __ldg(&w2[idx]);
}
template <int L, bool INV, typename V>
__device__ __forceinline__ void zgroup_fft(V (&v)[GroupShape<L>::E], V* scratch, const V* __restrict__ tw, int t) {
  if constexpr (sizeof(V) == 8) group_fft_rec<L, INV>(v, scratch, tw, t);
  else group_fft<L, INV>(v, scratch, tw, t);
}

// Real-to-complex pairing of the forward z transform.  Slot e of lane (t, p)
// holds Z(k), k = 2(t + G e) + p; its mirror Z(nz - k) is slot E-1-e of lane
// G-1-t (odd half) or lane (G-t) mod G (even half), except in lane t = 0 of
// the even half, which holds both members of its pairs itself (slots e and
// E-e; slot 0 pairs with itself through Z(nz) = Z(0), and slot E/2 is
// k = nz/2).  Every lane computes X(k) and X(nz - k) for its slots e < E/2,
// so it needs only the partner's slots E/2 .. E-1: half of the values cross
// lanes.  X(k) = (Z(k) + conj Z(nz-k) - i w^k (Z(k) - conj Z(nz-k))) / 2 with
// w = w_{2nz}; X(nz - k) swaps the pair and takes w^{nz-k} = -conj(w^k)
// (X(nz) = Re Z(0) - Im Z(0) is the case k = 0).  xh: X(nz/2), in lane t = 0
// of the even half only.
template <typename T, int NZ, int WARPS, bool CONJ>
__device__ __forceinline__ void zfwd_pairs(const SolveArgs<T>& a, const C2<T> (&v)[GroupShape<NZ / 2>::E], int t,
                                           int p, int lane, C2<T> (&xa)[GroupShape<NZ / 2>::E / 2],
                                           C2<T> (&xb)[GroupShape<NZ / 2>::E / 2], C2<T>& xh) {
  using V = C2<T>;
  constexpr int G = GroupShape<NZ / 2>::G, E = GroupShape<NZ / 2>::E;
  const bool zero_lane = (p == 0) && (t == 0);
  const int partner = (lane - t) + (p == 0 ? ((G - t) & (G - 1)) : (G - 1 - t));
  V zm[E / 2];                                        // Z(nz - k) of slot j
#pragma unroll
  for (int j = 0; j < E / 2; ++j) {
    const V snd = v[E - 1 - j];
    V r;
    r.x = __shfl_sync(0xffffffffu, snd.x, partner);
    r.y = __shfl_sync(0xffffffffu, snd.y, partner);
    zm[j] = zero_lane ? v[(E - j) % E] : r;
  }
  const V bk = __ldg(&a.w2_z[2 * t + p]);
  auto r2c = [](V z, V zmir, V w) {
    const V zc = cconj(zmir);
    const V s = cadd(z, zc);
    const V d = csub(z, zc);
    const V wd = cmul(w, d);
    const V x = mk<V>(T(0.5) * (s.x + wd.y), T(0.5) * (s.y - wd.x));   // (s - i w d)/2
    return CONJ ? cconj(x) : x;
  };
#pragma unroll
  for (int j = 0; j < E / 2; ++j) {
    const V w = zphase<T, NZ>(a.w2_z, bk, 2 * (t + G * j) + p, j);
    xa[j] = r2c(v[j], zm[j], w);
    xb[j] = r2c(zm[j], v[j], mk<V>(-w.x, w.y));
  }
  xh = zero_lane ? r2c(v[E / 2], v[E / 2], zphase<T, NZ>(a.w2_z, bk, G * E, E / 2)) : mk<V>(T(0), T(0));
}

// The staging column of the forward z transform holds its even kz in slots
// 0..nz/2 and its odd kz after them, so that the lanes of one parity write
// consecutive slots: k = 2(t + G j) + p goes to slot (p ? nz/2 + 1 : 0) + t + G j,
// nz - k to slot (p ? nz : nz/2) - t - G j, and nz/2 to slot nz/4.
template <typename T, int NZ>
__device__ __forceinline__ void zfwd_stage_col(C2<T>* col, const C2<T> (&xa)[GroupShape<NZ / 2>::E / 2],
                                               const C2<T> (&xb)[GroupShape<NZ / 2>::E / 2], C2<T> xh, int t,
                                               int p) {
  constexpr int G = GroupShape<NZ / 2>::G, E = GroupShape<NZ / 2>::E;
  C2<T>* mine = col + (p ? NZ / 2 + 1 : 0) + t;
  C2<T>* mirr = col + (p ? NZ : NZ / 2) - t;
#pragma unroll
  for (int j = 0; j < E / 2; ++j) {
    mine[G * j] = xa[j];
    mirr[-G * j] = xb[j];
  }
  if (p == 0 && t == 0) col[NZ / 4] = xh;
}

// Coalesced 16-byte stores (EPV complex of consecutive columns) of a staged
// tile into work[kz][col0 ..].  Thread (q0, cc) takes rows r0, r0 + QSTEP, ...,
// where r0 orders each block of 8 rows as 0 2 4 6 1 3 5 7, so that the two
// half-warps read rows of one parity each (conflict-free) and the row parity
// is fixed per thread.
template <typename T, int NZ, int WARPS>
__device__ __forceinline__ void zfwd_store_tile(const SolveArgs<T>& a, const C2<T>* stage, int col0) {
  using Cfg = ZCfg<T, NZ, WARPS>;
  using V = C2<T>;
  constexpr int EPV = 16 / int(sizeof(V));
  constexpr int VPR = Cfg::COLS / EPV;
  constexpr int QSTEP = Cfg::THREADS / VPR;
  static_assert(QSTEP % 8 == 0 && NZ % 8 == 0, "rows in blocks of 8");
  const int ncols = a.nx * a.ny;
  const int q0 = threadIdx.x / VPR;
  const int cc = (threadIdx.x % VPR) * EPV;
  const int r0 = (q0 & ~7) | ((q0 & 3) << 1) | ((q0 >> 2) & 1);
  if (col0 + cc >= ncols) return;
  const V* src = stage + cc * Cfg::LDS + ((r0 & 1) ? NZ / 2 + 1 : 0) + (r0 >> 1);
  V* dst = a.work + size_t(r0) * ncols + col0 + cc;
  for (int r = r0; r <= NZ; r += QSTEP, src += QSTEP / 2, dst += size_t(QSTEP) * ncols) {
    if constexpr (EPV == 2) {
      const V x0 = src[0], x1 = src[Cfg::LDS];
      *reinterpret_cast<float4*>(dst) = make_float4(x0.x, x0.y, x1.x, x1.y);
    } else {
      *dst = src[0];
    }
  }
}

// one CTA of 32*WARPS threads: columns [tile*COLS, (tile+1)*COLS)
// H16: the spectrum is stored as complex FP16 with one scale per tile
// (a.zscale[tile]); the reduction scratch follows Cfg::smem_bytes().
template <typename T, int NZ, int WARPS, bool CONJ, bool H16 = false>
__device__ __forceinline__ void zfwd_tile(const SolveArgs<T>& a, int tile, unsigned char* smem_raw) {
  using Cfg = ZCfg<T, NZ, WARPS>;
  using V = C2<T>;
  constexpr int L = Cfg::L, G = Cfg::G, E = Cfg::E;
  V* sbase = reinterpret_cast<V*>(smem_raw);
  V* stage = sbase;                                   // reused after the FFT

  const int ncols = a.nx * a.ny;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int t = lane % G;
  const int p = (lane / G) & 1;                       // parity of kz produced
  const int col_local = warp * Cfg::CPW + lane / Cfg::UNIT;
  const int col0 = tile * Cfg::COLS;
  const int col = col0 + col_local;
  const bool valid = col < ncols;
  V* scratch = sbase + (threadIdx.x / G) * GroupShape<L>::SSTRIDE;

  // packed column, z_m = (rho[2m], rho[2m+1]), m = t + G e
  V v[E];
  const V* src = reinterpret_cast<const V*>(a.rho + size_t(valid ? col : 0) * NZ);
#pragma unroll
  for (int e = 0; e < E; ++e) v[e] = valid ? __ldg(&src[t + G * e]) : mk<V>(0, 0);
  if (p) {
    const V b = __ldg(&a.w2_z[2 * t]);
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = cmul(v[e], zphase<T, NZ>(a.w2_z, b, 2 * (t + G * e), e));   // w_nz^m
  }
  zgroup_fft<L, false>(v, scratch, a.tw_z, t);        // v[e] = Z(2q + p), q = t + G e
  V xa[E / 2], xb[E / 2], xh;
  zfwd_pairs<T, NZ, WARPS, CONJ>(a, v, t, p, lane, xa, xb, xh);
  __syncthreads();                                    // FFT scratch becomes the staging tile
  zfwd_stage_col<T, NZ>(stage + col_local * Cfg::LDS, xa, xb, xh, t, p);
  if constexpr (H16) {
    float* red = reinterpret_cast<float*>(smem_raw + Cfg::smem_bytes());
    float mx = fmaxf(fabsf(float(xh.x)), fabsf(float(xh.y)));
#pragma unroll
    for (int j = 0; j < E / 2; ++j) {
      mx = fmaxf(mx, fmaxf(fabsf(float(xa[j].x)), fabsf(float(xa[j].y))));
      mx = fmaxf(mx, fmaxf(fabsf(float(xb[j].x)), fabsf(float(xb[j].y))));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    mx = 0.f;
#pragma unroll
    for (int w = 0; w < WARPS; ++w) mx = fmaxf(mx, red[w]);
    const float sc = slab_scale(mx), inv = 1.f / sc;
    auto slot = [](int k) { return (k & 1) ? NZ / 2 + 1 + (k >> 1) : (k >> 1); };
    if (threadIdx.x == 0) a.zscale[tile] = sc;
    // 16-byte stores of four complex-FP16 values (consecutive columns)
    constexpr int VPR = Cfg::COLS / 4;
    static_assert(Cfg::COLS % 4 == 0, "tile width");
    __half2* w16 = reinterpret_cast<__half2*>(a.work);
    for (int idx = threadIdx.x; idx < (NZ + 1) * VPR; idx += Cfg::THREADS) {
      const int r = idx / VPR;
      const int cc = (idx % VPR) * 4;
      if (col0 + cc < ncols) {
        union {
          uint4 u;
          __half2 h[4];
        } pk;                                       // 16-byte aligned by its uint4 member
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const V x = stage[(cc + q) * Cfg::LDS + slot(r)];
          pk.h[q] = __floats2half2_rn(float(x.x) * inv, float(x.y) * inv);
        }
        *reinterpret_cast<uint4*>(&w16[size_t(r) * ncols + col0 + cc]) = pk.u;
      }
    }
    return;
  }
  __syncthreads();
  zfwd_store_tile<T, NZ, WARPS>(a, stage, col0);
}

// H16: the spectrum is complex FP16 with one scale per transverse row
// (a.tscale[kz * nx + i]; the tile's columns lie in one row i)
template <typename T, int NZ, int WARPS, bool CONJ, bool H16 = false>
__device__ __forceinline__ void zinv_tile(const SolveArgs<T>& a, int tile, unsigned char* smem_raw) {
  using Cfg = ZCfg<T, NZ, WARPS>;
  using V = C2<T>;
  constexpr int L = Cfg::L, G = Cfg::G, E = Cfg::E;
  V* sbase = reinterpret_cast<V*>(smem_raw);
  V* stage = sbase;                                   // FFT scratch reuses it afterwards

  const int ncols = a.nx * a.ny;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int t = lane % G;
  const int p = (lane / G) & 1;
  const int col_local = warp * Cfg::CPW + lane / Cfg::UNIT;
  const int col0 = tile * Cfg::COLS;
  const int col = col0 + col_local;
  const bool valid = col < ncols;
  V* scratch = sbase + (threadIdx.x / G) * GroupShape<L>::SSTRIDE;

  V v[E];
  const V bk = __ldg(&a.w2_z[2 * t + p]);
  // Z(k) = X(k) + conj X(nz-k) + i w_{2nz}^{-k} (X(k) - conj X(nz-k)), k = 2(t+Ge)+p
  auto rebuild = [&](V x, V xm_, int e) {
    const V xm = cconj(xm_);
    const V s = cadd(x, xm);
    const V d = csub(x, xm);
    const V wd = cmulc<true>(d, zphase<T, NZ>(a.w2_z, bk, 2 * (t + G * e) + p, e));   // w_{2nz}^{-k} d
    return mk<V>(s.x - wd.y, s.y + wd.x);                      // s + i w d
  };
  if constexpr (H16) {
    __half2* st16 = reinterpret_cast<__half2*>(smem_raw);
    const __half2* w16 = reinterpret_cast<const __half2*>(a.work);
    for (int idx = threadIdx.x; idx < (NZ + 1) * Cfg::COLS; idx += Cfg::THREADS) {
      const int r = idx / Cfg::COLS;
      const int cc = idx % Cfg::COLS;
      if (col0 + cc < ncols) cp_async4(&st16[cc * Cfg::LDS + r], &w16[size_t(r) * ncols + col0 + cc]);
    }
    cp_async_wait_all();
    __syncthreads();
    const __half2* mycol = st16 + col_local * Cfg::LDS;
    const float* rs = a.tscale + (valid ? col : 0) / a.ny;     // + kz * nx
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k = 2 * (t + G * e) + p;
      const float2 f = __half22float2(mycol[k]);
      const float sc = __ldg(&rs[size_t(k) * a.nx]);
      v[e] = mk<V>(T(f.x * sc), T(f.y * sc));
    }
    const float2 f = __half22float2(mycol[NZ]);
    const float sc = __ldg(&rs[size_t(NZ) * a.nx]);
    V xN = mk<V>(T(f.x * sc), T(f.y * sc));
    __syncthreads();                                  // staging tile becomes FFT scratch
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
    for (int e = 0; e < E; ++e) v[e] = rebuild(v[e], m[e], e);
  } else {
    // the whole (nz+1) x COLS tile in flight at once (cp.async, one element
    // each); a column holds its even kz in slots 0..nz/2 and its odd kz after
    // them, so that the lanes of one parity read consecutive slots
    // (thread: column cc, rows r0, r0 + RSTEP, ...; RSTEP = 2G is even, so
    // the row parity and hence the half of the column are fixed per thread)
    {
      constexpr int RSTEP = Cfg::THREADS / Cfg::COLS;
      static_assert(RSTEP % 2 == 0, "row step keeps the parity");
      const int cc = threadIdx.x % Cfg::COLS, r0 = threadIdx.x / Cfg::COLS;
      if (col0 + cc < ncols) {
        V* dst = stage + cc * Cfg::LDS + ((r0 & 1) ? NZ / 2 + 1 : 0) + (r0 >> 1);
        const V* src = a.work + size_t(r0) * ncols + col0 + cc;
        for (int r = r0; r <= NZ; r += RSTEP, dst += RSTEP / 2, src += size_t(RSTEP) * ncols)
          cp_async_elem(dst, src);
      }
    }
    cp_async_wait_all();
    __syncthreads();
    // X(k) and its partner X(nz - k) straight from the staging tile (k = 0
    // pairs with X(nz)), combined before the tile becomes FFT scratch:
    // k = 2(t + G e) + p sits in slot (p ? nz/2 + 1 : 0) + t + G e, and
    // nz - k in slot (p ? nz : nz/2) - t - G e
    const V* mine = stage + col_local * Cfg::LDS + (p ? NZ / 2 + 1 : 0) + t;
    const V* mirr = stage + col_local * Cfg::LDS + (p ? NZ : NZ / 2) - t;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const V x = mine[G * e], xm = mirr[-G * e];
      v[e] = CONJ ? rebuild(cconj(x), cconj(xm), e) : rebuild(x, xm, e);
    }
    __syncthreads();                                  // staging tile becomes FFT scratch
  }
  zgroup_fft<L, true>(v, scratch, a.tw_z, t);                  // z_p(m), m = t + G e
  if (p) {
    const V b = __ldg(&a.w2_z[2 * t]);
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = cmulc<true>(v[e], zphase<T, NZ>(a.w2_z, b, 2 * (t + G * e), e));
  }
  // z(m) = z_0(m) + z_1(m): the lane of parity p keeps the sums for the slots
  // e = j + p E/2; it sends its partner (lane t of the other parity) its own
  // values of the partner's slots and adds what the partner sends back
  V out[E / 2];
#pragma unroll
  for (int j = 0; j < E / 2; ++j) {
    const V snd = p ? v[j] : v[j + E / 2];
    const V mine = p ? v[j + E / 2] : v[j];
    out[j].x = mine.x + __shfl_xor_sync(0xffffffffu, snd.x, G);
    out[j].y = mine.y + __shfl_xor_sync(0xffffffffu, snd.y, G);
  }
  if (valid) {
    V* dst = reinterpret_cast<V*>(a.phi + size_t(col) * NZ);
#pragma unroll
    for (int j = 0; j < E / 2; ++j) dst[t + G * (j + p * (E / 2))] = out[j];
  }
}

// ---------------------------------------------------------------------------
// Pipelined multi-tile versions: `count` tiles first, first+stride, ...; the
// input of the next tile is copied (cp.async) into the second buffer while
// the current tile is transformed, so that one CTA keeps HBM busy on its own.
// ---------------------------------------------------------------------------
template <typename T, int NZ, int WARPS, bool CONJ>
__device__ __forceinline__ void zfwd_tiles_pipe(const SolveArgs<T>& a, int first, int stride, int count,
                                                unsigned char* smem_raw) {
  using Cfg = ZCfg<T, NZ, WARPS>;
  using V = C2<T>;
  constexpr int L = Cfg::L, G = Cfg::G, E = Cfg::E;
  constexpr int INW = int(Cfg::INW);
  V* inb = reinterpret_cast<V*>(smem_raw);                    // [2][COLS][NZ/2]
  V* scr0 = inb + 2 * INW;
  V* stage = scr0 + Cfg::SCR;                                  // [COLS][LDS]
  const int ncols = a.nx * a.ny;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int t = lane % G;
  const int p = (lane / G) & 1;
  const int col_local = warp * Cfg::CPW + lane / Cfg::UNIT;
  V* scratch = scr0 + (threadIdx.x / G) * GroupShape<L>::SSTRIDE;
  // 16-byte pieces of one tile's input: COLS columns of NZ reals
  constexpr int PPC = NZ * int(sizeof(T)) / 16;
  auto issue = [&](int tile, V* buf) {
    const int col0 = tile * Cfg::COLS;
    for (int idx = threadIdx.x; idx < Cfg::COLS * PPC; idx += Cfg::THREADS) {
      const int cc = idx / PPC, piece = idx % PPC;
      if (col0 + cc < ncols)
        cp_async16(reinterpret_cast<unsigned char*>(buf + cc * (NZ / 2)) + 16 * piece,
                   reinterpret_cast<const unsigned char*>(a.rho + size_t(col0 + cc) * NZ) + 16 * piece);
    }
    cp_async_commit();
  };
  if (count > 0) issue(first, inb);
  for (int k = 0; k < count; ++k) {
    const int tile = first + k * stride;
    const int col0 = tile * Cfg::COLS;
    if (k + 1 < count) {
      issue(first + (k + 1) * stride, inb + ((k + 1) & 1) * INW);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const V* src = inb + (k & 1) * INW + col_local * (NZ / 2);
    V v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = src[t + G * e];
    if (p) {
      const V b = __ldg(&a.w2_z[2 * t]);
#pragma unroll
      for (int e = 0; e < E; ++e) v[e] = cmul(v[e], zphase<T, NZ>(a.w2_z, b, 2 * (t + G * e), e));
    }
    zgroup_fft<L, false>(v, scratch, a.tw_z, t);
    V xa[E / 2], xb[E / 2], xh;
    zfwd_pairs<T, NZ, WARPS, CONJ>(a, v, t, p, lane, xa, xb, xh);
    zfwd_stage_col<T, NZ>(stage + col_local * Cfg::LDS, xa, xb, xh, t, p);
    __syncthreads();
    zfwd_store_tile<T, NZ, WARPS>(a, stage, col0);
    __syncthreads();
  }
}

template <typename T, int NZ, int WARPS, bool CONJ>
__device__ __forceinline__ void zinv_tiles_pipe(const SolveArgs<T>& a, int first, int stride, int count,
                                                unsigned char* smem_raw) {
  using Cfg = ZCfg<T, NZ, WARPS>;
  using V = C2<T>;
  constexpr int L = Cfg::L, G = Cfg::G, E = Cfg::E;
  constexpr int STG = int(Cfg::STG);
  V* stg = reinterpret_cast<V*>(smem_raw);                    // [2][COLS][LDS]
  V* scr0 = stg + 2 * STG;
  const int ncols = a.nx * a.ny;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int t = lane % G;
  const int p = (lane / G) & 1;
  const int col_local = warp * Cfg::CPW + lane / Cfg::UNIT;
  V* scratch = scr0 + (threadIdx.x / G) * GroupShape<L>::SSTRIDE;
  auto issue = [&](int tile, V* buf) {
    const int col0 = tile * Cfg::COLS;
    for (int idx = threadIdx.x; idx < (NZ + 1) * Cfg::COLS; idx += Cfg::THREADS) {
      const int r = idx / Cfg::COLS, cc = idx % Cfg::COLS;
      if (col0 + cc < ncols) cp_async_elem(&buf[cc * Cfg::LDS + r], &a.work[size_t(r) * ncols + col0 + cc]);
    }
    cp_async_commit();
  };
  if (count > 0) issue(first, stg);
  for (int k = 0; k < count; ++k) {
    const int tile = first + k * stride;
    const int col = tile * Cfg::COLS + col_local;
    if (k + 1 < count) {
      issue(first + (k + 1) * stride, stg + ((k + 1) & 1) * STG);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const V* mycol = stg + (k & 1) * STG + col_local * Cfg::LDS;
    V v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = mycol[2 * (t + G * e) + p];
    V xN = mycol[NZ];
    if (CONJ) {
#pragma unroll
      for (int e = 0; e < E; ++e) v[e] = cconj(v[e]);
      xN = cconj(xN);
    }
    V m[E];
    mirror_fetch<L>(v, m, t, p, lane - t);
    if (p == 0 && t == 0) m[0] = xN;
    const V bk = __ldg(&a.w2_z[2 * t + p]);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const V xm = cconj(m[e]);
      const V s = cadd(v[e], xm);
      const V d = csub(v[e], xm);
      const V wd = cmulc<true>(d, zphase<T, NZ>(a.w2_z, bk, 2 * (t + G * e) + p, e));
      v[e] = mk<V>(s.x - wd.y, s.y + wd.x);
    }
    zgroup_fft<L, true>(v, scratch, a.tw_z, t);
    if (p) {
      const V b = __ldg(&a.w2_z[2 * t]);
#pragma unroll
      for (int e = 0; e < E; ++e) v[e] = cmulc<true>(v[e], zphase<T, NZ>(a.w2_z, b, 2 * (t + G * e), e));
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
      v[e].x += __shfl_xor_sync(0xffffffffu, v[e].x, G);
      v[e].y += __shfl_xor_sync(0xffffffffu, v[e].y, G);
    }
    if (col < ncols) {
      V* dst = reinterpret_cast<V*>(a.phi + size_t(col) * NZ);
#pragma unroll
      for (int e2 = 0; e2 < E / 2; ++e2) {
        const int e = e2 + p * (E / 2);
        dst[t + G * e] = p ? v[e2 + E / 2] : v[e2];
      }
    }
    __syncthreads();                 // this buffer is refilled by the next issue
  }
}

}  // namespace pp
