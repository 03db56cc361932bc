// FP32 projection and back-projection of the mode-space solve for meshes
// symmetric in y with ny/2 in {16, 32, 64, 128} rows per half: the same sums as
// mode_project / mode_back (modes_impl.cuh), laid out for occupancy.
//
// A CTA of 16 warps covers 16 x rows and 32 consecutive z (one per lane), so
// every warp load or store of the fields is a run of 32 z values.
//   projection:      A[x][n][z] = sum_{j < ny/2} Sy[j][n] (rho[x][j][z] +- rho[x][ny-1-j][z])
//                    (+ for odd n, - for even n), one thread per (x row, z) with
//                    the y-mode table as a kernel parameter (constant bank) and
//                    the warp's field rows staged through a cp.async ring; then
//                    the x-mode sums over the CTA's rows,
//                    P[m][n][z] = sum_x Sx[x][m] A[x][n][z], and the cluster's
//                    CTAs added up through distributed shared memory, in rank
//                    order (as mode_project).
//   back-projection: B[x][n][z] = sum_m Sx[x][m] psi[m][n][z] (psi chunk in
//                    shared memory, computed once per CTA), then
//                    phi[x][j][z] = O + E and phi[x][ny-1-j][z] = O - E with O, E
//                    the sums of Sy[j][n] B[x][n][z] over odd and even n, the
//                    table again a kernel parameter; a thread holds the B values
//                    of two x rows (up to 20 y-mode slots; the two warps of an x
//                    pair split the rows j) or of one, and sums slot pairs with
//                    the packed FP32 FMA (fma.rn.f32x2) where ny/2 <= 64.
//
// The two x-mode sums are small matrix products per CTA, [(n, z)] x [x] by
// [x] x [m] and [(n, z)] x [m] by [m] x [x], and run on the tensor cores as
// warp-level TF32 MMA (mma.sync m16n8k8) at FP32 accuracy: each operand v is
// split as v = hi + lo, hi = tf32(v) (round to nearest, 11 significant bits),
// lo = tf32(v - hi), and a product is taken as lo*hi + hi*lo + hi*hi with FP32
// accumulation (the dropped lo*lo is below 2^-22 of it).  Fragment layout of
// m16n8k8 (lane = 4g + t): A (16 x 8, row major) (g, t), (g+8, t), (g, t+4),
// (g+8, t+4); B (8 x 8, column major) (t, g), (t+4, g); C (16 x 8) (g, 2t),
// (g, 2t+1), (g+8, 2t), (g+8, 2t+1).  A tile's 16 rows are 16 z of one n; the
// shared-memory rows are padded so that the fragment reads and writes of a
// warp fall on 32 distinct banks.  (The same products on tcgen05 were slower:
// with K = 16 x rows per CTA, staging the operands in K-major core matrices
// costs more than the faster tensor pipe saves.)
#include "modes.cuh"
#include "modes_impl.cuh"

namespace pp {

namespace {

constexpr int kW = 16;                    // warps per CTA
constexpr int kX = 16;                    // x rows per CTA
constexpr int kZC = 32;                   // z values per CTA

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_rna(x);
  lo = tf32_rna(x - __uint_as_float(hi));
}
// d += a * b on one m16n8k8 tile
__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
// d += (ah + al) * (bh + bl), the three terms that matter, small ones first
__device__ __forceinline__ void mma3(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4],
                                     const uint32_t (&bh)[2], const uint32_t (&bl)[2]) {
  mma_tf32(d, al[0], al[1], al[2], al[3], bh[0], bh[1]);
  mma_tf32(d, ah[0], ah[1], ah[2], ah[3], bl[0], bl[1]);
  mma_tf32(d, ah[0], ah[1], ah[2], ah[3], bh[0], bh[1]);
}
// the A fragment of rows (g, g+8) and columns (k, k+4) of a row-major tile
// whose column k + 1 is cs floats after column k (p already at row g, column t);
// columns switched off read as zero
__device__ __forceinline__ void load_a(const float* p, int cs, bool on_lo, bool on_hi, uint32_t (&ah)[4],
                                       uint32_t (&al)[4]) {
  split_tf32(on_lo ? p[0] : 0.f, ah[0], al[0]);
  split_tf32(on_lo ? p[8] : 0.f, ah[1], al[1]);
  split_tf32(on_hi ? p[4 * cs] : 0.f, ah[2], al[2]);
  split_tf32(on_hi ? p[4 * cs + 8] : 0.f, ah[3], al[3]);
}

}  // namespace

// the y-mode table as a kernel parameter: with the y loops unrolled, each
// value is read at a compile-time offset of the constant bank
template <int NYH, int MYP>
struct SyTab {
  float s[NYH * MYP];
};

// Per-warp staging of the projection's field rows: a ring of kStages buffers
// of kPairs rows j and their mirrors ny-1-j (32 z each), filled by cp.async so
// that the next rows of each warp are in flight without holding registers.  A
// warp's ring and, after its y sums, its row of A[x][n][z] share one slot of
// shared memory (slot_a floats, 8 beyond a multiple of 32 so that the x-mode
// pass's fragment rows t and t + 4 fall on different banks).
constexpr int kPairs = 4;
constexpr int kStages = 3;
constexpr int kRing = kStages * 2 * kPairs * kZC;
template <int MYP>
constexpr int slot_a() { return ((kRing > MYP * kZC ? kRing : MYP * kZC) + 31) / 32 * 32 + 8; }
// row stride (floats) of the back-projection's psi chunk [m][n][z] (8 beyond a
// multiple of 32) and of its B[x][n][z] (4 beyond: rows 2t and 2t + 1 apart)
template <int MYP> constexpr int rows_p() { return MYP * kZC + 8; }
template <int MYP> constexpr int rows_b() { return MYP * kZC + 4; }
// column stride of the projection's x-mode sums P[m][n][z] (the DSMEM
// reduction reads runs of consecutive z)
constexpr int kCS = kZC + 1;
// x rows per thread of the back-projection's y sums (its registers hold
// XR * MYP values of B)
template <int MYP>
constexpr int back_rows_per_thread() { return MYP <= 20 ? 2 : 1; }

// one thread per (x row, z): the 16 warps of a CTA take its 16 x rows; the
// CTA's tile is z chunk zc, x block xb (its cluster: consecutive x blocks)
template <int NYH, int MYP>
__device__ __forceinline__ void project_fast(const ModeArgs<float>& a, const SyTab<NYH, MYP>& tab, int zc, int xb) {
  constexpr int RS = slot_a<MYP>();
  constexpr int KS = kX / 8;                                   // k steps over the CTA's x rows
  constexpr int NS = NYH / kPairs;                             // ring stages over the half rows
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* abuf = reinterpret_cast<float*>(smem_raw);            // [16][RS]: ring, then A[x][n][z]
  float* red = abuf + kX * RS;                                 // [mc][33]: P[m][n][z]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int z0 = zc * kZC;
  const int xb0 = xb * kX;
  const int ny = 2 * NYH;

  float* ring = abuf + warp * RS;
  const float* xrow = a.rho + size_t(xb0 + warp) * ny * a.nz + z0;
  // stage s: rows s*kPairs + r (r < kPairs) and their mirrors, 16 bytes a lane a copy
  auto issue = [&](int s) {
    float* buf = ring + (s % kStages) * (2 * kPairs * kZC);
#pragma unroll
    for (int k = 0; k < 2 * kPairs * kZC / 4 / 32; ++k) {
      const int idx = k * 32 + lane, r = idx >> 3, piece = idx & 7;
      const int j = r < kPairs ? s * kPairs + r : ny - 1 - (s * kPairs + r - kPairs);
      cp_async16(buf + r * kZC + 4 * piece, xrow + size_t(j) * a.nz + 4 * piece);
    }
    cp_async_commit();
  };
  float acc[MYP];
#pragma unroll
  for (int n = 0; n < MYP; ++n) acc[n] = 0.f;
#pragma unroll
  for (int s = 0; s < kStages - 1; ++s) issue(s);
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    // groups committed: stages 0 .. min(s + kStages - 2, NS - 1); stage s must be in
    if (s + kStages - 1 <= NS) cp_async_wait<kStages - 2>();
    else cp_async_wait<0>();
    __syncwarp();
    if (s + kStages - 1 < NS) issue(s + kStages - 1);          // the buffer read at stage s - 1
    const float* buf = ring + (s % kStages) * (2 * kPairs * kZC);
#pragma unroll
    for (int r = 0; r < kPairs; ++r) {
      const float u = buf[r * kZC + lane], v = buf[(kPairs + r) * kZC + lane];
      const float p = u + v, q = u - v;
      const int j = s * kPairs + r;
#pragma unroll
      for (int n = 0; n < MYP; ++n) acc[n] = fmaf(tab.s[j * MYP + n], n < MYP / 2 ? p : q, acc[n]);
    }
  }
  __syncwarp();                                                // ring reads done before A overwrites it
#pragma unroll
  for (int n = 0; n < MYP; ++n) abuf[warp * RS + n * kZC + lane] = acc[n];
  const int mtiles = (a.mxp + 7) / 8;
  const float* sxb = a.sx + size_t(xb0 + t) * a.mxp + g;     // B[k = x][col = m] = Sx[xb0 + x][m]
  __syncthreads();

  // P^T[(n, z)][m] = sum_x A[x][n][z] Sx[x][m]: tile = (n, 16 z), warp-strided
#pragma unroll 1
  for (int tile = warp; tile < 2 * MYP; tile += kW) {
    const int n = tile >> 1, zz = (tile & 1) * 16;
    uint32_t ah[KS][4], al[KS][4];
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) load_a(abuf + (8 * ks + t) * RS + n * kZC + zz + g, RS, true, true, ah[ks], al[ks]);
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      if (nt < mtiles) {
        const bool on = 8 * nt + g < a.mxp;
        float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
          uint32_t bh[2], bl[2];
          split_tf32(on ? __ldg(sxb + (8 * ks) * a.mxp + 8 * nt) : 0.f, bh[0], bl[0]);
          split_tf32(on ? __ldg(sxb + (8 * ks + 4) * a.mxp + 8 * nt) : 0.f, bh[1], bl[1]);
          mma3(d, ah[ks], al[ks], bh, bl);
        }
        const int m = 8 * nt + 2 * t;                  // mxp is a multiple of 4: m, m + 1 both in or out
        if (m < a.mxp) {
          float* r = red + (m * MYP + n) * kCS + zz + g;
          r[0] = d[0];
          r[MYP * kCS] = d[1];
          r[8] = d[2];
          r[MYP * kCS + 8] = d[3];
        }
      }
    }
  }

  // the cluster's CTAs added up in rank order, each CTA a slice of the columns
  mcg::cluster_group cl = mcg::this_cluster();
  cl.sync();
  const int ncl = int(cl.num_blocks()), rank = int(cl.block_rank());
  const int per = (a.mc + ncl - 1) / ncl;
  const int c0 = rank * per, c1 = c0 + per < a.mc ? c0 + per : a.mc;
  float* out = a.part + size_t(xb / ncl) * a.mc * a.nz + z0 + lane;
#pragma unroll 1
  for (int c = c0 + warp; c < c1; c += kW) {
    float v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = r < ncl ? cl.map_shared_rank(red, r)[c * kCS + lane] : 0.f;
    float sum = 0.f;
#pragma unroll
    for (int r = 0; r < 8; ++r) sum += v[r];
    out[size_t(c) * a.nz] = sum;
  }
  cl.sync();
}

// d = a * b + c on both halves of a pair (the packed FP32 FMA of sm_100 and
// later: one instruction for two FMAs, each rounded as fmaf)
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{.reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}

// rows j = J0 .. J0 + NJ - 1 of XR x rows (xs apart) and their mirrors
// ny-1-j, the y-mode table read at compile-time offsets of the constant bank
template <int NYH, int MYP, int XR, int J0, int NJ>
__device__ __forceinline__ void back_rows(const float (&bv)[XR][MYP], const SyTab<NYH, MYP>& tab, float* base,
                                          int nz, int xs) {
  constexpr int H = MYP / 2;
  float* lo = base + J0 * nz;
  float* hi = base + (2 * NYH - 1 - J0) * nz;
#pragma unroll
  for (int jj = 0; jj < NJ; ++jj) {
    const int j = J0 + jj;
    float o[XR], e[XR];
#pragma unroll
    for (int i = 0; i < XR; ++i) o[i] = e[i] = 0.f;
#pragma unroll
    for (int n = 0; n < MYP; ++n) {
      const float s = tab.s[j * MYP + n];
#pragma unroll
      for (int i = 0; i < XR; ++i) {
        if (n < H) o[i] = fmaf(s, bv[i][n], o[i]);
        else e[i] = fmaf(s, bv[i][n], e[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < XR; ++i) {
      lo[i * xs] = o[i] + e[i];
      hi[i * xs] = o[i] - e[i];
    }
    lo += nz;
    hi -= nz;
    // one running pointer per mirror, not one precomputed address per row
    asm volatile("" : "+l"(lo), "+l"(hi));
  }
}

// the same with bv[i][p] holding slots 2p and 2p + 1, summed as pairs by packed FMAs (MYP / 2
// is even, so no pair straddles the odd and even halves)
template <int NYH, int MYP, int XR, int J0, int NJ>
__device__ __forceinline__ void back_rows2(const float2 (&bv)[XR][MYP / 2], const SyTab<NYH, MYP>& tab, float* base,
                                          int nz, int xs) {
  constexpr int H = MYP / 2;
  static_assert(H % 2 == 0, "slot pairs must not straddle the odd and even halves");
  float* lo = base + J0 * nz;
  float* hi = base + (2 * NYH - 1 - J0) * nz;
#pragma unroll
  for (int jj = 0; jj < NJ; ++jj) {
    const int j = J0 + jj;
    float2 o[XR], e[XR];
#pragma unroll
    for (int i = 0; i < XR; ++i) o[i] = e[i] = make_float2(0.f, 0.f);
#pragma unroll
    for (int p = 0; p < MYP / 2; ++p) {
      const float2 s = make_float2(tab.s[j * MYP + 2 * p], tab.s[j * MYP + 2 * p + 1]);
#pragma unroll
      for (int i = 0; i < XR; ++i) {
        if (2 * p < H) o[i] = ffma2(s, bv[i][p], o[i]);
        else e[i] = ffma2(s, bv[i][p], e[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < XR; ++i) {
      const float os = o[i].x + o[i].y, es = e[i].x + e[i].y;
      lo[i * xs] = os + es;
      hi[i * xs] = os - es;
    }
    lo += nz;
    hi -= nz;
    // one running pointer per mirror, not one precomputed address per row
    asm volatile("" : "+l"(lo), "+l"(hi));
  }
}

template <int NYH, int MYP>
__device__ __forceinline__ void back_fast(const ModeArgs<float>& a, const SyTab<NYH, MYP>& tab, int zc, int xb) {
  constexpr int RS = rows_p<MYP>(), BS = rows_b<MYP>();
  constexpr int XT = kX / 8;                         // n tiles over the CTA's x rows
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* ps = reinterpret_cast<float*>(smem_raw);    // psi chunk [mx][RS]: psi[m][n][z]
  float* bvs = ps + size_t(a.mx) * RS;               // x-mode sums [16][BS]: B[x][n][z]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int pair = warp % (kW / 2), half = warp / (kW / 2);
  const int z0 = zc * kZC;
  const int xb0 = xb * kX;
  const int ny = 2 * NYH;
  for (int idx = threadIdx.x; idx < a.mx * MYP * (kZC / 4); idx += 32 * kW) {
    const int c = idx / (kZC / 4), piece = idx % (kZC / 4);
    cp_async16(ps + (c / MYP) * RS + (c % MYP) * kZC + 4 * piece, a.psi + size_t(c) * a.nz + z0 + 4 * piece);
  }
  cp_async_commit();
  const int ksteps = (a.mxp + 7) / 8;
  const float* sxb = a.sx + size_t(xb0 + g) * a.mxp + t;     // B[k = m][col = x] = Sx[xb0 + x][m]
  cp_async_wait<0>();
  __syncthreads();

  // B^T[(n, z)][x] = sum_m psi[m][n][z] Sx[x][m]: tile = (n, 16 z), warp-strided
#pragma unroll 1
  for (int tile = warp; tile < 2 * MYP; tile += kW) {
    const int n = tile >> 1, zz = (tile & 1) * 16;
    float d[XT][4];
#pragma unroll
    for (int nt = 0; nt < XT; ++nt) d[nt][0] = d[nt][1] = d[nt][2] = d[nt][3] = 0.f;
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
      if (ks < ksteps) {
        // rows m >= mx of psi are zero (read as zero; the rows stay inside
        // the buffer: m < mx + 8 and B's 16 rows follow the chunk)
        const int m = 8 * ks + t;
        uint32_t ah[4], al[4];
        load_a(ps + m * RS + n * kZC + zz + g, RS, m < a.mx, m + 4 < a.mx, ah, al);
#pragma unroll
        for (int nt = 0; nt < XT; ++nt) {
          uint32_t bh[2], bl[2];
          const float* sp = sxb + size_t(8 * nt) * a.mxp + 8 * ks;
          split_tf32(m < a.mxp ? __ldg(sp) : 0.f, bh[0], bl[0]);
          split_tf32(m + 4 < a.mxp ? __ldg(sp + 4) : 0.f, bh[1], bl[1]);
          mma3(d[nt], ah, al, bh, bl);
        }
      }
    }
#pragma unroll
    for (int nt = 0; nt < XT; ++nt) {
      float* r = bvs + (8 * nt + 2 * t) * BS + n * kZC + zz + g;
      r[0] = d[nt][0];
      r[BS] = d[nt][1];
      r[8] = d[nt][2];
      r[BS + 8] = d[nt][3];
    }
  }
  __syncthreads();

  // XR x rows a thread: two (the two warps of an x pair split the rows j)
  // up to 20 y-mode slots, else one (a warp takes all rows j of its x row)
  constexpr int XR = back_rows_per_thread<MYP>();
  const int x0 = XR == 2 ? 2 * pair : warp;
  float* base = a.phi + size_t(xb0 + x0) * ny * a.nz + z0 + lane;
  if constexpr (NYH <= 64) {
    // packed FMAs over slot pairs (at ny/2 = 128 the longer unrolled row
    // loop spills with them, so that size keeps one FMA per slot)
    float2 bv[XR][MYP / 2];
#pragma unroll
    for (int i = 0; i < XR; ++i)
#pragma unroll
      for (int p = 0; p < MYP / 2; ++p)
        bv[i][p] = make_float2(bvs[(x0 + i) * BS + 2 * p * kZC + lane], bvs[(x0 + i) * BS + (2 * p + 1) * kZC + lane]);
    if (XR == 1)
      back_rows2<NYH, MYP, XR, 0, NYH>(bv, tab, base, a.nz, ny * a.nz);
    else if (half == 0)
      back_rows2<NYH, MYP, XR, 0, NYH / 2>(bv, tab, base, a.nz, ny * a.nz);
    else
      back_rows2<NYH, MYP, XR, NYH / 2, NYH / 2>(bv, tab, base, a.nz, ny * a.nz);
  } else {
    float bv[XR][MYP];
#pragma unroll
    for (int i = 0; i < XR; ++i)
#pragma unroll
      for (int n = 0; n < MYP; ++n) bv[i][n] = bvs[(x0 + i) * BS + n * kZC + lane];
    if (XR == 1)
      back_rows<NYH, MYP, XR, 0, NYH>(bv, tab, base, a.nz, ny * a.nz);
    else if (half == 0)
      back_rows<NYH, MYP, XR, 0, NYH / 2>(bv, tab, base, a.nz, ny * a.nz);
    else
      back_rows<NYH, MYP, XR, NYH / 2, NYH / 2>(bv, tab, base, a.nz, ny * a.nz);
  }
}

// one solve: grid (nz / 32, nx / 16)
template <int NYH, int MYP>
__global__ void __launch_bounds__(32 * kW, 2)
    mode_project_fast_kernel(ModeArgs<float> a, const __grid_constant__ SyTab<NYH, MYP> tab) {
  project_fast<NYH, MYP>(a, tab, int(blockIdx.x), int(blockIdx.y));
}
template <int NYH, int MYP>
__global__ void __launch_bounds__(32 * kW, 2)
    mode_back_fast_kernel(ModeArgs<float> a, const __grid_constant__ SyTab<NYH, MYP> tab) {
  back_fast<NYH, MYP>(a, tab, int(blockIdx.x), int(blockIdx.y));
}

// a group of solves of one shape and one y-mode table (ModeGroup): grid
// (n * nz / 32, nx / 16), solve s taking the z chunks s * nz/32 ..; the
// same arithmetic per solve as the single-solve kernels
template <int NYH, int MYP>
__global__ void __launch_bounds__(32 * kW, 2)
    mode_project_group_kernel(const __grid_constant__ ModeGroup g, const __grid_constant__ SyTab<NYH, MYP> tab) {
  const int zpc = g.nz / kZC, s = int(blockIdx.x) / zpc;
  ModeArgs<float> a = g.args[s];
  a.rho = g.rho[s];
  project_fast<NYH, MYP>(a, tab, int(blockIdx.x) % zpc, int(blockIdx.y));
}
template <int NYH, int MYP>
__global__ void __launch_bounds__(32 * kW, 2)
    mode_back_group_kernel(const __grid_constant__ ModeGroup g, const __grid_constant__ SyTab<NYH, MYP> tab) {
  const int zpc = g.nz / kZC, s = int(blockIdx.x) / zpc;
  ModeArgs<float> a = g.args[s];
  a.phi = g.phi[s];
  back_fast<NYH, MYP>(a, tab, int(blockIdx.x) % zpc, int(blockIdx.y));
}

namespace {

template <typename K>
cudaError_t big_smem(K kern, size_t smem) {
  if (smem > kMaxSmem) return cudaErrorInvalidConfiguration;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
}

// stage `which` (0 projection, 1 back-projection) of one solve (g == nullptr)
// or of a group of solves shaped like `a`
template <int NYH, int MYP>
cudaError_t launch_fast(int which, const ModeArgs<float>& a, const ModeGroup* g, const float* sy_host,
                        cudaStream_t st) {
  const int xblocks = a.nx / kX;
  const dim3 grid(unsigned((g ? g->n : 1) * (a.nz / kZC)), unsigned(xblocks));
  SyTab<NYH, MYP> tab;
  for (int i = 0; i < NYH * MYP; ++i) tab.s[i] = sy_host[i];
  cudaError_t e;
  if (which == 0) {
    const size_t smem = sizeof(float) * (size_t(kX) * slot_a<MYP>() + size_t(a.mc) * kCS);
    void (*kern)(ModeArgs<float>, const SyTab<NYH, MYP>) = mode_project_fast_kernel<NYH, MYP>;
    void (*gkern)(const ModeGroup, const SyTab<NYH, MYP>) = mode_project_group_kernel<NYH, MYP>;
    if ((e = g ? big_smem(gkern, smem) : big_smem(kern, smem)) != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(32 * kW, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = unsigned(mode_cluster(xblocks));
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return g ? cudaLaunchKernelEx(&cfg, gkern, *g, tab) : cudaLaunchKernelEx(&cfg, kern, a, tab);
  }
  const size_t smem = sizeof(float) * (size_t(a.mx) * rows_p<MYP>() + size_t(kX) * rows_b<MYP>());
  void (*kern)(ModeArgs<float>, const SyTab<NYH, MYP>) = mode_back_fast_kernel<NYH, MYP>;
  void (*gkern)(const ModeGroup, const SyTab<NYH, MYP>) = mode_back_group_kernel<NYH, MYP>;
  if ((e = g ? big_smem(gkern, smem) : big_smem(kern, smem)) != cudaSuccess) return e;
  if (g) gkern<<<grid, 32 * kW, smem, st>>>(*g, tab);
  else kern<<<grid, 32 * kW, smem, st>>>(a, tab);
  return cudaGetLastError();
}

template <int NYH>
cudaError_t launch_fast2(int which, int myp, const ModeArgs<float>& a, const ModeGroup* g, const float* sy_host,
                         cudaStream_t st) {
  switch (myp) {
    case 8: return launch_fast<NYH, 8>(which, a, g, sy_host, st);
    case 12: return launch_fast<NYH, 12>(which, a, g, sy_host, st);
    case 16: return launch_fast<NYH, 16>(which, a, g, sy_host, st);
    case 20: return launch_fast<NYH, 20>(which, a, g, sy_host, st);
    case 24: return launch_fast<NYH, 24>(which, a, g, sy_host, st);
    case 32: return launch_fast<NYH, 32>(which, a, g, sy_host, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_fast_any(int stage, int myp, const ModeArgs<float>& a, const ModeGroup* g, const float* sy_host,
                            cudaStream_t st) {
  const int which = stage == 0 ? 0 : 1;
  switch (a.ny / 2) {
    case 16: return launch_fast2<16>(which, myp, a, g, sy_host, st);
    case 32: return launch_fast2<32>(which, myp, a, g, sy_host, st);
    case 64: return launch_fast2<64>(which, myp, a, g, sy_host, st);
    case 128: return launch_fast2<128>(which, myp, a, g, sy_host, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool mode_fast_ok(int ny, int nx, int myp, bool fy) {
  const int nyh = ny / 2;
  return fy && (nyh == 16 || nyh == 32 || nyh == 64 || nyh == 128) && nx % kX == 0 &&
         (myp == 8 || myp == 12 || myp == 16 || myp == 20 || myp == 24 || myp == 32);
}

// stage 0 (projection) or 2 (back-projection) of an FP32 handle that
// mode_fast_ok accepts
cudaError_t launch_mode_fast(int stage, int myp, const ModeArgs<float>& a, const float* sy_host, cudaStream_t st) {
  return launch_fast_any(stage, myp, a, nullptr, sy_host, st);
}

// the same stage for a group of such solves of one shape and one y-mode table
// (g->args[s] shaped like a)
cudaError_t launch_mode_fast_group(int stage, int myp, const ModeArgs<float>& a, const ModeGroup& g,
                                   const float* sy_host, cudaStream_t st) {
  if (g.n < 1 || g.n > kMaxModeGroup) return cudaErrorInvalidValue;
  return launch_fast_any(stage, myp, a, &g, sy_host, st);
}

}  // namespace pp
