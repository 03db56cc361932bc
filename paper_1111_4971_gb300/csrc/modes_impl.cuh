// Mode-space form of the pipe operator: the solve of Sec. 2 Eq. 10 with its
// transverse transforms pruned to the frequencies where the transformed Green
// function is not zero.
//
// Why this is the same operator.  The Green function is the truncated sine
// series of Eq. 7,
//     G = (8 pi / ab) sum_{m <= Mx, n <= My} kappa_mn^{-1} sin(m pi x/a) sin(m pi x'/a)
//                                          sin(n pi y/b) sin(n pi y'/b) f_mn(z - z'),
// f_mn = e^{-kappa |w|} (Eq. 9) or the longitudinal IGF g_z (Eq. 15-16), so
// the discrete sum of Eq. 4 factorises exactly into
//     rhot[m][n][k] = sum_{i,j} Sx[m][i] Sy[n][j] rho[i][j][k]          (projection)
//     psi[m][n][k]  = sum_{k'} K_mn(k - k') rhot[m][n][k']             (z convolution)
//     phi[i][j][k]  = sum_{m,n} Sx[m][i] Sy[n][j] psi[m][n][k]          (back-projection)
// with Sx[m][i] = sin(m pi x_i / a), Sy likewise, and
// K_mn(d) = hx hy hz (8 pi / ab) kappa_mn^{-1} f_mn(d hz).  On a mesh that
// spans the pipe the 2n-point transforms of Eq. 10 along x and y are, for a
// Green table built from these modes, nonzero only at |kx| <= Mx, |ky| <= My
// (the closed-form spectrum), and their products with the transformed density
// are exactly these mode sums; the projection is those transforms evaluated at
// the Mx x My frequencies that survive the product, and the back-projection
// the inverse transforms restricted to them.  The form holds on any mesh
// inside the pipe (windows included).  The z convolution is the zero-padded
// 2nz-point transform of Appendix A (Eq. A.1-A.4): a real-to-complex FFT of
// each mode's column, the product with the DCT-I of the doubled kernel table
// (scaled by 1 / 2nz), and the inverse, with the z-axis routines of the full
// solve.
//
// The operator is symmetric (G(r, r') = G(r', r)): the projection and the
// back-projection use the same tables and the z kernel is even, so the
// adjoint is the same computation.
//
// Kernels (one warp lane per z value of a 32-value z chunk, so that every
// global access is a run of 32 consecutive z):
//   mode_project_kernel  rho -> part[g][c][k]  (c = m' * MYP + n'; the
//                        projection of one group of x blocks, those of one
//                        thread-block cluster; the z kernel sums the groups)
//   mode_z_kernel        part -> psi[c][k]
//   mode_back_kernel     psi -> phi
// FY: the mesh is symmetric about the pipe's mid-plane in y
// (y_{ny-1-j} = b - y_j), so Sy[n][ny-1-j] = (-1)^{n+1} Sy[n][j]; the tables
// then hold the odd n first and the even n after them (MYP/2 slots each), and
// each sum over j runs over half the rows on rho(j) + rho(ny-1-j) (odd n) and
// rho(j) - rho(ny-1-j) (even n).
#pragma once

#include <cooperative_groups.h>

#include "zfft_impl.cuh"

namespace pp {

namespace mcg = cooperative_groups;

template <typename T>
struct ModeArgs {
  const T* rho;          // [nx][ny][nz]
  T* phi;                // [nx][ny][nz]
  T* part;               // [nx / (XB * cluster)][mc][nz]
  T* psi;                // [mc][nz]
  const T* sx;           // [nx][mxp]
  const T* sy;           // [FY ? ny/2 : ny][MYP]
  const T* gz;           // [mc][nz+1]: DCT-I of the doubled kernel table / 2nz
  const C2<T>* tw_z;     // z group-FFT twiddles (length nz/2)
  const C2<T>* w2_z;     // w_{2nz}^j, j < 2nz
  int nx, ny, nz;
  int mx;                // x modes
  int mxp;               // x modes padded to a multiple of 4 (columns of sx)
  int mc;                // mxp * MYP mode columns
  const T* kb;           // banded operator: [mc][nb+1] real-space z kernel K_c(d), d = 0..nb
  int nb;                // neighbour planes of the banded operator (Eq. 18), -1: the full z convolution
};

template <typename T, int MYP, bool FY>
struct ProjCfg {
  using S = ModeShape<T>;
  static constexpr int ROWS = FY ? 2 * S::YK : S::YK;
  static constexpr size_t STAGE = size_t(S::XB) * ROWS * S::ZC;     // elements
  static constexpr size_t ABUF = size_t(S::XB) * MYP * S::ZC;
  __host__ __device__ static size_t union_elems(int mxp) { return mode_proj_union<T>(mxp, MYP, FY); }
};

// four consecutive table values from shared memory (16-byte aligned)
template <typename T>
__device__ __forceinline__ void load4(const T* p, T (&s)[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    s[0] = v.x; s[1] = v.y; s[2] = v.z; s[3] = v.w;
  } else {
    const double2 u = reinterpret_cast<const double2*>(p)[0], v = reinterpret_cast<const double2*>(p)[1];
    s[0] = u.x; s[1] = u.y; s[2] = v.x; s[3] = v.y;
  }
}

// Projection of one (z chunk, x block): grid (nz / ZC, nx / XB), launched in
// clusters of consecutive x blocks of one z chunk.  The rows of the block
// arrive YK at a time (with their mirror rows under FY) in a ring of STAGES
// buffers filled by cp.async; each thread accumulates, for its XPW x rows and
// its z, the MYP y-mode sums; these go through shared memory so that each
// warp then sums, over the block's XB rows, the x modes of its passes into
// the block's projection (shared memory).  The cluster's CTAs then add up
// their blocks' projections through distributed shared memory, each CTA a
// slice of the mode columns, in a fixed order (rank 0 first), and write one
// partial per cluster.
template <typename T, int MYP, bool FY>
__device__ __forceinline__ void mode_project(const ModeArgs<T>& a, unsigned char* smem_raw) {
  using S = ModeShape<T>;
  using Cfg = ProjCfg<T, MYP, FY>;
  static_assert(MYP % 4 == 0, "mode slots in fours");
  T* slab = reinterpret_cast<T*>(smem_raw);
  T* abuf = slab;                                   // once the slab is consumed
  T* red = abuf + Cfg::ABUF;                        // one round of the block's projection [.][ZC]
  T* sy = slab + Cfg::union_elems(a.mxp);
  T* sxs = sy + (FY ? a.ny / 2 : a.ny) * MYP;       // x-mode rows of the block [XB][mxp]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int z0 = int(blockIdx.x) * S::ZC;
  const int xb0 = int(blockIdx.y) * S::XB;
  const int nyk = FY ? a.ny / 2 : a.ny;
  const int nchunks = nyk / S::YK;
  constexpr int PPR = S::ZC * int(sizeof(T)) / 16;  // 16-byte pieces of a row's z chunk

  // stage c: rows yc .. yc+YK-1 and (FY) ny-yc-YK .. ny-yc-1, yc = c * YK
  auto issue = [&](int c) {
    T* dst = slab + size_t(c % S::STAGES) * Cfg::STAGE;
    const int yc = c * S::YK;
    for (int idx = threadIdx.x; idx < S::XB * Cfg::ROWS * PPR; idx += S::THREADS) {
      const int piece = idx % PPR;
      const int r = (idx / PPR) % Cfg::ROWS;
      const int xl = idx / (PPR * Cfg::ROWS);
      const int y = r < S::YK ? yc + r : a.ny - yc - S::YK + (r - S::YK);
      const T* src = a.rho + (size_t(xb0 + xl) * a.ny + y) * a.nz + z0;
      cp_async16(reinterpret_cast<unsigned char*>(dst + size_t(xl * Cfg::ROWS + r) * S::ZC) + 16 * piece,
                 reinterpret_cast<const unsigned char*>(src) + 16 * piece);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int c = 0; c < S::STAGES - 1; ++c) {
    if (c < nchunks) issue(c);
    else cp_async_commit();
  }
  for (int i = threadIdx.x; i < nyk * MYP; i += S::THREADS) sy[i] = a.sy[i];
  for (int i = threadIdx.x; i < S::XB * a.mxp; i += S::THREADS) sxs[i] = a.sx[size_t(xb0) * a.mxp + i];

  T acc[S::XPW][MYP];
#pragma unroll
  for (int i = 0; i < S::XPW; ++i)
#pragma unroll
    for (int n = 0; n < MYP; ++n) acc[i][n] = T(0);

#pragma unroll 1
  for (int c = 0; c < nchunks; ++c) {
    cp_async_wait<S::STAGES - 2>();
    __syncthreads();               // stage c landed for every thread; stage c-1 is free
    if (c + S::STAGES - 1 < nchunks) issue(c + S::STAGES - 1);
    else cp_async_commit();
    const T* st = slab + size_t(c % S::STAGES) * Cfg::STAGE;
#pragma unroll
    for (int j = 0; j < S::YK; ++j) {
      T pa[S::XPW], qa[S::XPW];
#pragma unroll
      for (int i = 0; i < S::XPW; ++i) {
        const int xl = warp * S::XPW + i;
        const T u = st[(xl * Cfg::ROWS + j) * S::ZC + lane];
        if constexpr (FY) {
          const T v = st[(xl * Cfg::ROWS + 2 * S::YK - 1 - j) * S::ZC + lane];
          pa[i] = u + v;
          qa[i] = u - v;
        } else {
          pa[i] = u;
          qa[i] = u;
        }
      }
      const T* srow = sy + (c * S::YK + j) * MYP;
#pragma unroll
      for (int g = 0; g < MYP; g += 4) {
        T s4[4];
        load4(srow + g, s4);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const bool odd_slot = !FY || (g + k < MYP / 2);
#pragma unroll
          for (int i = 0; i < S::XPW; ++i) acc[i][g + k] = fma(s4[k], odd_slot ? pa[i] : qa[i], acc[i][g + k]);
        }
      }
    }
  }
  cp_async_wait<0>();
  __syncthreads();                 // the slab becomes the buffer of y-mode sums
#pragma unroll
  for (int i = 0; i < S::XPW; ++i)
#pragma unroll
    for (int n = 0; n < MYP; ++n) abuf[((warp * S::XPW + i) * MYP + n) * S::ZC + lane] = acc[i][n];
  __syncthreads();

  // x modes, in rounds of mode_round_modes: warp w takes the passes of MQ
  // modes q = w, w + WARPS, ... of the round; then the cluster's blocks are
  // summed for the round's columns: CTA `rank` takes a slice of them and
  // reads them from every CTA in rank order
  mcg::cluster_group cl = mcg::this_cluster();
  const int ncl = int(cl.num_blocks()), rank = int(cl.block_rank());
  T* out = a.part + size_t(blockIdx.y / ncl) * a.mc * a.nz + z0 + lane;
  const int mpr = mode_round_modes<T>(a.mxp);
#pragma unroll 1
  for (int m0 = 0; m0 < a.mxp; m0 += mpr) {
    const int m1 = m0 + mpr < a.mxp ? m0 + mpr : a.mxp;
#pragma unroll 1
    for (int q = m0 / S::MQ + warp; q * S::MQ < m1; q += S::WARPS) {
      T acc2[S::MQ][MYP];
#pragma unroll
      for (int k = 0; k < S::MQ; ++k)
#pragma unroll
        for (int n = 0; n < MYP; ++n) acc2[k][n] = T(0);
#pragma unroll 2
      for (int xl = 0; xl < S::XB; ++xl) {
        T s[S::MQ];
#pragma unroll
        for (int k = 0; k < S::MQ; ++k) s[k] = sxs[xl * a.mxp + q * S::MQ + k];
#pragma unroll
        for (int n = 0; n < MYP; ++n) {
          const T av = abuf[(xl * MYP + n) * S::ZC + lane];
#pragma unroll
          for (int k = 0; k < S::MQ; ++k) acc2[k][n] = fma(s[k], av, acc2[k][n]);
        }
      }
#pragma unroll
      for (int k = 0; k < S::MQ; ++k)
#pragma unroll
        for (int n = 0; n < MYP; ++n) red[((q * S::MQ + k - m0) * MYP + n) * S::ZC + lane] = acc2[k][n];
    }
    cl.sync();                     // every block's projection of the round is complete
    const int nc = (m1 - m0) * MYP;
    const int per = (nc + ncl - 1) / ncl;
    const int c0 = rank * per, c1 = c0 + per < nc ? c0 + per : nc;
#pragma unroll 1
    for (int c = c0 + warp; c < c1; c += S::WARPS) {
      T sum = T(0);
#pragma unroll 1
      for (int r = 0; r < ncl; ++r) sum += cl.map_shared_rank(red, r)[c * S::ZC + lane];
      out[size_t(m0 * MYP + c) * a.nz] = sum;
    }
    cl.sync();                     // no CTA overwrites (or leaves) while its projection is still read
  }
}

// Back-projection of one (z chunk, x block): each thread forms, for its XPW x
// rows and its z, the MYP sums over the x modes (psi read from L2), then
// walks the y rows (pairs of mirror rows under FY) with the y-mode table in
// shared memory, writing phi one row of 32 z values per warp store.
template <typename T, int MYP, bool FY>
__device__ __forceinline__ void mode_back(const ModeArgs<T>& a, unsigned char* smem_raw) {
  using S = ModeShape<T>;
  const int nyk = FY ? a.ny / 2 : a.ny;
  T* ps = reinterpret_cast<T*>(smem_raw);           // psi chunk [mx * MYP][ZC]
  T* sy = ps + size_t(a.mx) * MYP * S::ZC;
  T* sxs = sy + nyk * MYP;                          // x-mode rows of the block [XB][mxp]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int z0 = int(blockIdx.x) * S::ZC;
  const int xb0 = int(blockIdx.y) * S::XB;
  const int x0 = xb0 + warp * S::XPW;
  {
    constexpr int PPR = S::ZC * int(sizeof(T)) / 16;
    for (int idx = threadIdx.x; idx < a.mx * MYP * PPR; idx += S::THREADS) {
      const int c = idx / PPR, piece = idx % PPR;
      cp_async16(reinterpret_cast<unsigned char*>(ps + size_t(c) * S::ZC) + 16 * piece,
                 reinterpret_cast<const unsigned char*>(a.psi + size_t(c) * a.nz + z0) + 16 * piece);
    }
    cp_async_commit();
  }
  for (int i = threadIdx.x; i < nyk * MYP; i += S::THREADS) sy[i] = a.sy[i];
  for (int i = threadIdx.x; i < S::XB * a.mxp; i += S::THREADS) sxs[i] = a.sx[size_t(xb0) * a.mxp + i];
  cp_async_wait<0>();
  __syncthreads();                 // psi chunk and tables in shared memory

  T bv[S::XPW][MYP];
#pragma unroll
  for (int i = 0; i < S::XPW; ++i)
#pragma unroll
    for (int n = 0; n < MYP; ++n) bv[i][n] = T(0);
#pragma unroll 2
  for (int m = 0; m < a.mx; ++m) {
    T s[S::XPW];
#pragma unroll
    for (int i = 0; i < S::XPW; ++i) s[i] = sxs[(warp * S::XPW + i) * a.mxp + m];
#pragma unroll
    for (int n = 0; n < MYP; ++n) {
      const T p = ps[(m * MYP + n) * S::ZC + lane];
#pragma unroll
      for (int i = 0; i < S::XPW; ++i) bv[i][n] = fma(s[i], p, bv[i][n]);
    }
  }

#pragma unroll 1
  for (int yh = 0; yh < nyk; ++yh) {
    const T* srow = sy + yh * MYP;
    T o[S::XPW], e[S::XPW];
#pragma unroll
    for (int i = 0; i < S::XPW; ++i) o[i] = e[i] = T(0);
#pragma unroll
    for (int g = 0; g < MYP; g += 4) {
      T s4[4];
      load4(srow + g, s4);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const bool odd_slot = !FY || (g + k < MYP / 2);
#pragma unroll
        for (int i = 0; i < S::XPW; ++i) {
          if (odd_slot) o[i] = fma(s4[k], bv[i][g + k], o[i]);
          else e[i] = fma(s4[k], bv[i][g + k], e[i]);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < S::XPW; ++i) {
      T* row = a.phi + (size_t(x0 + i) * a.ny + yh) * a.nz + z0 + lane;
      if constexpr (FY) {
        row[0] = o[i] + e[i];
        row[size_t(a.ny - 1 - 2 * yh) * a.nz] = o[i] - e[i];
      } else {
        row[0] = o[i];
      }
    }
  }
}

// z convolution of the mode columns, one column per group of L/4 threads
// (L = nz; a CTA of 256 threads takes 1024/L columns):
//   1. the packed column z_m = rhot(2m) + i rhot(2m+1), m < L/2 (the sum of
//      the groups' partial projections); z_m = 0 for m >= L/2 is the zero
//      padding of Appendix A, never stored;
//   2. Z = the L-point forward FFT of z (radix-4 Stockham in shared memory,
//      a radix-2 stage first when log2 L is odd; the first stage skips the
//      known-zero half of its inputs);
//   3. for each pair (k, L-k): the 2L-point real spectrum
//      X(k) = [Z(k) + conj Z(L-k) - i w^k (Z(k) - conj Z(L-k))] / 2, w = e^{-i pi / L},
//      times the kernel spectrum g(k), and the packed inverse input
//      Z'(k) = Y(k) + conj Y(L-k) + i w^{-k} (Y(k) - conj Y(L-k));
//   4. z' = the unnormalised L-point inverse FFT of Z' (the last stage only
//      computes the outputs m < L/2), y(2m) = Re z'_m, y(2m+1) = Im z'_m: the
//      first nz outputs of the 2nz-point inverse, which is psi.
// Twiddles come from the 2L-entry table w2[j] = e^{-2 pi i j / (2L)}, copied
// into shared memory at the start and rearranged there stage by stage so that
// the lanes of a stage read consecutive entries.
// the twiddles of the radix-4 stages with Ls > 1, stage after stage, each as
// [r-1][j] = w_{4 Ls}^{r j} (r = 1..3, j < Ls), so that the lanes of a stage
// (consecutive j) read consecutive entries; about L values in all
template <typename T>
__device__ __forceinline__ void stockham_twiddles(C2<T>* tws, const C2<T>* w2, int L) {
  int off = 0;
  for (int Ls = (__popc(L - 1) & 1) ? 2 : 4; Ls < L; Ls *= 4) {
    const int tstep = L / (2 * Ls);                  // w_{4 Ls}^{q} = w2[q * L / (2 Ls)]
    for (int i = int(threadIdx.x); i < 3 * Ls; i += int(blockDim.x)) {
      const int r = i / Ls + 1, j = i % Ls;
      tws[off + i] = w2[r * j * tstep];
    }
    off += 3 * Ls;
  }
}

template <typename T, bool INV>
__device__ __forceinline__ C2<T>* stockham(C2<T>* src, C2<T>* dst, int L, int tid, int nthr, const C2<T>* tws,
                                          bool prune_in, bool prune_out) {
  using V = C2<T>;
  int Ls = 1;
  if (__popc(L - 1) & 1) {                           // radix-2 stage first
    for (int t = tid; t < L / 2; t += nthr) {
      const V a0 = src[t];
      const V a1 = prune_in ? mk<V>(T(0), T(0)) : src[t + L / 2];
      dst[2 * t] = cadd(a0, a1);
      dst[2 * t + 1] = csub(a0, a1);
    }
    Ls = 2;
    prune_in = false;
    V* tmp = src; src = dst; dst = tmp;
    __syncthreads();
  }
  while (Ls < L) {
    const bool last = 4 * Ls == L;
    for (int t = tid; t < L / 4; t += nthr) {
      const int j = t % Ls;
      V a[4];
      a[0] = src[t];
      a[1] = src[t + L / 4];
      if (prune_in) {
        a[2] = a[3] = mk<V>(T(0), T(0));
      } else {
        a[2] = src[t + L / 2];
        a[3] = src[t + 3 * L / 4];
      }
      if (Ls > 1) {
#pragma unroll
        for (int r = 1; r < 4; ++r) a[r] = cmulc<INV>(a[r], tws[(r - 1) * Ls + j]);
      }
      dft_reg<4, INV>(a);
      V* o = dst + (t - j) * 4 + j;
      o[0] = a[0];
      o[Ls] = a[1];
      if (!(last && prune_out)) {
        o[2 * Ls] = a[2];
        o[3 * Ls] = a[3];
      }
    }
    if (Ls > 1) tws += 3 * Ls;
    Ls *= 4;
    prune_in = false;
    V* tmp = src; src = dst; dst = tmp;
    __syncthreads();
  }
  return src;
}

template <typename T>
__device__ __forceinline__ void mode_z(const ModeArgs<T>& a, int groups, unsigned char* smem_raw) {
  using V = C2<T>;
  const int L = a.nz;
  const int nthr = L / 4;                            // threads per column
  const int per = int(blockDim.x) / nthr;            // columns per CTA
  const int cl = int(threadIdx.x) / nthr, tid = int(threadIdx.x) % nthr;
  const int col = int(blockIdx.x) * per + cl;
  const bool valid = col < a.mc;
  // the twiddle table w2 (2L values, shared by the CTA's columns) first, then
  // two buffers of L values per column; the table arrives by cp.async, all of
  // it in flight at once, so its latency is paid once and not per stage
  V* w2 = reinterpret_cast<V*>(smem_raw);
  V* tws = w2 + 2 * L;                               // the stages' twiddles (< L values)
  V* bufa = tws + L + size_t(cl) * 2 * L;
  V* bufb = bufa + L;
  {
    constexpr int EPP = 16 / int(sizeof(V));          // values per 16-byte piece
    for (int i = int(threadIdx.x); i < 2 * L / EPP; i += int(blockDim.x)) cp_async16(w2 + EPP * i, a.w2_z + EPP * i);
    cp_async_commit();
  }
  // the kernel spectrum at this thread's pairs (k, L-k), read ahead
  const T* g = a.gz + size_t(valid ? col : 0) * (L + 1);
  T gk[3], gm[3];
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    const int k = tid + u * nthr;
    gk[u] = (valid && k <= L / 2) ? __ldg(&g[k]) : T(0);
    gm[u] = (valid && k <= L / 2) ? __ldg(&g[L - k]) : T(0);
  }
  // 1. packed column, summed over the groups
  for (int m = tid; m < L / 2; m += nthr) {
    V z = mk<V>(T(0), T(0));
    if (valid) {
#pragma unroll 4
      for (int s = 0; s < groups; ++s)
        z = cadd(z, __ldg(reinterpret_cast<const V*>(a.part + (size_t(s) * a.mc + col) * L) + m));
    }
    bufa[m] = z;
  }
  cp_async_wait<0>();
  __syncthreads();
  stockham_twiddles<T>(tws, w2, L);
  __syncthreads();
  // 2. forward transform
  V* Z = stockham<T, false>(bufa, bufb, L, tid, nthr, tws, true, false);
  V* Zp = Z == bufa ? bufb : bufa;
  // 3. real spectrum, kernel product, packed inverse input
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    const int k = tid + u * nthr;
    if (k > L / 2) continue;
    const V zk = Z[k], zm = Z[(L - k) & (L - 1)];
    const V wk = w2[k];                              // w^k
    const V wm = w2[L - k];                          // w^{L-k}
    auto unpack = [](V x, V xm, V w) {               // (x + conj xm - i w (x - conj xm)) / 2
      const V c = cconj(xm);
      const V s = cadd(x, c), d = csub(x, c);
      const V wd = cmul(w, d);
      return mk<V>(T(0.5) * (s.x + wd.y), T(0.5) * (s.y - wd.x));
    };
    auto repack = [](V y, V ym, V w) {               // y + conj ym + i conj(w) (y - conj ym)
      const V c = cconj(ym);
      const V s = cadd(y, c), d = csub(y, c);
      const V wd = cmulc<true>(d, w);
      return mk<V>(s.x - wd.y, s.y + wd.x);
    };
    const V yk = cscale(unpack(zk, zm, wk), gk[u]);
    const V ym = cscale(unpack(zm, zk, wm), gm[u]);
    Zp[k] = repack(yk, ym, wk);
    if (k > 0 && k < L / 2) Zp[L - k] = repack(ym, yk, wm);
  }
  __syncthreads();
  // 4. inverse transform, first L/2 outputs: psi
  V* zo = stockham<T, true>(Zp, Z, L, tid, nthr, tws, false, true);
  if (valid) {
    V* dst = reinterpret_cast<V*>(a.psi + size_t(col) * L);
    for (int m = tid; m < L / 2; m += nthr) dst[m] = zo[m];
  }
}

}  // namespace pp
