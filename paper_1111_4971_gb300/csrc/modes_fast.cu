// FP32 projection and back-projection of the mode-space solve for meshes
// symmetric in y with ny/2 in {16, 32, 64} rows per half: the same sums as
// mode_project / mode_back (modes_impl.cuh), laid out for occupancy.
//
// A CTA of 16 warps covers 16 x rows and 32 consecutive z (one per lane), so
// every warp load or store of the fields is a run of 32 z values.
//   projection:      A[x][n][z] = sum_{j < ny/2} Sy[j][n] (rho[x][j][z] +- rho[x][ny-1-j][z])
//                    (+ for odd n, - for even n), one thread per (x row, z) with
//                    the y-mode table as a kernel parameter (constant bank);
//                    then the CTA's rows summed against the x modes and the
//                    cluster's CTAs added up through distributed shared memory,
//                    in rank order (as mode_project).
//   back-projection: B[x][n][z] = sum_m Sx[x][m] psi[m][n][z] (psi chunk in shared
//                    memory, computed once per CTA); each thread holds a 2 x MYP
//                    tile (two x rows, all y modes) so that each y-mode value read
//                    from shared memory (16-byte broadcasts) serves two FMAs, and
//                    the two warps of an x pair split the rows: phi[x][j][z] = O + E and
//                    phi[x][ny-1-j][z] = O - E with O, E the sums of
//                    Sy[j][n] B[x][n][z] over odd and even n.
#include "modes.cuh"
#include "modes_impl.cuh"

namespace pp {

namespace {

constexpr int kW = 16;                    // warps per CTA
constexpr int kX = 16;                    // x rows per CTA
constexpr int kZC = 32;                   // z values per CTA

__device__ __forceinline__ void row4(const float* p, float (&s)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  s[0] = v.x; s[1] = v.y; s[2] = v.z; s[3] = v.w;
}

}  // namespace

// two CTAs per SM (64 registers) up to 20 y-mode slots, one beyond
template <int MYP>
constexpr int fast_min_blocks() { return MYP <= 20 ? 2 : 1; }

// the y-mode table as a kernel parameter: with the y loop unrolled, each
// value is read at a compile-time offset of the constant bank
template <int NYH, int MYP>
struct SyTab {
  float s[NYH * MYP];
};

// one thread per (x row, z): the 16 warps of a CTA take its 16 x rows
template <int NYH, int MYP>
__global__ void __launch_bounds__(32 * kW, 2)
    mode_project_fast_kernel(ModeArgs<float> a, const __grid_constant__ SyTab<NYH, MYP> tab) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* abuf = reinterpret_cast<float*>(smem_raw);            // [16][MYP][32]
  float* red = abuf + kX * MYP * kZC;                          // [mc][32]
  float* sxs = red + size_t(a.mc) * kZC;                       // [16][mxp]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int z0 = int(blockIdx.x) * kZC;
  const int xb0 = int(blockIdx.y) * kX;
  const int ny = 2 * NYH;
  for (int i = threadIdx.x; i < kX * a.mxp; i += 32 * kW) sxs[i] = a.sx[size_t(xb0) * a.mxp + i];

  const float* col = a.rho + size_t(xb0 + warp) * ny * a.nz + z0 + lane;
  float acc[MYP];
#pragma unroll
  for (int n = 0; n < MYP; ++n) acc[n] = 0.f;
#pragma unroll
  for (int j = 0; j < NYH; ++j) {
    const float u = __ldg(&col[size_t(j) * a.nz]);
    const float v = __ldg(&col[size_t(ny - 1 - j) * a.nz]);
    const float p = u + v, q = u - v;
#pragma unroll
    for (int n = 0; n < MYP; ++n) acc[n] = fmaf(tab.s[j * MYP + n], n < MYP / 2 ? p : q, acc[n]);
  }
#pragma unroll
  for (int n = 0; n < MYP; ++n) abuf[(warp * MYP + n) * kZC + lane] = acc[n];
  __syncthreads();

  // x modes over the CTA's rows: warp w takes (n, m quad) units w, w + 16, ...
  const int quads = a.mxp / 4;
#pragma unroll 1
  for (int u = warp; u < MYP * quads; u += kW) {
    const int n = u % MYP, q4 = u / MYP;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll 4
    for (int xl = 0; xl < kX; ++xl) {
      const float av = abuf[(xl * MYP + n) * kZC + lane];
      const float4 sx4 = *reinterpret_cast<const float4*>(&sxs[xl * a.mxp + 4 * q4]);
      s0 = fmaf(sx4.x, av, s0);
      s1 = fmaf(sx4.y, av, s1);
      s2 = fmaf(sx4.z, av, s2);
      s3 = fmaf(sx4.w, av, s3);
    }
    red[((4 * q4 + 0) * MYP + n) * kZC + lane] = s0;
    red[((4 * q4 + 1) * MYP + n) * kZC + lane] = s1;
    red[((4 * q4 + 2) * MYP + n) * kZC + lane] = s2;
    red[((4 * q4 + 3) * MYP + n) * kZC + lane] = s3;
  }

  // the cluster's CTAs added up in rank order, each CTA a slice of the columns
  mcg::cluster_group cl = mcg::this_cluster();
  cl.sync();
  const int ncl = int(cl.num_blocks()), rank = int(cl.block_rank());
  const int per = (a.mc + ncl - 1) / ncl;
  const int c0 = rank * per, c1 = c0 + per < a.mc ? c0 + per : a.mc;
  float* out = a.part + size_t(blockIdx.y / ncl) * a.mc * a.nz + z0 + lane;
#pragma unroll 1
  for (int c = c0 + warp; c < c1; c += kW) {
    float sum = 0.f;
#pragma unroll 1
    for (int r = 0; r < ncl; ++r) sum += cl.map_shared_rank(red, r)[c * kZC + lane];
    out[size_t(c) * a.nz] = sum;
  }
  cl.sync();
}

template <int NYH, int MYP>
__global__ void __launch_bounds__(32 * kW, fast_min_blocks<MYP>()) mode_back_fast_kernel(ModeArgs<float> a) {
  constexpr int Q = NYH / 2;
  constexpr int H = MYP / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* ps = reinterpret_cast<float*>(smem_raw);    // psi chunk [mx * MYP][32]
  float* bvs = ps + size_t(a.mx) * MYP * kZC;        // x-mode sums [16][MYP][32]
  float* sxs = bvs + kX * MYP * kZC;                 // [16][mxp]
  float* sy = sxs + kX * a.mxp;                      // [NYH][MYP]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int pair = warp % (kW / 2), half = warp / (kW / 2);
  const int z0 = int(blockIdx.x) * kZC;
  const int xb0 = int(blockIdx.y) * kX;
  const int ny = 2 * NYH;
  for (int idx = threadIdx.x; idx < a.mx * MYP * (kZC / 4); idx += 32 * kW) {
    const int c = idx / (kZC / 4), piece = idx % (kZC / 4);
    cp_async16(ps + size_t(c) * kZC + 4 * piece, a.psi + size_t(c) * a.nz + z0 + 4 * piece);
  }
  cp_async_commit();
  for (int i = threadIdx.x; i < kX * a.mxp; i += 32 * kW) sxs[i] = a.sx[size_t(xb0) * a.mxp + i];
  for (int i = threadIdx.x; i < NYH * MYP; i += 32 * kW) sy[i] = a.sy[i];
  cp_async_wait<0>();
  __syncthreads();

  // x-mode sums of the pair's two rows, this warp's half of the y modes
  {
    float b[2][H];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int n = 0; n < H; ++n) b[i][n] = 0.f;
#pragma unroll 2
    for (int m = 0; m < a.mx; ++m) {
      const float s0 = sxs[(2 * pair) * a.mxp + m], s1 = sxs[(2 * pair + 1) * a.mxp + m];
#pragma unroll
      for (int n = 0; n < H; ++n) {
        const float pv = ps[(m * MYP + half * H + n) * kZC + lane];
        b[0][n] = fmaf(s0, pv, b[0][n]);
        b[1][n] = fmaf(s1, pv, b[1][n]);
      }
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int n = 0; n < H; ++n) bvs[((2 * pair + i) * MYP + half * H + n) * kZC + lane] = b[i][n];
  }
  __syncthreads();

  float bv[2][MYP];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int n = 0; n < MYP; ++n) bv[i][n] = bvs[((2 * pair + i) * MYP + n) * kZC + lane];
  // this warp's half of the rows j (and their mirrors); 32-bit offsets from
  // the pair's first row (the field is below 2^31 values)
  float* base = a.phi + size_t(xb0 + 2 * pair) * ny * a.nz + z0 + lane;
  const int xs = ny * a.nz, step = a.nz;
  int lo = half * Q * a.nz;
  int hi = (ny - 1 - half * Q) * a.nz;
#pragma unroll 4
  for (int jj = 0; jj < Q; ++jj) {
    const float* srow = sy + (half * Q + jj) * MYP;
    float o0 = 0.f, e0 = 0.f, o1 = 0.f, e1 = 0.f;
#pragma unroll
    for (int g = 0; g < MYP; g += 4) {
      float s[4];
      row4(srow + g, s);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (g + k < H) {
          o0 = fmaf(s[k], bv[0][g + k], o0);
          o1 = fmaf(s[k], bv[1][g + k], o1);
        } else {
          e0 = fmaf(s[k], bv[0][g + k], e0);
          e1 = fmaf(s[k], bv[1][g + k], e1);
        }
      }
    }
    base[lo] = o0 + e0;
    base[hi] = o0 - e0;
    base[lo + xs] = o1 + e1;
    base[hi + xs] = o1 - e1;
    lo += step;
    hi -= step;
  }
}

namespace {

template <typename K>
cudaError_t big_smem(K kern, size_t smem) {
  if (smem > kMaxSmem) return cudaErrorInvalidConfiguration;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
}

template <int NYH, int MYP>
cudaError_t launch_fast(int which, const ModeArgs<float>& a, const float* sy_host, cudaStream_t st) {
  const int xblocks = a.nx / kX;
  const dim3 grid(unsigned(a.nz / kZC), unsigned(xblocks));
  cudaError_t e;
  if (which == 0) {
    SyTab<NYH, MYP> tab;
    for (int i = 0; i < NYH * MYP; ++i) tab.s[i] = sy_host[i];
    const size_t smem = sizeof(float) * (size_t(kX) * MYP * kZC + size_t(a.mc) * kZC + size_t(kX) * a.mxp);
    void (*kern)(ModeArgs<float>, const SyTab<NYH, MYP>) = mode_project_fast_kernel<NYH, MYP>;
    if ((e = big_smem(kern, smem)) != cudaSuccess) return e;
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
    return cudaLaunchKernelEx(&cfg, kern, a, tab);
  }
  const size_t smem = sizeof(float) * (size_t(a.mx) * MYP * kZC + size_t(kX) * MYP * kZC + size_t(kX) * a.mxp +
                                       size_t(NYH) * MYP);
  void (*kern)(ModeArgs<float>) = mode_back_fast_kernel<NYH, MYP>;
  if ((e = big_smem(kern, smem)) != cudaSuccess) return e;
  kern<<<grid, 32 * kW, smem, st>>>(a);
  return cudaGetLastError();
}

template <int NYH>
cudaError_t launch_fast2(int which, int myp, const ModeArgs<float>& a, const float* sy_host, cudaStream_t st) {
  switch (myp) {
    case 8: return launch_fast<NYH, 8>(which, a, sy_host, st);
    case 12: return launch_fast<NYH, 12>(which, a, sy_host, st);
    case 16: return launch_fast<NYH, 16>(which, a, sy_host, st);
    case 20: return launch_fast<NYH, 20>(which, a, sy_host, st);
    case 24: return launch_fast<NYH, 24>(which, a, sy_host, st);
    case 32: return launch_fast<NYH, 32>(which, a, sy_host, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool mode_fast_ok(int ny, int nx, int myp, bool fy) {
  const int nyh = ny / 2;
  return fy && (nyh == 16 || nyh == 32 || nyh == 64) && nx % kX == 0 &&
         (myp == 8 || myp == 12 || myp == 16 || myp == 20 || myp == 24 || myp == 32);
}

// stage 0 (projection) or 2 (back-projection) of an FP32 handle that
// mode_fast_ok accepts
cudaError_t launch_mode_fast(int stage, int myp, const ModeArgs<float>& a, const float* sy_host, cudaStream_t st) {
  const int which = stage == 0 ? 0 : 1;
  switch (a.ny / 2) {
    case 16: return launch_fast2<16>(which, myp, a, sy_host, st);
    case 32: return launch_fast2<32>(which, myp, a, sy_host, st);
    case 64: return launch_fast2<64>(which, myp, a, sy_host, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pp
