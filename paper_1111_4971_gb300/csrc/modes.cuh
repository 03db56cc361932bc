// Host-side declarations of the mode-space solve (modes_impl.cuh).
#pragma once

#include <cuda_runtime.h>

namespace pp {

template <typename T>
struct ModeArgs;

// tile shape of the projection and back-projection kernels
template <typename T>
struct ModeShape {
  static constexpr int WARPS = 4;
  static constexpr int THREADS = 32 * WARPS;
  static constexpr int ZC = 32;                              // z values per CTA, one per lane
  static constexpr int XPW = sizeof(T) == 4 ? 4 : 2;         // x rows per warp
  static constexpr int XB = WARPS * XPW;                     // x rows per CTA
  static constexpr int YK = 4;                               // y rows per stage (and their mirrors)
  static constexpr int STAGES = 3;
  static constexpr int MQ = sizeof(T) == 4 ? 4 : 2;          // x modes per pass of the projection
  // the projection's x modes in this many rounds, each summed over the
  // cluster before the next: the block's projection buffer holds one round
  // (FP64: half the modes, so that two CTAs fit in an SM's shared memory)
  static constexpr int RED_PASSES = sizeof(T) == 4 ? 1 : 2;
};

// x modes of one round of the projection (a multiple of MQ)
template <typename T>
__host__ __device__ inline int mode_round_modes(int mxp) {
  using S = ModeShape<T>;
  return (mxp + S::RED_PASSES * S::MQ - 1) / (S::RED_PASSES * S::MQ) * S::MQ;
}

// shared memory of the projection (elements): the ring of row stages, which
// after the y loop holds the y-mode sums [XB][myp][ZC] and one round of the
// block's projection [mode_round_modes * myp][ZC]; then the y-mode table and
// the block's x rows
template <typename T>
__host__ __device__ inline size_t mode_proj_union(int mxp, int myp, bool fy) {
  using S = ModeShape<T>;
  const size_t slab = size_t(S::STAGES) * S::XB * (fy ? 2 * S::YK : S::YK) * S::ZC;
  const size_t after = size_t(S::XB) * myp * S::ZC + size_t(mode_round_modes<T>(mxp)) * myp * S::ZC;
  return slab > after ? slab : after;
}
template <typename T>
__host__ __device__ inline size_t mode_proj_smem(int ny, int mxp, int myp, bool fy) {
  return sizeof(T) * (mode_proj_union<T>(mxp, myp, fy) + size_t(fy ? ny / 2 : ny) * myp +
                      size_t(ModeShape<T>::XB) * mxp);
}
// shared memory of the back-projection: the psi chunk [mx * myp][ZC], the
// y-mode table, the block's x rows
template <typename T>
__host__ __device__ inline size_t mode_back_smem(int ny, int mx, int mxp, int myp, bool fy) {
  return sizeof(T) * (size_t(mx) * myp * ModeShape<T>::ZC + size_t(fy ? ny / 2 : ny) * myp +
                      size_t(ModeShape<T>::XB) * mxp);
}

// y-mode slots of the tables (MYP, a multiple of 4 in {8, 12, 16, 20, 24, 32}):
// with the mirror fold, the odd modes 1, 3, .. and the even modes 2, 4, ..
// take MYP/2 slots each; without it, the modes 1..my in order
inline int mode_slots(int my, bool fold) {
  int need = fold ? 2 * ((my + 1) / 2) : my;
  need = (need + 3) / 4 * 4;
  if (need <= 8) return 8;
  if (need <= 24) return need;
  return need <= 32 ? 32 : -1;
}
// the y mode held by slot s of MYP slots
inline int mode_of_slot(int s, int myp, bool fold) {
  if (!fold) return s + 1;
  return s < myp / 2 ? 2 * s + 1 : 2 * (s - myp / 2) + 2;
}

// CTAs per cluster of the projection: the largest divisor of its x blocks
// that is at most 4; the projection writes xblocks / mode_cluster(xblocks)
// partial sums, which the z convolution adds on load.  (Clusters of 8, one
// partial at 128 x rows, kept every CTA in the distributed-shared-memory
// reduction longer than the second partial costs the z kernel.)
inline int mode_cluster(int xblocks) {
  for (int d = 4; d > 1; --d)
    if (xblocks % d == 0) return d;
  return 1;
}

// stage 0: projection rho -> part, 1: z convolution part -> psi,
// 2: back-projection psi -> phi
template <typename T>
cudaError_t launch_mode_stage(int stage, int myp, bool fy, const ModeArgs<T>& a, cudaStream_t st);

// A group of FP32 mode-form solves of one shape (nx, ny, nz, mode layout)
// and one y-mode table, run by one launch per stage (the batched call):
// args[s] (device memory) holds solve s's tables and scratch, rho / phi its
// field arrays (kernel parameters, so that a captured launch keeps them).
constexpr int kMaxModeGroup = 64;
struct ModeGroup {
  const ModeArgs<float>* args;
  const float* rho[kMaxModeGroup];
  float* phi[kMaxModeGroup];
  int n;
  int nz;
};

// the FP32 z convolution, one warp-level FFT per mode column (modes_z.cu):
// nz in 32..1024, groups partial projections summed on load
cudaError_t launch_mode_z_warp(const ModeArgs<float>& a, int groups, cudaStream_t st);
// the same for a group (columns of solve s in the CTAs s * cps ..)
cudaError_t launch_mode_z_warp_group(const ModeArgs<float>& a, int groups, const ModeGroup& g, cudaStream_t st);

// the FP32 projection and back-projection laid out for occupancy
// (modes_fast.cu): meshes symmetric in y with ny/2 in {16, 32, 64, 128}
bool mode_fast_ok(int ny, int nx, int myp, bool fy);
// sy_host: the FP32 y-mode table [ny/2][myp] in host memory (the projection's parameter)
cudaError_t launch_mode_fast(int stage, int myp, const ModeArgs<float>& a, const float* sy_host, cudaStream_t st);
cudaError_t launch_mode_fast_group(int stage, int myp, const ModeArgs<float>& a, const ModeGroup& g,
                                   const float* sy_host, cudaStream_t st);

}  // namespace pp
