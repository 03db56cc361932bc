// Shared declarations of the solve kernels (z transforms, transverse stage).
#pragma once

#include "fft_common.cuh"

namespace pp {

// Per-solve launch parameters (all device pointers).
//   rho/phi : [nx][ny][nz] real, z contiguous
//   work    : [nz+1][nx][ny] complex  (z half-spectrum, kz-plane major)
//   green   : [nz+1][ny+1][nx+1] real octant of the scaled Green spectrum
//   tw_t / w2_t : transverse group-FFT twiddles (length n) and w_{2n}^j, j<2n
//   tw_z / w2_z : z group-FFT twiddles (length nz/2) and w_{2nz}^j, j<2nz
template <typename T>
struct SolveArgs {
  const T* rho;
  T* phi;
  C2<T>* work;
  const T* green;
  const C2<T>* tw_t;
  const C2<T>* w2_t;
  const C2<T>* tw_t2;   // paired-layout twiddles of the 2n-point transverse FFTs
  const C2<T>* tw_t2c;  // cyclic-layout twiddles of the 2n-point transverse FFTs
  const C2<T>* tw_z;
  const C2<T>* w2_z;
  int nx, ny, nz;
  int sx, sy;        // correlation shifts 2*x0/hx, 2*y0/hy (integers)
  int images;        // 1: four-term pipe operator, 0: free-space (one term)
  // complex-FP16 spectra (PIPE_F32_C16 handles only): `work` then holds
  // __half2 values with per-slab FP32 scales, zscale[tile] for the z-forward
  // tiles of zcols columns and tscale[kz * nx + i] for the transverse rows
  float* zscale;
  float* tscale;
  int zcols;
  // global scratch planes [nz+1][nx][ny] for the n-point routine when a plane
  // does not fit in shared memory (FP64 at 128 x 128); null otherwise
  C2<T>* tbuf;
  // device error word of the handle (PIPE_ETIMEOUT when a bounded wait of the
  // staged transverse kernel gave up); null: not recorded
  int* err;
  // failure-detection tests of the staged transverse kernel: its first CTA
  // leaves out bulk copy number stage_drop - 1 (0: none) and every wait polls
  // at most stage_polls times (0: the default limit)
  int stage_drop;
  long long stage_polls;
};

// z transforms: one CTA handles COLS consecutive (i,j) columns.
template <typename T, int NZ, int WARPS>
struct ZCfg {
  static constexpr int L = NZ / 2;                 // sub-FFT length
  using S = GroupShape<L>;
  static constexpr int G = S::G;
  static constexpr int E = S::E;
  static constexpr int UNIT = 2 * G;               // lanes per column (even + odd half)
  static_assert(UNIT <= 32, "column unit must fit a warp");
  static constexpr int CPW = 32 / UNIT;            // columns per warp
  static constexpr int COLS = WARPS * CPW;         // columns per CTA
  static constexpr int THREADS = 32 * WARPS;
  static constexpr int GROUPS = THREADS / G;
  // staging tile, column major [COLS][LDS]: a lane's column is contiguous; the
  // stride (in complex values) makes the row-wise accesses (fixed kz,
  // consecutive columns: the 16-byte store reads of the forward kernel and the
  // asynchronous copies of the inverse) conflict-free: 2 (mod 16) for 8-byte
  // values served per half-warp, odd for 16-byte values served per quarter-warp
  static constexpr int LDS = NZ + (sizeof(T) == 4 ? 2 : 1);
  // single-tile routines: the FFT scratch tiles and the staging tile are live
  // at different times and share the allocation
  static constexpr size_t SCR = size_t(GROUPS) * S::SSTRIDE;
  static constexpr size_t STG = size_t(COLS) * LDS;
  static constexpr size_t smem_bytes() { return sizeof(C2<T>) * (SCR > STG ? SCR : STG); }
  // pipelined multi-tile routines: the next tile streams into its own buffer
  // while the current one is transformed
  static constexpr size_t INW = size_t(COLS) * (NZ / 2);     // packed real input of a tile
  static constexpr size_t fwd_pipe_smem() { return sizeof(C2<T>) * (2 * INW + SCR + STG); }
  static constexpr size_t inv_pipe_smem() { return sizeof(C2<T>) * (2 * STG + SCR); }
};

template <typename T, int NZ, int WARPS, bool CONJ, bool H16 = false>
__global__ void zfwd_kernel(SolveArgs<T> a);
template <typename T, int NZ, int WARPS, bool CONJ, bool H16 = false>
__global__ void zinv_kernel(SolveArgs<T> a);

// transverse stage: one cluster of 2*H CTAs per kz plane, THREADS per CTA.
template <typename T, int N, int H_, int THREADS_>
struct TCfg {
  using S = GroupShape<N>;
  static constexpr int G = S::G;
  static constexpr int E = S::E;
  static constexpr int H = H_;                   // row blocks
  static constexpr int ROWS = N / H;
  static constexpr int LD = ROWS + 1;            // padded column stride of the y-spectrum tile
  static constexpr int THREADS = THREADS_;
  static constexpr int GROUPS = THREADS / G;
  static constexpr int CLUSTER = 2 * H;
  static constexpr size_t smem_bytes() {
    return sizeof(C2<T>) * (size_t(N) * LD + size_t(GROUPS) * S::SSTRIDE);
  }
};
constexpr size_t kMaxSmem = 227 * 1024;

// transverse stage of the pipe operator (full-span meshes): one cluster of HB
// CTAs per kz plane; CTA h holds rows [h*N/HB, (h+1)*N/HB) of u[ky = 1..N][i].
// The tile is unpadded with the row index XOR-swizzled by the column
// (conflict-free row and column accesses).
template <typename T, int N, int HB, int THREADS>
struct TSymCfg {
  static constexpr int L = 2 * N;
  using S = PairShape<L>;
  static constexpr int G = S::G;
  static constexpr int E = S::E;
  static constexpr int ROWS = N / HB;
  static constexpr int LD = ROWS;
  static constexpr int SWM = (ROWS < 16 ? ROWS : 16) - 1;
  static constexpr int YBUF = N * LD;
  static constexpr int GROUPS = THREADS / G;
  static constexpr size_t smem_bytes() {
    return sizeof(C2<T>) * (size_t(YBUF) + 3 * size_t(L) + size_t(GROUPS) * S::SSTRIDE);
  }
};

template <typename T, int N, int H, int THREADS, bool ADJ>
__global__ void transverse_kernel(SolveArgs<T> a);

// host launchers (defined next to the kernels)
template <typename T>
cudaError_t launch_z(bool forward, int warps, int pipe, bool conj, const SolveArgs<T>& a, cudaStream_t st);
template <typename T>
cudaError_t launch_transverse(bool adjoint, int h, int threads, const SolveArgs<T>& a, cudaStream_t st);
// complex-FP16 spectra with FP32 arithmetic (single-tile z kernels, n-point
// transverse routine); z_tile_cols gives the z-forward tile width (the slab
// of its scales) for nz and the CTA size in warps
cudaError_t launch_z_c16(bool forward, int warps, bool conj, const SolveArgs<float>& a, cudaStream_t st);
cudaError_t launch_transverse_c16(bool adjoint, int threads, const SolveArgs<float>& a, cudaStream_t st);
int z_tile_cols(int nz, int warps);
// transverse stage for general (window) meshes: the four full tables of Eq. 10
template <typename T>
cudaError_t launch_transverse_gen(bool adjoint, int threads, const SolveArgs<T>& a, cudaStream_t st);
// banded z reduction (Eq. 17-18): two kernels on `work` as [nz/2][ny][nx]
template <typename T>
cudaError_t launch_banded(int threads, const SolveArgs<T>& a, int n_nb, cudaStream_t st);
template <typename T>
cudaError_t launch_transverse_sym(bool adjoint, int kind, int hb, int threads, const SolveArgs<T>& a,
                                  cudaStream_t st);

}  // namespace pp
