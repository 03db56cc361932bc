// Internal layout of pipe_handle (opaque in the C ABI).
#pragma once

#include <cuda_runtime.h>

#include "../../include/pipe_poisson.h"

namespace pp {
// Kernel variant choices for one handle (filled by default_plan, refined by
// pipe_autotune).
struct Plan {
  int z_warps;     // warps per CTA of the z transforms (8 or 16)
  int z_pipe;      // 1: pipelined multi-tile z kernels, 0: one tile per CTA
  int t_h;         // transverse stage: row blocks per kz plane (CTAs per cluster)
  int t_threads;   // threads per transverse CTA
  int t_kind = 0;  // 0: 2N-point transverse routines (any mesh), 1: N-point routine
                   //    (cell-centred meshes, s = 2 x0 / h = 1 on both axes)
};
}  // namespace pp

struct pipe_handle {
  int device = 0;
  pipe_geometry geom{};
  pipe_grid grid{};
  int kind = 0;          // 0 ordinary, 1 IGF, 2 free space
  int banded = -1;       // >= 0: the banded reduction with this many neighbour planes
  int general = 0;       // 1: window mesh, the four full transformed tables of Eq. 10
  int sx = 0, sy = 0;    // correlation shifts 2*x0/hx, 2*y0/hy
  int images = 1;        // four-term pipe operator (1) or free space (0)
  double* green64 = nullptr;
  float* green32 = nullptr;
  void* work = nullptr;  // (nz+1)*nx*ny complex of the dtype
  float2* tab32 = nullptr;
  double2* tab64 = nullptr;
  float2 *tw_t32 = nullptr, *w2_t32 = nullptr, *tw_z32 = nullptr, *w2_z32 = nullptr, *tw_t2_32 = nullptr,
         *tw_t2c_32 = nullptr;
  double2 *tw_t64 = nullptr, *w2_t64 = nullptr, *tw_z64 = nullptr, *w2_z64 = nullptr, *tw_t2_64 = nullptr,
          *tw_t2c_64 = nullptr;
  void* tbuf = nullptr;        // n-point scratch planes (FP64 at 128 x 128), see SolveArgs::tbuf
  int* err = nullptr;          // device error word (in the tab32 allocation), see pipe_status
  int inject_drop = 0;         // pipe_inject_stage_fault: consumed by the next solve
  long long inject_polls = 0;
  void* stage_rho = nullptr;   // device staging for pipe_poisson_solve_host
  void* stage_phi = nullptr;
  // pipe_poisson_solve_host_stream: two device staging buffers per direction,
  // the two copy streams and the events that order them (created on first use)
  void* ring_rho[2] = {nullptr, nullptr};
  void* ring_phi[2] = {nullptr, nullptr};
  cudaStream_t copy_in = nullptr;
  cudaStream_t copy_out = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr};
  cudaEvent_t ev_done[2] = {nullptr, nullptr};
  cudaEvent_t ev_out[2] = {nullptr, nullptr};
  // mode-space solve (modes_impl.cuh): its tables, FP64 and FP32, and its
  // scratch (the x blocks' projections, then the z-convolved mode columns)
  int modes_ok = 0;            // the mode path can run this handle
  int use_modes = 0;           // solves take the mode path (plan t_kind 3)
  int fft_ok = 1;              // the padded-transform path's buffers exist
  int mxp = 0, myp = 0, fy = 0;
  double *msx64 = nullptr, *msy64 = nullptr, *mgz64 = nullptr;
  float *msx32 = nullptr, *msy32 = nullptr, *mgz32 = nullptr;
  double* mkb64 = nullptr;     // banded operator in mode space: [mxp*myp][nb+1] real-space z kernel
  float* mkb32 = nullptr;
  void* mwork = nullptr;       // part [xblocks][mc][nz], then psi [mc][nz], of the dtype
  float* msy_host = nullptr;   // FP32 y-mode table in host memory (the projection's kernel parameter)
  int mfast = 0;               // FP32 projection / back-projection in their occupancy layout
  pp::Plan plan{8, 0, 1, 256};
  pp::Plan free_plan{8, 0, 1, 256};   // transverse shape of the free-space stage
  void* batch = nullptr;       // batched work list owned by this handle
};

namespace pp {
template <typename T>
struct SolveArgs;
// launch arguments of the padded-transform form with `work` as its working buffer
template <typename T>
SolveArgs<T> make_args(pipe_handle* h, const void* rho, void* phi, void* work);
// that form's three stages (z forward, transverse stage, z inverse) on a's buffers
template <typename T>
int transform_chain(pipe_handle* h, const SolveArgs<T>& a, bool adjoint, cudaStream_t st);
// looks up (again) the device address of the no-alloc solve's fixed array on
// the current device `dev`; the setups call it so that the array is reserved
// when a handle is created
int noalloc_reserve(int dev);
Plan default_plan(int n, int nz, bool f64, bool cell_centred);   // pipe operator
Plan default_free_plan(int n, int nz, bool f64);   // free-space stage
void batch_release(pipe_handle* h);
int handle_solve(pipe_handle* h, const void* rho, void* phi, bool adjoint, cudaStream_t st);
// the mode-space solve with `scratch` (mode_scratch_bytes) as its working buffer
int mode_solve(pipe_handle* h, const void* rho, void* phi, void* scratch, cudaStream_t st);
size_t mode_scratch_bytes(const pipe_handle* h);
// x blocks of the projection (nx / rows per CTA of the dtype)
int mode_xblocks(const pipe_handle* h);
// the FP32 mode-form arguments of a handle with its own scratch as part /
// psi (rho, phi null): the batched call's grouped launches
template <typename T> struct ModeArgs;
ModeArgs<float> mode_args_f32(const pipe_handle* h);
}  // namespace pp
