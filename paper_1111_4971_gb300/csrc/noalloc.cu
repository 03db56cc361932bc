// pipe_poisson_solve_noalloc: the forward solve with its working buffer taken
// from a fixed device array that is part of this library, so the call itself
// never allocates device memory.
//
// Who needs it: programs that must not let a library allocate device memory
// once they are running -- a host application that reserves the GPU's memory
// for its own pool before loading plugins (a cudaMalloc from a plugin then
// fails or fragments that pool), or a time-critical loop that cannot afford
// an allocation stalling or failing in the middle of a run.  They set up a
// handle once during initialisation and then call this entry point.
//
// The working buffer (the z half-spectrum, (nz+1)*nx*ny complex values of the
// handle's dtype) lives in g_noalloc_scratch below, a static device array of
// kNoAllocScratchBytes that every GPU which loads the library keeps until the
// process exits.  Host code cannot use the array's name as a device address,
// so the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and caches it.  All calls
// share the one array: two calls whose kernels overlap on the GPU (different
// streams, or different handles on the same device at once) overwrite each
// other's data.  Nothing in the array has to start at zero: a solve writes
// every element it reads.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/pipe_poisson.h"
#include "handle.cuh"
#include "solver.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;     // 64 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// device address of the array on the current device `dev` (looked up once)
int noalloc_scratch(int dev, void** out) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (dev < 0 || dev >= kMaxDevices) return PIPE_EUNSUPPORTED;
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return PIPE_ECUDA;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return PIPE_OK;
}

template <typename T>
pp::SolveArgs<T> noalloc_args(pipe_handle* h, const void* rho, void* phi, void* work);
template <>
pp::SolveArgs<float> noalloc_args<float>(pipe_handle* h, const void* rho, void* phi, void* work) {
  pp::SolveArgs<float> a{};
  a.rho = static_cast<const float*>(rho); a.phi = static_cast<float*>(phi);
  a.work = static_cast<float2*>(work); a.green = h->green32;
  a.tw_t = h->tw_t32; a.w2_t = h->w2_t32; a.tw_z = h->tw_z32; a.w2_z = h->w2_z32; a.tw_t2 = h->tw_t2_32;
  a.tw_t2c = h->tw_t2c_32;
  a.nx = h->grid.nx; a.ny = h->grid.ny; a.nz = h->grid.nz;
  a.sx = h->sx; a.sy = h->sy; a.images = h->images;
  a.err = h->err;                      // the handle's error word (set up with it)
  return a;
}
template <>
pp::SolveArgs<double> noalloc_args<double>(pipe_handle* h, const void* rho, void* phi, void* work) {
  pp::SolveArgs<double> a{};
  a.rho = static_cast<const double*>(rho); a.phi = static_cast<double*>(phi);
  a.work = static_cast<double2*>(work); a.green = h->green64;
  a.tw_t = h->tw_t64; a.w2_t = h->w2_t64; a.tw_z = h->tw_z64; a.w2_z = h->w2_z64; a.tw_t2 = h->tw_t2_64;
  a.tw_t2c = h->tw_t2c_64;
  a.tbuf = static_cast<double2*>(h->tbuf);
  a.nx = h->grid.nx; a.ny = h->grid.ny; a.nz = h->grid.nz;
  a.sx = h->sx; a.sy = h->sy; a.images = h->images;
  a.err = h->err;                      // the handle's error word (set up with it)
  return a;
}

// the same three stages as pipe_poisson_solve, with `work` as the buffer
template <typename T>
int noalloc_run(pipe_handle* h, const void* rho, void* phi, void* work, cudaStream_t st) {
  const pp::SolveArgs<T> a = noalloc_args<T>(h, rho, phi, work);
  const pp::Plan& p = h->plan;
  cudaError_t e = pp::launch_z<T>(true, p.z_warps, p.z_pipe, false, a, st);
  if (e == cudaSuccess)
    e = h->images ? pp::launch_transverse_sym<T>(false, p.t_kind, p.t_h, p.t_threads, a, st)
                  : pp::launch_transverse<T>(false, h->free_plan.t_h, h->free_plan.t_threads, a, st);
  if (e == cudaSuccess) e = pp::launch_z<T>(false, p.z_warps, p.z_pipe, false, a, st);
  return e == cudaSuccess ? PIPE_OK : PIPE_ECUDA;
}

}  // namespace

extern "C" int pipe_poisson_solve_noalloc(pipe_handle* h, const void* rho, void* phi, void* stream) {
  if (!h || !rho || !phi) return PIPE_EINVAL;
  if ((reinterpret_cast<uintptr_t>(rho) | reinterpret_cast<uintptr_t>(phi)) % 16) return PIPE_EINVAL;
  if (h->banded >= 0 || h->general || h->grid.dtype == PIPE_F32_C16) return PIPE_EUNSUPPORTED;
  const size_t cbytes = h->grid.dtype == PIPE_F64 ? 16 : 8;
  const size_t need = size_t(h->grid.nz + 1) * h->grid.nx * h->grid.ny * cbytes;
  if (need > kNoAllocScratchBytes) return PIPE_EUNSUPPORTED;     // larger than the fixed array
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return PIPE_ECUDA;
  if (prev != h->device && cudaSetDevice(h->device) != cudaSuccess) return PIPE_ECUDA;
  void* work = nullptr;
  int st = noalloc_scratch(h->device, &work);
  if (st == PIPE_OK) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = h->grid.dtype == PIPE_F64 ? noalloc_run<double>(h, rho, phi, work, s)
                                   : noalloc_run<float>(h, rho, phi, work, s);
  }
  if (prev != h->device) cudaSetDevice(prev);
  return st;
}
