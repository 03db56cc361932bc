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
// The working buffer (the handle's form decides it: the z half-spectrum,
// (nz+1)*nx*ny complex values of the dtype, for the padded-transform form;
// the x blocks' projections and the convolved mode columns for the
// mode-space form) lives in g_noalloc_scratch below, a static device array of
// kNoAllocScratchBytes that every GPU which loads the library keeps until the
// process exits.  Host code cannot use the array's name as a device address,
// so its address is looked up with cudaGetSymbolAddress, with the device
// current, whenever a handle is set up on that device (noalloc_reserve, which
// the setups call: the array is then reserved while the handle is created,
// not at the first solve) and cached per device; a call on a device where no
// lookup succeeded yet makes it first.  All calls share the one array: two
// calls whose kernels overlap on the GPU (different streams, or different
// handles on the same device at once) overwrite each other's data.  Nothing
// in the array has to start at zero: a solve writes every element it reads.
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

int lookup(int dev, bool refresh, void** out) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (dev < 0 || dev >= kMaxDevices) return PIPE_EUNSUPPORTED;
  if (refresh || !g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      g_noalloc_ptr[dev] = nullptr;
      return PIPE_ECUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  if (out) *out = g_noalloc_ptr[dev];
  return PIPE_OK;
}

}  // namespace

namespace pp {
int noalloc_reserve(int dev) { return lookup(dev, true, nullptr); }
}  // namespace pp

extern "C" int pipe_poisson_solve_noalloc(pipe_handle* h, const void* rho, void* phi, void* stream) {
  if (!h || !rho || !phi) return PIPE_EINVAL;
  if ((reinterpret_cast<uintptr_t>(rho) | reinterpret_cast<uintptr_t>(phi)) % 16) return PIPE_EINVAL;
  if (h->banded >= 0 || h->grid.dtype == PIPE_F32_C16) return PIPE_EUNSUPPORTED;
  if (!h->use_modes && (h->general || !h->fft_ok)) return PIPE_EUNSUPPORTED;
  const size_t cbytes = h->grid.dtype == PIPE_F64 ? 16 : 8;
  const size_t need = h->use_modes ? pp::mode_scratch_bytes(h)
                                   : size_t(h->grid.nz + 1) * h->grid.nx * h->grid.ny * cbytes;
  if (need > kNoAllocScratchBytes) return PIPE_EUNSUPPORTED;     // larger than the fixed array
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return PIPE_ECUDA;
  if (prev != h->device && cudaSetDevice(h->device) != cudaSuccess) return PIPE_ECUDA;
  void* work = nullptr;
  int st = lookup(h->device, false, &work);
  if (st == PIPE_OK) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (h->use_modes) {
      st = pp::mode_solve(h, rho, phi, work, s);
    } else if (h->grid.dtype == PIPE_F64) {
      st = pp::transform_chain<double>(h, pp::make_args<double>(h, rho, phi, work), false, s);
    } else {
      st = pp::transform_chain<float>(h, pp::make_args<float>(h, rho, phi, work), false, s);
    }
  }
  if (prev != h->device) cudaSetDevice(prev);
  return st;
}
