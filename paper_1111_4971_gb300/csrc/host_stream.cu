// pipe_poisson_solve_host_stream: a sequence of solves from host memory with
// the transfers overlapped.  Solve k runs on the caller's stream while the
// input of solve k+1 is copied in on one copy stream and the result of solve
// k-1 is copied out on another, through two device staging buffers per
// direction.  Events order the three streams: an input buffer is refilled
// only after the solve that read it, an output buffer is overwritten only
// after its copy to the host.  The workspace of the handle is used by one
// solve at a time (all solves are on the caller's stream).
#include <cuda_runtime.h>

#include "../../include/pipe_poisson.h"
#include "handle.cuh"

namespace {

int ensure_ring(pipe_handle* h, size_t bytes) {
  if (h->ring_rho[0]) return PIPE_OK;
  for (int k = 0; k < 2; ++k) {
    if (cudaMalloc(&h->ring_rho[k], bytes) != cudaSuccess) return PIPE_ENOMEM;
    if (cudaMalloc(&h->ring_phi[k], bytes) != cudaSuccess) return PIPE_ENOMEM;
    if (cudaEventCreateWithFlags(&h->ev_in[k], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_done[k], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_out[k], cudaEventDisableTiming) != cudaSuccess)
      return PIPE_ECUDA;
  }
  if (cudaStreamCreateWithFlags(&h->copy_in, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->copy_out, cudaStreamNonBlocking) != cudaSuccess)
    return PIPE_ECUDA;
  return PIPE_OK;
}

}  // namespace

extern "C" int pipe_poisson_solve_host_stream(pipe_handle* h, const void* const* rho_host, void* const* phi_host,
                                              int count, void* stream) {
  if (!h || !rho_host || !phi_host || count < 1) return PIPE_EINVAL;
  for (int k = 0; k < count; ++k)
    if (!rho_host[k] || !phi_host[k]) return PIPE_EINVAL;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return PIPE_ECUDA;
  if (prev != h->device && cudaSetDevice(h->device) != cudaSuccess) return PIPE_ECUDA;
  const size_t bytes = size_t(h->grid.nx) * h->grid.ny * h->grid.nz * (h->grid.dtype == PIPE_F64 ? 8 : 4);
  int st = ensure_ring(h, bytes);
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  bool ok = (st == PIPE_OK);
  for (int k = 0; ok && k < count; ++k) {
    const int s = k & 1;
    // input slot s was read by solve k-2; output slot s was copied back for k-2
    if (k >= 2) ok = cudaStreamWaitEvent(h->copy_in, h->ev_done[s], 0) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(h->ring_rho[s], rho_host[k], bytes, cudaMemcpyHostToDevice, h->copy_in) == cudaSuccess;
    ok = ok && cudaEventRecord(h->ev_in[s], h->copy_in) == cudaSuccess;
    ok = ok && cudaStreamWaitEvent(cs, h->ev_in[s], 0) == cudaSuccess;
    if (ok && k >= 2) ok = cudaStreamWaitEvent(cs, h->ev_out[s], 0) == cudaSuccess;
    if (ok) {
      st = pp::handle_solve(h, h->ring_rho[s], h->ring_phi[s], false, cs);
      ok = (st == PIPE_OK);
    }
    ok = ok && cudaEventRecord(h->ev_done[s], cs) == cudaSuccess;
    ok = ok && cudaStreamWaitEvent(h->copy_out, h->ev_done[s], 0) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(phi_host[k], h->ring_phi[s], bytes, cudaMemcpyDeviceToHost, h->copy_out) == cudaSuccess;
    ok = ok && cudaEventRecord(h->ev_out[s], h->copy_out) == cudaSuccess;
  }
  if (ok) ok = cudaStreamSynchronize(h->copy_out) == cudaSuccess && cudaStreamSynchronize(cs) == cudaSuccess;
  if (st == PIPE_OK && !ok) st = PIPE_ECUDA;
  if (prev != h->device) cudaSetDevice(prev);
  return st;
}
