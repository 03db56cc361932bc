// Batched solves and the autotuner (filled in below the single-solve path).
#include <cuda_runtime.h>

#include "../../include/pipe_poisson.h"
#include "handle.cuh"

namespace pp {
void batch_release(pipe_handle*) {}
}  // namespace pp

extern "C" int pipe_poisson_solve_batched(pipe_handle* const*, const void* const*, void* const*, int,
                                          void*) {
  return PIPE_EUNSUPPORTED;
}
extern "C" int pipe_batch_status(pipe_handle* const*, int) { return PIPE_OK; }
