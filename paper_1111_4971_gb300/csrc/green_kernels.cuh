// Host-side entry points of the FP64 setup kernels (green.cu).
#pragma once

#include <cuda_runtime.h>

namespace pp {

struct GreenSpec {
  int nx, ny, nz;
  double hx, hy, hz;
  double a, b;
  int modes_m, modes_n;
  int igf;
  double scale;     // hx*hy*hz / (8 nx ny nz); hx*hy*hz / (4 nx ny) for 2-D spectra
};

// twiddle tables of one axis (see tables_kernel)
template <typename V>
void launch_tables(V* tw, V* w2, int L, int G, int n2, cudaStream_t st);

// FP64 octant spectrum of the pipe Green function R / R_int, scaled; FP32 copy.
// Synchronous on `st`.  Uses temporary device memory (freed before return).
// transform_z = false stops after the x and y transforms: planes r = 0..nz of
// 2-D spectra of the tables at z-offsets r*hz (the banded reduction).
cudaError_t build_pipe_spectrum(const GreenSpec& s, double* g64, float* g32, cudaStream_t st,
                                bool transform_z = true);

// Same for the free-space 1/r table (Hockney).
cudaError_t build_free_spectrum(const GreenSpec& s, double self_value, double* g64, float* g32,
                                cudaStream_t st);

}  // namespace pp
