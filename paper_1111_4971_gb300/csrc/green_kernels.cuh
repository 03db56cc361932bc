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

// The four transformed tables of Eq. 10 for a general (window) mesh with
// origin (x0, y0): FP64 and FP32 copies of [4][nz+1][2ny][2nx] complex values
// (cc, cr, rc, rr), scaled by s.scale.  Synchronous on `st`.
cudaError_t build_general_spectra(const GreenSpec& s, double x0, double y0, double2* t64, float2* t32,
                                  cudaStream_t st);

// Same for the free-space 1/r table (Hockney).
cudaError_t build_free_spectrum(const GreenSpec& s, double self_value, double* g64, float* g32,
                                cudaStream_t st);

// Tables of the mode-space solve: FP64 and FP32 copies of sx [nx][mxp],
// sy [fold ? ny/2 : ny][myp] and gz [mxp*myp][nz+1] (see green.cu).
// Synchronous on `st`.  Uses temporary device memory (freed before return).
// The banded operator's real-space z kernel in the mode slots, kb [mxp*myp][nb+1]
// (FP64 and FP32).  Synchronous on `st`.  Uses temporary device memory.
cudaError_t build_mode_band(const GreenSpec& s, int mxp, int myp, int fold, int nb, double* kb64, float* kb32,
                            cudaStream_t st);

cudaError_t build_mode_tables(const GreenSpec& s, double x0, double y0, int mxp, int myp, int fold,
                              double* sx64, float* sx32, double* sy64, float* sy32, double* gz64,
                              float* gz32, cudaStream_t st);

}  // namespace pp
