// Kernel-variant plans and the autotuner.
//
// A plan picks, for one (n, nz, dtype) shape, the CTA size of the z
// transforms and the cluster shape / CTA size of the transverse stage.  The
// autotuner times every variant that fits the device with CUDA events on the
// caller's stream and keeps the fastest; results are cached per shape for the
// process and, if PIPE_TUNE_CACHE names a file, persisted there as lines
// "n nz dtype z_warps z_pipe t_h t_threads t_kind".
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

#include "../../include/pipe_poisson.h"
#include "handle.cuh"
#include "solver.cuh"

namespace pp {

Plan default_plan(int n, int nz, bool f64, bool cell_centred) {
  Plan p;
  // timed on GB300: FP32 z transforms in 4-warp CTAs where a column fills
  // a warp (nz >= 512), else 8; FP32 one CTA per plane, on cell-centred
  // meshes with the n-point routine (256 threads; 512 at n = 64; at n = 128
  // its staged persistent form), else the cyclic 2n-point routine (512
  // threads); FP64 2-CTA clusters of 128 threads at n = 128
  p.z_warps = (!f64 && nz >= 512) ? 4 : 8;
  p.z_pipe = 0;
  p.t_kind = 0;
  if (!f64) {
    p.t_h = 1;
    if (cell_centred) { p.t_kind = n == 128 ? 2 : 1; p.t_threads = n == 64 ? 512 : 256; }
    else p.t_threads = 512;
  } else if (n < 128) {
    p.t_h = 1;
    p.t_threads = 256;
    if (cell_centred) p.t_kind = 1;
  } else {
    p.t_h = 2;
    p.t_threads = 128;
    // FP64 128^2 on cell-centred meshes: the n-point routine with its plane
    // buffers in global memory (the handle allocates them)
    if (cell_centred) { p.t_kind = 1; p.t_h = 1; p.t_threads = 256; }
  }
  return p;
}

Plan default_free_plan(int n, int nz, bool f64) {
  Plan p;
  p.z_warps = 8;
  p.z_pipe = 0;
  const size_t c = f64 ? 16 : 8;
  p.t_h = (n >= 128 || c * n * (n + 1) > 150 * 1024) ? 2 : 1;
  p.t_threads = 256;
  return p;
}

namespace {
using Key = std::tuple<int, int, int>;
std::mutex g_mu;
std::map<Key, Plan>& cache() {
  static std::map<Key, Plan> m;
  return m;
}

void load_file_cache() {
  static bool loaded = false;
  if (loaded) return;
  loaded = true;
  const char* path = std::getenv("PIPE_TUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  int n, nz, dt, zw, th, tt, tk;
  int zp;
  while (std::fscanf(f, "%d %d %d %d %d %d %d %d", &n, &nz, &dt, &zw, &zp, &th, &tt, &tk) == 8)
    cache()[Key(n, nz, dt)] = Plan{zw, zp, th, tt, tk};
  std::fclose(f);
}

void save_file_cache(const Key& k, const Plan& p) {
  const char* path = std::getenv("PIPE_TUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%d %d %d %d %d %d %d %d\n", std::get<0>(k), std::get<1>(k), std::get<2>(k), p.z_warps,
               p.z_pipe, p.t_h, p.t_threads, p.t_kind);
  std::fclose(f);
}

template <typename T>
SolveArgs<T> args_for(pipe_handle* h, void* rho, void* phi);
template <>
SolveArgs<float> args_for<float>(pipe_handle* h, void* rho, void* phi) {
  SolveArgs<float> a{};
  a.rho = static_cast<const float*>(rho); a.phi = static_cast<float*>(phi);
  a.work = static_cast<float2*>(h->work); a.green = h->green32;
  a.tw_t = h->tw_t32; a.w2_t = h->w2_t32; a.tw_z = h->tw_z32; a.w2_z = h->w2_z32;
  a.tw_t2 = h->tw_t2_32;
  a.tw_t2c = h->tw_t2c_32;
  a.nx = h->grid.nx; a.ny = h->grid.ny; a.nz = h->grid.nz;
  a.sx = h->sx; a.sy = h->sy; a.images = h->images;
  return a;
}
template <>
SolveArgs<double> args_for<double>(pipe_handle* h, void* rho, void* phi) {
  SolveArgs<double> a{};
  a.rho = static_cast<const double*>(rho); a.phi = static_cast<double*>(phi);
  a.work = static_cast<double2*>(h->work); a.green = h->green64;
  a.tw_t = h->tw_t64; a.w2_t = h->w2_t64; a.tw_z = h->tw_z64; a.w2_z = h->w2_z64;
  a.tw_t2 = h->tw_t2_64;
  a.tw_t2c = h->tw_t2c_64;
  a.tbuf = static_cast<double2*>(h->tbuf);
  a.nx = h->grid.nx; a.ny = h->grid.ny; a.nz = h->grid.nz;
  a.sx = h->sx; a.sy = h->sy; a.images = h->images;
  return a;
}

// mean time (ms) of `reps` runs of f on st, after 2 warm-ups; < 0 if f fails
template <typename F>
float time_ms(F&& f, cudaStream_t st, int reps) {
  for (int i = 0; i < 2; ++i)
    if (f() != cudaSuccess) { cudaGetLastError(); return -1.f; }
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a, st);
  for (int i = 0; i < reps; ++i) f();
  cudaEventRecord(b, st);
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms / reps;
}

template <typename T>
int tune(pipe_handle* h, cudaStream_t st, Plan* out) {
  const size_t n = size_t(h->grid.nx) * h->grid.ny * h->grid.nz;
  void *rho = nullptr, *phi = nullptr;
  if (cudaMalloc(&rho, n * sizeof(T)) != cudaSuccess) return PIPE_ENOMEM;
  if (cudaMalloc(&phi, n * sizeof(T)) != cudaSuccess) { cudaFree(rho); return PIPE_ENOMEM; }
  cudaMemsetAsync(rho, 0, n * sizeof(T), st);
  SolveArgs<T> a = args_for<T>(h, rho, phi);
  Plan best = h->images ? h->plan : h->free_plan;
  float bz = 1e30f, bt = 1e30f;
  const int reps = 5;
  if (h->banded >= 0) {                 // the banded form: only its CTA size
    for (int th : {128, 256, 512}) {
      float ms = time_ms([&] { return launch_banded<T>(th, a, h->banded, st); }, st, reps);
      if (ms > 0 && ms < bt) { bt = ms; best.t_threads = th; }
    }
    cudaStreamSynchronize(st);
    cudaFree(rho);
    cudaFree(phi);
    if (bt > 1e29f) return PIPE_ECUDA;
    *out = best;
    return PIPE_OK;
  }
  for (int zw : {4, 8, 16})
    for (int zp : {0, 1}) {
      float ms = time_ms([&] {
        cudaError_t e = launch_z<T>(true, zw, zp, false, a, st);
        if (e != cudaSuccess) return e;
        return launch_z<T>(false, zw, zp, false, a, st);
      }, st, reps);
      if (ms > 0 && ms < bz) { bz = ms; best.z_warps = zw; best.z_pipe = zp; }
    }
  if (h->general) {                     // window meshes: the general routine's CTA size
    for (int th : {128, 256, 512}) {
      float ms = time_ms([&] { return launch_transverse_gen<T>(false, th, a, st); }, st, reps);
      if (ms > 0 && ms < bt) { bt = ms; best.t_threads = th; }
    }
  } else if (h->images) {
    // {kind, CTAs per plane, threads}; kinds 1 and 2 only for cell-centred meshes
    const int shapes[13][3] = {{0, 1, 128}, {0, 1, 256}, {0, 1, 512}, {0, 2, 128}, {0, 2, 256},
                               {0, 4, 128}, {0, 4, 256}, {1, 1, 128}, {1, 1, 256}, {1, 1, 512},
                               {2, 1, 128}, {2, 1, 256}, {2, 1, 512}};
    for (auto& sh : shapes) {
      if (sh[0] >= 1 && !(h->sx == 1 && h->sy == 1)) continue;
      float ms = time_ms([&] { return launch_transverse_sym<T>(false, sh[0], sh[1], sh[2], a, st); }, st,
                         reps);
      if (ms > 0 && ms < bt) { bt = ms; best.t_kind = sh[0]; best.t_h = sh[1]; best.t_threads = sh[2]; }
    }
  } else {
    const int shapes[4][2] = {{1, 256}, {1, 512}, {2, 256}, {2, 512}};
    for (auto& sh : shapes) {
      float ms = time_ms([&] { return launch_transverse<T>(false, sh[0], sh[1], a, st); }, st, reps);
      if (ms > 0 && ms < bt) { bt = ms; best.t_h = sh[0]; best.t_threads = sh[1]; }
    }
  }
  cudaStreamSynchronize(st);
  cudaFree(rho);
  cudaFree(phi);
  if (bz > 1e29f || bt > 1e29f) return PIPE_ECUDA;
  *out = best;
  return PIPE_OK;
}
}  // namespace

}  // namespace pp

using namespace pp;

namespace pp {
namespace {
// where both forms can run the handle: time a few full solves of each (the
// transform form with its tuned plan) and keep the faster
int choose_form(pipe_handle* h, cudaStream_t st) {
  const size_t n = size_t(h->grid.nx) * h->grid.ny * h->grid.nz * (h->grid.dtype == PIPE_F64 ? 8 : 4);
  void *rho = nullptr, *phi = nullptr;
  if (cudaMalloc(&rho, n) != cudaSuccess) return PIPE_ENOMEM;
  if (cudaMalloc(&phi, n) != cudaSuccess) { cudaFree(rho); return PIPE_ENOMEM; }
  cudaMemsetAsync(rho, 0, n, st);
  float ms[2] = {-1.f, -1.f};
  for (int m = 0; m < 2; ++m) {
    h->use_modes = m;
    ms[m] = time_ms([&] { return handle_solve(h, rho, phi, false, st) == PIPE_OK ? cudaSuccess
                                                                                 : cudaErrorUnknown; },
                    st, 5);
  }
  cudaStreamSynchronize(st);
  cudaFree(rho);
  cudaFree(phi);
  if (ms[0] < 0 && ms[1] < 0) return PIPE_ECUDA;
  h->use_modes = (ms[1] > 0 && (ms[0] < 0 || ms[1] <= ms[0])) ? 1 : 0;
  return PIPE_OK;
}
}  // namespace
}  // namespace pp

static int autotune_transforms(pipe_handle* h, void* stream);

extern "C" int pipe_autotune(pipe_handle* h, void* stream) {
  if (!h) return PIPE_EINVAL;
  if (!h->fft_ok) return PIPE_OK;                        // mode-space form only: nothing to choose
  const int s = autotune_transforms(h, stream);
  if (s != PIPE_OK || !h->modes_ok) return s;
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != h->device) cudaSetDevice(h->device);
  const int c = choose_form(h, static_cast<cudaStream_t>(stream));
  if (dev >= 0 && dev != h->device) cudaSetDevice(dev);
  return c;
}

// the transform form's plan: per shape, timed once per process (and cached)
static int autotune_transforms(pipe_handle* h, void* stream) {
  if (h->grid.dtype == PIPE_F32_C16) return PIPE_OK;     // fixed variant: nothing to choose
  // banded handles are keyed by their neighbour count as well
  const Key k(h->grid.nx, h->grid.nz,
              h->grid.dtype + (h->images ? 0 : 3) + (h->general ? 6 : 0) +
                  (h->banded >= 0 ? 9 * (h->banded + 1) : 0));
  {
    std::lock_guard<std::mutex> lk(g_mu);
    load_file_cache();
    auto it = cache().find(k);
    if (it != cache().end()) {
      if (h->images) h->plan = it->second;
      else { h->plan.z_warps = it->second.z_warps; h->plan.z_pipe = it->second.z_pipe; h->free_plan = it->second; }
      return PIPE_OK;
    }
  }
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != h->device) cudaSetDevice(h->device);
  Plan p;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int s = h->grid.dtype == PIPE_F64 ? tune<double>(h, st, &p) : tune<float>(h, st, &p);
  if (dev >= 0 && dev != h->device) cudaSetDevice(dev);
  if (s != PIPE_OK) return s;
  if (h->images) h->plan = p;
  else { h->plan.z_warps = p.z_warps; h->plan.z_pipe = p.z_pipe; h->free_plan = p; }
  std::lock_guard<std::mutex> lk(g_mu);
  cache()[k] = p;
  save_file_cache(k, p);
  return PIPE_OK;
}

extern "C" int pipe_get_plan(pipe_handle* h, int* z_warps, int* z_pipe, int* t_h, int* t_threads,
                             int* t_kind) {
  if (!h || !z_warps || !z_pipe || !t_h || !t_threads || !t_kind) return PIPE_EINVAL;
  const Plan& p = h->images ? h->plan : h->free_plan;
  *z_warps = h->plan.z_warps;
  *z_pipe = h->plan.z_pipe;
  *t_h = p.t_h;
  *t_threads = p.t_threads;
  *t_kind = h->use_modes ? 3 : p.t_kind;
  return PIPE_OK;
}

extern "C" int pipe_set_plan(pipe_handle* h, int z_warps, int z_pipe, int t_h, int t_threads, int t_kind) {
  if (!h) return PIPE_EINVAL;
  if ((z_warps != 4 && z_warps != 8 && z_warps != 16) || (z_pipe != 0 && z_pipe != 1) || (t_h != 1 && t_h != 2 && t_h != 4) ||
      (t_threads != 128 && t_threads != 256 && t_threads != 512) || t_kind < 0 || t_kind > 3)
    return PIPE_EINVAL;
  if (t_kind == 3) {                    // the mode-space form; the transform plan is kept
    if (!h->modes_ok) return PIPE_EUNSUPPORTED;
    h->use_modes = 1;
    return PIPE_OK;
  }
  if (!h->fft_ok) return PIPE_EUNSUPPORTED;
  if (t_kind >= 1) {
    // the N-point routine: pipe operator on cell-centred meshes, one CTA per
    // plane, the N x N plane buffer in shared memory (kind 1: or in global
    // scratch planes where the setup allocated them)
    if (!h->images || h->sx != 1 || h->sy != 1 || t_h != 1) return PIPE_EUNSUPPORTED;
    const size_t c = h->grid.dtype == PIPE_F64 ? 16 : 8;
    if (c * h->grid.nx * h->grid.ny > 200 * 1024 && (t_kind == 2 || !h->tbuf)) return PIPE_EUNSUPPORTED;
  }
  h->use_modes = 0;
  if (h->images) h->plan = Plan{z_warps, z_pipe, t_h, t_threads, t_kind};
  else {
    h->plan.z_warps = z_warps;
    h->plan.z_pipe = z_pipe;
    h->free_plan = Plan{z_warps, z_pipe, t_h, t_threads, 0};
  }
  return PIPE_OK;
}
