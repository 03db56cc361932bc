// C ABI of the pipe Poisson solver: handle management, validation, dispatch.
// The declarations and their documentation are in include/pipe_poisson.h.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <type_traits>

#include "../../include/pipe_poisson.h"
#include "green_kernels.cuh"
#include "handle.cuh"
#include "modes.cuh"
#include "modes_impl.cuh"
#include "solver.cuh"

using namespace pp;

namespace {

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// lanes per FFT group, mirroring GroupShape (cyclic FFTs) and PairShape (paired)
int sub_fft_group(int L) { return (L <= 32) ? 4 : (L <= 128 ? 8 : (L <= 512 ? 16 : 32)); }
int pair_fft_group(int L) { return (L == 16) ? 2 : (L <= 64 ? 4 : (L <= 256 ? 8 : 16)); }

// check that x is within rel of an integer; return it
bool near_int(double x, int* out) {
  const double r = std::nearbyint(x);
  if (std::fabs(x - r) > 1e-9 * std::fmax(1.0, std::fabs(x))) return false;
  *out = int(r);
  return true;
}

// PIPE_EINVAL for a malformed grid, else PIPE_EUNSUPPORTED for sizes outside
// the padded-transform path, else PIPE_OK
int validate_grid(const pipe_grid* g) {
  if (!g) return PIPE_EINVAL;
  if (g->nx <= 0 || g->ny <= 0 || g->nz <= 0) return PIPE_EINVAL;
  if (!(g->hx > 0) || !(g->hy > 0) || !(g->hz > 0)) return PIPE_EINVAL;
  if (!std::isfinite(g->hx) || !std::isfinite(g->hy) || !std::isfinite(g->hz)) return PIPE_EINVAL;
  if (g->dtype != PIPE_F32 && g->dtype != PIPE_F64 && g->dtype != PIPE_F32_C16) return PIPE_EINVAL;
  if (!is_pow2(g->nx) || !is_pow2(g->ny) || !is_pow2(g->nz)) return PIPE_EUNSUPPORTED;
  if (g->nx != g->ny) return PIPE_EUNSUPPORTED;
  if (g->nx < 16 || g->nx > 128) return PIPE_EUNSUPPORTED;
  if (g->nz < 32 || g->nz > 1024) return PIPE_EUNSUPPORTED;
  return PIPE_OK;
}

int status_of(cudaError_t e) {
  if (e == cudaSuccess) return PIPE_OK;
  if (e == cudaErrorMemoryAllocation) return PIPE_ENOMEM;
  if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return PIPE_ENODEVICE;
  return PIPE_ECUDA;
}

size_t cplx_size(int dtype) { return dtype == PIPE_F64 ? 16 : 8; }

// allocate everything but the Green spectrum; fill the twiddle tables
int alloc_common(pipe_handle* h) {
  const pipe_grid& g = h->grid;
  cudaError_t e;
  if (h->fft_ok) {
  // Green planes: the 3-D octant, the n_nb + 1 2-D spectra of the banded form,
  // or (general meshes) four complex tables [4][nz+1][2ny][2nx]
  const size_t oct = h->general ? size_t(8) * (g.nz + 1) * (2 * g.ny) * (2 * g.nx)
                                : size_t(g.nx + 1) * (g.ny + 1) * (h->banded >= 0 ? h->banded + 1 : g.nz + 1);
  const size_t work = size_t(g.nz + 1) * g.nx * g.ny * cplx_size(g.dtype);
  if ((e = cudaMalloc(&h->green64, oct * sizeof(double))) != cudaSuccess) return status_of(e);
  if ((e = cudaMalloc(&h->green32, oct * sizeof(float))) != cudaSuccess) return status_of(e);
  if ((e = cudaMalloc(&h->work, work)) != cudaSuccess) return status_of(e);
  }
  const int n = g.nx, Lz = g.nz / 2;
  // float2 and double2 tables: tw_t (n), w2_t (2n), tw_z (nz/2), w2_z (2nz)
  const size_t cnt = size_t(n) + 2 * n + Lz + 2 * g.nz + 2 * n + 2 * n;
  // one more float2 after the tables holds the device error word
  if ((e = cudaMalloc(&h->tab32, (cnt + 1) * sizeof(float2))) != cudaSuccess) return status_of(e);
  h->err = reinterpret_cast<int*>(h->tab32 + cnt);
  if ((e = cudaMemset(h->err, 0, sizeof(int))) != cudaSuccess) return status_of(e);
  if ((e = cudaMalloc(&h->tab64, cnt * sizeof(double2))) != cudaSuccess) return status_of(e);
  h->tw_t32 = h->tab32; h->w2_t32 = h->tw_t32 + n; h->tw_z32 = h->w2_t32 + 2 * n; h->w2_z32 = h->tw_z32 + Lz;
  h->tw_t2_32 = h->w2_z32 + 2 * g.nz;
  h->tw_t2c_32 = h->tw_t2_32 + 2 * n;
  h->tw_t64 = h->tab64; h->w2_t64 = h->tw_t64 + n; h->tw_z64 = h->w2_t64 + 2 * n; h->w2_z64 = h->tw_z64 + Lz;
  h->tw_t2_64 = h->w2_z64 + 2 * g.nz;
  h->tw_t2c_64 = h->tw_t2_64 + 2 * n;
  cudaStream_t st = nullptr;
  launch_tables<float2>(h->tw_t32, h->w2_t32, n, sub_fft_group(n), 2 * n, st);
  launch_tables<float2>(h->tw_z32, h->w2_z32, Lz, sub_fft_group(Lz), 2 * g.nz, st);
  launch_tables<double2>(h->tw_t64, h->w2_t64, n, sub_fft_group(n), 2 * n, st);
  launch_tables<double2>(h->tw_z64, h->w2_z64, Lz, sub_fft_group(Lz), 2 * g.nz, st);
  launch_tables<float2>(h->tw_t2_32, nullptr, 2 * n, pair_fft_group(2 * n), 0, st);
  launch_tables<double2>(h->tw_t2_64, nullptr, 2 * n, pair_fft_group(2 * n), 0, st);
  launch_tables<float2>(h->tw_t2c_32, nullptr, 2 * n, sub_fft_group(2 * n), 0, st);
  launch_tables<double2>(h->tw_t2c_64, nullptr, 2 * n, sub_fft_group(2 * n), 0, st);
  if ((e = cudaGetLastError()) != cudaSuccess) return status_of(e);
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return status_of(e);
  return PIPE_OK;
}

void free_handle(pipe_handle* h) {
  if (!h) return;
  DeviceGuard dg(h->device);
  cudaDeviceSynchronize();
  cudaFree(h->green64); cudaFree(h->green32); cudaFree(h->work);
  cudaFree(h->tab32); cudaFree(h->tab64);
  cudaFree(h->stage_rho); cudaFree(h->stage_phi);
  cudaFree(h->tbuf);
  cudaFree(h->msx64); cudaFree(h->msy64); cudaFree(h->mgz64);
  cudaFree(h->msx32); cudaFree(h->msy32); cudaFree(h->mgz32);
  cudaFree(h->mwork);
  cudaFree(h->mkb64); cudaFree(h->mkb32);
  std::free(h->msy_host);
  for (int k = 0; k < 2; ++k) {
    cudaFree(h->ring_rho[k]);
    cudaFree(h->ring_phi[k]);
    if (h->ev_in[k]) cudaEventDestroy(h->ev_in[k]);
    if (h->ev_done[k]) cudaEventDestroy(h->ev_done[k]);
    if (h->ev_out[k]) cudaEventDestroy(h->ev_out[k]);
  }
  if (h->copy_in) cudaStreamDestroy(h->copy_in);
  if (h->copy_out) cudaStreamDestroy(h->copy_out);
  batch_release(h);
  delete h;
}

}  // namespace

namespace pp {

template <>
SolveArgs<float> make_args<float>(pipe_handle* h, const void* rho, void* phi, void* work) {
  SolveArgs<float> a{};
  a.rho = static_cast<const float*>(rho); a.phi = static_cast<float*>(phi);
  a.work = static_cast<float2*>(work); a.green = h->green32;
  a.tw_t = h->tw_t32; a.w2_t = h->w2_t32; a.tw_z = h->tw_z32; a.w2_z = h->w2_z32;
  a.tw_t2 = h->tw_t2_32;
  a.tw_t2c = h->tw_t2c_32;
  a.nx = h->grid.nx; a.ny = h->grid.ny; a.nz = h->grid.nz;
  a.sx = h->sx; a.sy = h->sy; a.images = h->images;
  a.err = h->err;
  if (h->grid.dtype == PIPE_F32_C16) {
    // work: (nz+1) nx ny complex-FP16 values, then the two scale tables
    const size_t nodes = size_t(h->grid.nx) * h->grid.ny;
    a.zscale = reinterpret_cast<float*>(static_cast<char*>(work) + (h->grid.nz + 1) * nodes * 4);
    a.tscale = a.zscale + nodes;
    a.zcols = z_tile_cols(h->grid.nz, h->plan.z_warps);
  }
  return a;
}
template <>
SolveArgs<double> make_args<double>(pipe_handle* h, const void* rho, void* phi, void* work) {
  SolveArgs<double> a{};
  a.rho = static_cast<const double*>(rho); a.phi = static_cast<double*>(phi);
  a.work = static_cast<double2*>(work); a.green = h->green64;
  a.tw_t = h->tw_t64; a.w2_t = h->w2_t64; a.tw_z = h->tw_z64; a.w2_z = h->w2_z64;
  a.tw_t2 = h->tw_t2_64;
  a.tw_t2c = h->tw_t2c_64;
  a.nx = h->grid.nx; a.ny = h->grid.ny; a.nz = h->grid.nz;
  a.sx = h->sx; a.sy = h->sy; a.images = h->images;
  a.tbuf = static_cast<double2*>(h->tbuf);
  a.err = h->err;
  return a;
}

template <typename T>
cudaError_t transverse_stage(pipe_handle* h, bool adjoint, const SolveArgs<T>& a, cudaStream_t st) {
  if (h->general) return launch_transverse_gen<T>(adjoint, h->plan.t_threads, a, st);
  if (h->images)
    return launch_transverse_sym<T>(adjoint, h->plan.t_kind, h->plan.t_h, h->plan.t_threads, a, st);
  return launch_transverse<T>(adjoint, h->free_plan.t_h, h->free_plan.t_threads, a, st);
}

// the three stages of the padded-transform form on the buffers of `a`
template <typename T>
int transform_chain(pipe_handle* h, const SolveArgs<T>& a, bool adjoint, cudaStream_t st) {
  const int zw = h->plan.z_warps, zp = h->plan.z_pipe;
  cudaError_t e;
  if ((e = launch_z<T>(true, zw, zp, adjoint, a, st)) != cudaSuccess) return status_of(e);
  if ((e = transverse_stage<T>(h, adjoint, a, st)) != cudaSuccess) return status_of(e);
  if ((e = launch_z<T>(false, zw, zp, adjoint, a, st)) != cudaSuccess) return status_of(e);
  return PIPE_OK;
}
template int transform_chain<float>(pipe_handle*, const SolveArgs<float>&, bool, cudaStream_t);
template int transform_chain<double>(pipe_handle*, const SolveArgs<double>&, bool, cudaStream_t);

}  // namespace pp

namespace {

template <typename T>
int run_solve(pipe_handle* h, const void* rho, void* phi, bool adjoint, cudaStream_t st) {
  SolveArgs<T> a = make_args<T>(h, rho, phi, h->work);
  a.stage_drop = h->inject_drop;               // a pending failure-detection test
  a.stage_polls = h->inject_polls;
  h->inject_drop = 0;
  h->inject_polls = 0;
  cudaError_t e;
  // the banded operator is symmetric: the adjoint is the same computation;
  // so is the mode-space form (full or banded)
  if (h->use_modes) return mode_solve(h, rho, phi, h->mwork, st);
  if (h->banded >= 0) return status_of(launch_banded<T>(h->plan.t_threads, a, h->banded, st));
  if constexpr (std::is_same<T, float>::value) {
    if (h->grid.dtype == PIPE_F32_C16) {
      const int zw = h->plan.z_warps;
      if ((e = launch_z_c16(true, zw, adjoint, a, st)) != cudaSuccess) return status_of(e);
      if ((e = launch_transverse_c16(adjoint, h->plan.t_threads, a, st)) != cudaSuccess) return status_of(e);
      if ((e = launch_z_c16(false, zw, adjoint, a, st)) != cudaSuccess) return status_of(e);
      return PIPE_OK;
    }
  }
  return transform_chain<T>(h, a, adjoint, st);
}

int check_ptr(const void* p) {
  if (!p) return PIPE_EINVAL;
  if (reinterpret_cast<uintptr_t>(p) % 16 != 0) return PIPE_EINVAL;
  return PIPE_OK;
}

int finish_setup(pipe_handle* h, pipe_handle** out) {
  *out = h;
  return PIPE_OK;
}

}  // namespace

namespace pp {
int mode_xblocks(const pipe_handle* h) {
  const int xb = h->grid.nx / (h->grid.dtype == PIPE_F64 ? ModeShape<double>::XB : ModeShape<float>::XB);
  return xb / mode_cluster(xb);
}

size_t mode_scratch_bytes(const pipe_handle* h) {
  const size_t mc = size_t(h->mxp) * h->myp;
  return (h->grid.dtype == PIPE_F64 ? 8 : 4) * size_t(mode_xblocks(h) + 1) * mc * h->grid.nz;
}

template <typename T>
ModeArgs<T> mode_args(const pipe_handle* h, const void* rho, void* phi, void* part, void* psi) {
  constexpr bool D = sizeof(T) == 8;
  ModeArgs<T> a{};
  a.rho = static_cast<const T*>(rho);
  a.phi = static_cast<T*>(phi);
  a.part = static_cast<T*>(part);
  a.psi = static_cast<T*>(psi);
  a.sx = reinterpret_cast<const T*>(D ? static_cast<const void*>(h->msx64) : static_cast<const void*>(h->msx32));
  a.sy = reinterpret_cast<const T*>(D ? static_cast<const void*>(h->msy64) : static_cast<const void*>(h->msy32));
  a.gz = reinterpret_cast<const T*>(D ? static_cast<const void*>(h->mgz64) : static_cast<const void*>(h->mgz32));
  a.tw_z = reinterpret_cast<const C2<T>*>(D ? static_cast<const void*>(h->tw_z64) : static_cast<const void*>(h->tw_z32));
  a.w2_z = reinterpret_cast<const C2<T>*>(D ? static_cast<const void*>(h->w2_z64) : static_cast<const void*>(h->w2_z32));
  a.nx = h->grid.nx; a.ny = h->grid.ny; a.nz = h->grid.nz;
  a.mx = h->geom.modes_m;
  a.mxp = h->mxp;
  a.mc = h->mxp * h->myp;
  a.kb = reinterpret_cast<const T*>(D ? static_cast<const void*>(h->mkb64) : static_cast<const void*>(h->mkb32));
  a.nb = h->banded;
  return a;
}

template <typename T>
int mode_stage(const pipe_handle* h, int stage, const void* rho, void* phi, void* part, void* psi,
               cudaStream_t st) {
  const ModeArgs<T> a = mode_args<T>(h, rho, phi, part, psi);
  if constexpr (sizeof(T) == 4) {
    if (h->mfast && stage != 1) return status_of(launch_mode_fast(stage, h->myp, a, h->msy_host, st));
  }
  return status_of(launch_mode_stage<T>(stage, h->myp, h->fy != 0, a, st));
}

ModeArgs<float> mode_args_f32(const pipe_handle* h) {
  void* psi = static_cast<char*>(h->mwork) + sizeof(float) * size_t(mode_xblocks(h)) * h->mxp * h->myp * h->grid.nz;
  return mode_args<float>(h, nullptr, nullptr, h->mwork, psi);
}

int mode_solve(pipe_handle* h, const void* rho, void* phi, void* scratch, cudaStream_t st) {
  const size_t esz = h->grid.dtype == PIPE_F64 ? 8 : 4;
  void* psi = static_cast<char*>(scratch) + esz * size_t(mode_xblocks(h)) * h->mxp * h->myp * h->grid.nz;
  int s = PIPE_OK;
  for (int stage = 0; stage < 3 && s == PIPE_OK; ++stage)
    s = h->grid.dtype == PIPE_F64 ? mode_stage<double>(h, stage, rho, phi, scratch, psi, st)
                                  : mode_stage<float>(h, stage, rho, phi, scratch, psi, st);
  return s;
}

int handle_solve(pipe_handle* h, const void* rho, void* phi, bool adjoint, cudaStream_t st) {
  return h->grid.dtype == PIPE_F64 ? run_solve<double>(h, rho, phi, adjoint, st)
                                   : run_solve<float>(h, rho, phi, adjoint, st);
}
}  // namespace pp

extern "C" {

const char* pipe_version(void) { return "pipe-poisson-gb300 0.1 (sm_103a)"; }

const char* pipe_strerror(int s) {
  switch (s) {
    case PIPE_OK: return "ok";
    case PIPE_EINVAL: return "invalid argument";
    case PIPE_ENOMEM: return "out of memory";
    case PIPE_EUNSUPPORTED: return "unsupported size or geometry";
    case PIPE_ECUDA: return "CUDA error";
    case PIPE_ETIMEOUT: return "device-side wait timed out";
    case PIPE_ENODEVICE: return "no CUDA device";
    default: return "unknown status";
  }
}

double pipe_selftest_twiddles(void) {
  // reference: long double cos/sin of the exactly reduced angle 2 pi (k mod n) / n
  const long double two_pi = 6.283185307179586476925286766559005768L;
  double worst = 0.0;
  auto check = [&](long k, long n) {
    long kr = k % n;
    if (kr < 0) kr += n;
    const long double ang = two_pi * (long double)kr / (long double)n;
    worst = std::fmax(worst, std::fabs(ccos2pi(k, n) - double(cosl(ang))));
    worst = std::fmax(worst, std::fabs(csin2pi(k, n) - double(sinl(ang))));
  };
  for (long n = 1; n <= 4096; n *= 2)
    for (long k = -n; k <= 2 * n; ++k) check(k, n);
  for (long n : {3L, 5L, 12L, 100L, 1000L})
    for (long k = 0; k < n; ++k) check(k, n);
  return worst;
}

static int setup_pipe(const pipe_geometry* geom, const pipe_grid* grid, int igf, int n_nb,
                      pipe_handle** out) {
  if (!out) return PIPE_EINVAL;
  *out = nullptr;
  if (!geom) return PIPE_EINVAL;
  if (igf != PIPE_GREEN_ORDINARY && igf != PIPE_GREEN_IGF) return PIPE_EINVAL;
  int st = validate_grid(grid);
  if (st == PIPE_EINVAL) return st;
  if (!(geom->a > 0) || !(geom->b > 0) || !std::isfinite(geom->a) || !std::isfinite(geom->b))
    return PIPE_EINVAL;
  if (geom->modes_m < 1 || geom->modes_n < 1) return PIPE_EINVAL;
  // the mesh must lie inside the pipe
  const double tol = 1e-12;
  if (geom->x0 < -tol * geom->a || geom->y0 < -tol * geom->b) return PIPE_EINVAL;
  if (geom->x0 + (grid->nx - 1) * grid->hx > geom->a * (1 + tol)) return PIPE_EINVAL;
  if (geom->y0 + (grid->ny - 1) * grid->hy > geom->b * (1 + tol)) return PIPE_EINVAL;
  // the mode-space form (modes_impl.cuh): any mesh inside the pipe with
  // nx, ny multiples of 16 (up to 4096), nz a power of two in 32..1024 and at
  // most 32 modes per axis, FP32 or FP64, full or banded operator
  const bool fold = std::fabs(2.0 * geom->y0 + (grid->ny - 1) * grid->hy - geom->b) <= 1e-12 * geom->b;
  bool modes_ok = n_nb < grid->nz && (grid->dtype == PIPE_F32 || grid->dtype == PIPE_F64) &&
                  grid->nx % 16 == 0 && grid->ny % 16 == 0 && grid->nx <= 4096 && grid->ny <= 4096 &&
                  is_pow2(grid->nz) && grid->nz >= 32 && grid->nz <= 1024 && geom->modes_m <= 32 &&
                  mode_slots(geom->modes_n, fold) > 0;
  if (modes_ok) {                       // its kernels' shared memory must fit
    const int myp = mode_slots(geom->modes_n, fold), mxp = (geom->modes_m + 3) / 4 * 4;
    const bool f64 = grid->dtype == PIPE_F64;
    const size_t ps = f64 ? mode_proj_smem<double>(grid->ny, mxp, myp, fold)
                          : mode_proj_smem<float>(grid->ny, mxp, myp, fold);
    const size_t bs = f64 ? mode_back_smem<double>(grid->ny, geom->modes_m, mxp, myp, fold)
                          : mode_back_smem<float>(grid->ny, geom->modes_m, mxp, myp, fold);
    if (ps > kMaxSmem || bs > kMaxSmem) modes_ok = false;
  }
  // the padded-transform form of Eq. 10: st is PIPE_OK or the reason it
  // cannot take this mesh
  if (st == PIPE_OK && (geom->modes_m > 4096 || geom->modes_n > 4096)) st = PIPE_EUNSUPPORTED;
  // meshes spanning the pipe with integer correlation shifts use the real
  // octant; any other mesh inside the pipe (a transverse window) the four
  // full tables, for planes up to 64 x 64
  int sx = 0, sy = 0;
  const bool spanning = std::fabs(grid->nx * grid->hx - geom->a) <= 1e-12 * geom->a &&
                        std::fabs(grid->ny * grid->hy - geom->b) <= 1e-12 * geom->b &&
                        near_int(2.0 * geom->x0 / grid->hx, &sx) && near_int(2.0 * geom->y0 / grid->hy, &sy);
  if (!spanning) {
    if (st == PIPE_OK && (grid->nx > 64 || n_nb >= 0 || grid->dtype == PIPE_F32_C16)) st = PIPE_EUNSUPPORTED;
    sx = sy = -1;
  }
  if (st != PIPE_OK && !modes_ok) return st;

  if (grid->dtype == PIPE_F32_C16 && (sx != 1 || sy != 1 || n_nb >= 0)) return PIPE_EUNSUPPORTED;
  if (n_nb >= 0) {
    // the banded form: in mode space (a stencil on each mode column) where the
    // mode form takes the mesh; its transform form takes cell-centred meshes
    // (n-point transverse routine, planes paired along z, the nx*ny plane
    // buffer in shared memory)
    if (n_nb >= grid->nz) return PIPE_EINVAL;
    if (st == PIPE_OK && (sx != 1 || sy != 1 || cplx_size(grid->dtype) * grid->nx * grid->ny > 200 * 1024))
      st = PIPE_EUNSUPPORTED;
    if (st != PIPE_OK && !modes_ok) return st;
  }
  const bool fft_ok = st == PIPE_OK;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return PIPE_ENODEVICE;
  pipe_handle* h = new (std::nothrow) pipe_handle();
  if (!h) return PIPE_ENOMEM;
  cudaGetDevice(&h->device);
  // reserve the no-alloc solve's fixed array on this device now, while the
  // program is initialising (a failure is reported by that entry point)
  noalloc_reserve(h->device);
  h->geom = *geom;
  h->grid = *grid;
  h->kind = igf;
  h->sx = sx;
  h->sy = sy;
  h->images = 1;
  h->banded = n_nb;
  h->general = spanning ? 0 : 1;
  h->fft_ok = fft_ok ? 1 : 0;
  h->modes_ok = modes_ok ? 1 : 0;
  h->plan = default_plan(grid->nx, grid->nz, grid->dtype == PIPE_F64, sx == 1 && sy == 1);
  if (n_nb >= 0) h->plan.t_threads = 256;
  if (h->general) h->plan.t_threads = grid->dtype == PIPE_F64 ? 128 : 256;
  h->free_plan = default_free_plan(grid->nx, grid->nz, grid->dtype == PIPE_F64);
  if ((st = alloc_common(h)) != PIPE_OK) { free_handle(h); return st; }
  GreenSpec s;
  s.nx = grid->nx; s.ny = grid->ny; s.nz = grid->nz;
  s.hx = grid->hx; s.hy = grid->hy; s.hz = grid->hz;
  s.a = geom->a; s.b = geom->b;
  s.modes_m = geom->modes_m; s.modes_n = geom->modes_n;
  s.igf = igf;
  if (modes_ok) {
    h->fy = fold ? 1 : 0;
    h->mxp = (geom->modes_m + 3) / 4 * 4;
    h->myp = mode_slots(geom->modes_n, fold);
    const size_t nsx = size_t(grid->nx) * h->mxp, nsy = size_t(fold ? grid->ny / 2 : grid->ny) * h->myp;
    const size_t ngz = size_t(h->mxp) * h->myp * (grid->nz + 1);
    if (cudaMalloc(&h->msx64, nsx * 8) != cudaSuccess || cudaMalloc(&h->msx32, nsx * 4) != cudaSuccess ||
        cudaMalloc(&h->msy64, nsy * 8) != cudaSuccess || cudaMalloc(&h->msy32, nsy * 4) != cudaSuccess ||
        cudaMalloc(&h->mgz64, ngz * 8) != cudaSuccess || cudaMalloc(&h->mgz32, ngz * 4) != cudaSuccess ||
        cudaMalloc(&h->mwork, mode_scratch_bytes(h)) != cudaSuccess) {
      free_handle(h);
      return PIPE_ENOMEM;
    }
    cudaError_t e = build_mode_tables(s, geom->x0, geom->y0, h->mxp, h->myp, h->fy, h->msx64, h->msx32,
                                      h->msy64, h->msy32, h->mgz64, h->mgz32, nullptr);
    if (e != cudaSuccess) { free_handle(h); return status_of(e); }
    if (n_nb >= 0) {                     // the banded operator's z stencil
      const size_t nkb = size_t(h->mxp) * h->myp * (n_nb + 1);
      if (cudaMalloc(&h->mkb64, nkb * 8) != cudaSuccess || cudaMalloc(&h->mkb32, nkb * 4) != cudaSuccess) {
        free_handle(h);
        return PIPE_ENOMEM;
      }
      if ((e = build_mode_band(s, h->mxp, h->myp, h->fy, n_nb, h->mkb64, h->mkb32, nullptr)) != cudaSuccess) {
        free_handle(h);
        return status_of(e);
      }
    }
    if (grid->dtype == PIPE_F32 && mode_fast_ok(grid->ny, grid->nx, h->myp, fold)) {
      h->msy_host = static_cast<float*>(std::malloc(nsy * sizeof(float)));
      if (!h->msy_host) { free_handle(h); return PIPE_ENOMEM; }
      if ((e = cudaMemcpy(h->msy_host, h->msy32, nsy * sizeof(float), cudaMemcpyDeviceToHost)) != cudaSuccess) {
        free_handle(h);
        return status_of(e);
      }
      h->mfast = 1;
    }
    // the default: the mode-space form where the modes are at most half the
    // transverse mesh (or where the padded transforms cannot take the mesh)
    const int nmin = grid->nx < grid->ny ? grid->nx : grid->ny;
    h->use_modes = (!fft_ok || 2 * (h->mxp > h->myp ? h->mxp : h->myp) <= nmin) ? 1 : 0;
  }
  if (!fft_ok) return finish_setup(h, out);
  // FP64 planes too large for shared memory: the n-point routine's plane
  // buffers in global memory (one per kz plane)
  if (!h->general && n_nb < 0 && sx == 1 && sy == 1 && cplx_size(grid->dtype) * grid->nx * grid->ny > 200 * 1024) {
    const size_t tb = size_t(grid->nz + 1) * grid->nx * grid->ny * cplx_size(grid->dtype);
    if (cudaMalloc(&h->tbuf, tb) != cudaSuccess) { free_handle(h); return PIPE_ENOMEM; }
  }
  s.scale = grid->hx * grid->hy * grid->hz / (8.0 * grid->nx * grid->ny * grid->nz);
  if (n_nb >= 0) {                       // 2-D spectra of the offsets 0..n_nb
    s.nz = n_nb;
    s.scale = grid->hx * grid->hy * grid->hz / (4.0 * grid->nx * grid->ny);
  }
  cudaError_t e = h->general
      ? build_general_spectra(s, geom->x0, geom->y0, reinterpret_cast<double2*>(h->green64),
                              reinterpret_cast<float2*>(h->green32), nullptr)
      : build_pipe_spectrum(s, h->green64, h->green32, nullptr, n_nb < 0);
  if (e != cudaSuccess) { free_handle(h); return status_of(e); }
  return finish_setup(h, out);
}

int pipe_green_setup(const pipe_geometry* geom, const pipe_grid* grid, int igf, pipe_handle** out) {
  return setup_pipe(geom, grid, igf, -1, out);
}

int pipe_banded_setup(const pipe_geometry* geom, const pipe_grid* grid, int igf, int n_neighbors,
                      pipe_handle** out) {
  if (out) *out = nullptr;
  if (n_neighbors < 0) return PIPE_EINVAL;
  return setup_pipe(geom, grid, igf, n_neighbors, out);
}

int pipe_free_space_setup(const pipe_grid* grid, double self_value, pipe_handle** out) {
  if (!out) return PIPE_EINVAL;
  *out = nullptr;
  int st = validate_grid(grid);
  if (st != PIPE_OK) return st;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return PIPE_ENODEVICE;
  pipe_handle* h = new (std::nothrow) pipe_handle();
  if (!h) return PIPE_ENOMEM;
  cudaGetDevice(&h->device);
  // reserve the no-alloc solve's fixed array on this device now, while the
  // program is initialising (a failure is reported by that entry point)
  noalloc_reserve(h->device);
  std::memset(&h->geom, 0, sizeof(h->geom));
  h->grid = *grid;
  h->kind = 2;
  h->sx = h->sy = 0;
  h->images = 0;
  h->plan = default_plan(grid->nx, grid->nz, grid->dtype == PIPE_F64, false);
  h->free_plan = default_free_plan(grid->nx, grid->nz, grid->dtype == PIPE_F64);
  if ((st = alloc_common(h)) != PIPE_OK) { free_handle(h); return st; }
  if (!(self_value > 0)) self_value = 1.0 / std::fmin(grid->hx, std::fmin(grid->hy, grid->hz));
  GreenSpec s;
  s.nx = grid->nx; s.ny = grid->ny; s.nz = grid->nz;
  s.hx = grid->hx; s.hy = grid->hy; s.hz = grid->hz;
  s.a = s.b = 0; s.modes_m = s.modes_n = 0; s.igf = 0;
  s.scale = grid->hx * grid->hy * grid->hz / (8.0 * grid->nx * grid->ny * grid->nz);
  cudaError_t e = build_free_spectrum(s, self_value, h->green64, h->green32, nullptr);
  if (e != cudaSuccess) { free_handle(h); return status_of(e); }
  return finish_setup(h, out);
}

void pipe_green_destroy(pipe_handle* h) { free_handle(h); }

int pipe_poisson_solve(pipe_handle* h, const void* rho, void* phi, void* stream) {
  if (!h) return PIPE_EINVAL;
  int st;
  if ((st = check_ptr(rho)) != PIPE_OK || (st = check_ptr(phi)) != PIPE_OK) return st;
  DeviceGuard dg(h->device);
  if (!dg.ok) return PIPE_ECUDA;
  return handle_solve(h, rho, phi, false, static_cast<cudaStream_t>(stream));
}

int pipe_poisson_adjoint(pipe_handle* h, const void* dphi, void* drho, void* stream) {
  if (!h) return PIPE_EINVAL;
  int st;
  if ((st = check_ptr(dphi)) != PIPE_OK || (st = check_ptr(drho)) != PIPE_OK) return st;
  DeviceGuard dg(h->device);
  if (!dg.ok) return PIPE_ECUDA;
  return handle_solve(h, dphi, drho, true, static_cast<cudaStream_t>(stream));
}

int pipe_poisson_solve_host(pipe_handle* h, const void* rho_host, void* phi_host, void* stream) {
  if (!h || !rho_host || !phi_host) return PIPE_EINVAL;
  DeviceGuard dg(h->device);
  if (!dg.ok) return PIPE_ECUDA;
  const size_t bytes = size_t(h->grid.nx) * h->grid.ny * h->grid.nz *
                       (h->grid.dtype == PIPE_F64 ? 8 : 4);
  cudaError_t e;
  if (!h->stage_rho) {
    if ((e = cudaMalloc(&h->stage_rho, bytes)) != cudaSuccess) return status_of(e);
    if ((e = cudaMalloc(&h->stage_phi, bytes)) != cudaSuccess) return status_of(e);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if ((e = cudaMemcpyAsync(h->stage_rho, rho_host, bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return status_of(e);
  int s = handle_solve(h, h->stage_rho, h->stage_phi, false, st);
  if (s != PIPE_OK) return s;
  if ((e = cudaMemcpyAsync(phi_host, h->stage_phi, bytes, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return status_of(e);
  return status_of(cudaStreamSynchronize(st));
}

int pipe_inject_stage_fault(pipe_handle* h, int drop_copy, long long poll_limit) {
  if (!h || drop_copy < 0 || poll_limit < 1) return PIPE_EINVAL;
  h->inject_drop = drop_copy + 1;
  h->inject_polls = poll_limit;
  return PIPE_OK;
}

int pipe_status(pipe_handle* h) {
  if (!h || !h->err) return PIPE_EINVAL;
  DeviceGuard dg(h->device);
  int word = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&word, h->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(h->err, 0, sizeof(int));
  if (e != cudaSuccess) return status_of(e);
  return word;
}

int pipe_green_spectrum(pipe_handle* h, double* out, size_t count) {
  if (!h || !out) return PIPE_EINVAL;
  if (!h->fft_ok) return PIPE_EUNSUPPORTED;
  const int planes = h->banded >= 0 ? h->banded + 1 : h->grid.nz + 1;
  const size_t oct = h->general ? size_t(8) * (h->grid.nz + 1) * (2 * h->grid.ny) * (2 * h->grid.nx)
                                : size_t(h->grid.nx + 1) * (h->grid.ny + 1) * planes;
  if (count != oct) return PIPE_EINVAL;
  DeviceGuard dg(h->device);
  return status_of(cudaMemcpy(out, h->green64, oct * sizeof(double), cudaMemcpyDeviceToHost));
}

int pipe_stage_z_forward(pipe_handle* h, const void* rho, void* spec, int adjoint, void* stream) {
  if (!h) return PIPE_EINVAL;
  if (!h->fft_ok) return PIPE_EUNSUPPORTED;                 // mode-space handle only
  if (h->banded >= 0 || h->grid.dtype == PIPE_F32_C16) return PIPE_EUNSUPPORTED;      // no z spectrum in the banded form
  int st;
  if ((st = check_ptr(rho)) != PIPE_OK || (st = check_ptr(spec)) != PIPE_OK) return st;
  DeviceGuard dg(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (h->grid.dtype == PIPE_F64)
    e = launch_z<double>(true, h->plan.z_warps, h->plan.z_pipe, adjoint != 0, make_args<double>(h, rho, nullptr, spec), s);
  else
    e = launch_z<float>(true, h->plan.z_warps, h->plan.z_pipe, adjoint != 0, make_args<float>(h, rho, nullptr, spec), s);
  return status_of(e);
}

int pipe_stage_transverse(pipe_handle* h, void* spec, int adjoint, void* stream) {
  if (!h) return PIPE_EINVAL;
  if (!h->fft_ok) return PIPE_EUNSUPPORTED;                 // mode-space handle only
  if (h->banded >= 0 || h->grid.dtype == PIPE_F32_C16) return PIPE_EUNSUPPORTED;      // no z spectrum in the banded form
  int st;
  if ((st = check_ptr(spec)) != PIPE_OK) return st;
  DeviceGuard dg(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (h->grid.dtype == PIPE_F64)
    e = transverse_stage<double>(h, adjoint != 0, make_args<double>(h, nullptr, nullptr, spec), s);
  else
    e = transverse_stage<float>(h, adjoint != 0, make_args<float>(h, nullptr, nullptr, spec), s);
  return status_of(e);
}

int pipe_stage_z_inverse(pipe_handle* h, const void* spec, void* phi, int adjoint, void* stream) {
  if (!h) return PIPE_EINVAL;
  if (!h->fft_ok) return PIPE_EUNSUPPORTED;                 // mode-space handle only
  if (h->banded >= 0 || h->grid.dtype == PIPE_F32_C16) return PIPE_EUNSUPPORTED;      // no z spectrum in the banded form
  int st;
  if ((st = check_ptr(spec)) != PIPE_OK || (st = check_ptr(phi)) != PIPE_OK) return st;
  DeviceGuard dg(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  void* sp = const_cast<void*>(spec);
  if (h->grid.dtype == PIPE_F64)
    e = launch_z<double>(false, h->plan.z_warps, h->plan.z_pipe, adjoint != 0, make_args<double>(h, nullptr, phi, sp), s);
  else
    e = launch_z<float>(false, h->plan.z_warps, h->plan.z_pipe, adjoint != 0, make_args<float>(h, nullptr, phi, sp), s);
  return status_of(e);
}

int pipe_mode_layout(pipe_handle* h, int* mx, int* mxp, int* myp, int* fold, int* xblocks) {
  if (!h || !mx || !mxp || !myp || !fold || !xblocks) return PIPE_EINVAL;
  if (!h->modes_ok) return PIPE_EUNSUPPORTED;
  *mx = h->geom.modes_m;
  *mxp = h->mxp;
  *myp = h->myp;
  *fold = h->fy;
  *xblocks = mode_xblocks(h);
  return PIPE_OK;
}

int pipe_mode_spectrum(pipe_handle* h, double* out, size_t count) {
  if (!h || !out) return PIPE_EINVAL;
  if (!h->modes_ok) return PIPE_EUNSUPPORTED;
  if (count != size_t(h->mxp) * h->myp * (h->grid.nz + 1)) return PIPE_EINVAL;
  DeviceGuard dg(h->device);
  return status_of(cudaMemcpy(out, h->mgz64, count * sizeof(double), cudaMemcpyDeviceToHost));
}

int pipe_stage_modes(pipe_handle* h, int stage, const void* in, void* out, void* stream) {
  if (!h) return PIPE_EINVAL;
  if (!h->modes_ok) return PIPE_EUNSUPPORTED;
  if (stage < 0 || stage > 2) return PIPE_EINVAL;
  int st;
  if ((st = check_ptr(in)) != PIPE_OK || (st = check_ptr(out)) != PIPE_OK) return st;
  DeviceGuard dg(h->device);
  if (!dg.ok) return PIPE_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* vin = const_cast<void*>(in);
  // stage 0: rho -> part; 1: part -> psi; 2: psi -> phi
  void* rho = stage == 0 ? vin : nullptr;
  void* part = stage == 0 ? out : (stage == 1 ? vin : nullptr);
  void* psi = stage == 1 ? out : (stage == 2 ? vin : nullptr);
  void* phi = stage == 2 ? out : nullptr;
  return h->grid.dtype == PIPE_F64 ? mode_stage<double>(h, stage, rho, phi, part, psi, s)
                                   : mode_stage<float>(h, stage, rho, phi, part, psi, s);
}

}  // extern "C"
