// Batched solves: many independent pipe solves (different grids, geometries,
// Green functions) in one persistent kernel launch.
//
// The launch runs one CTA per SM (as many as are co-resident).
// CTAs take items (a group of z-forward tiles, one transverse kz plane, or a
// group of z-inverse tiles of one solve) from a work list with an atomic
// counter.  Every item appears in the list after all items it depends on,
// so an item only ever waits for items that were handed out before it and
// are being processed by running CTAs: the launch cannot deadlock.  A transverse item of solve s waits until all
// z-forward tiles of s are done, a z-inverse item until all planes of s are
// done; completion is counted per solve and stage (release: fence + atomic
// add; acquire: ld.acquire.gpu).  Every wait is bounded: after spin_limit
// polls (or once another wait has failed) the CTA records PIPE_ETIMEOUT in
// the status word, skips the item and continues, so the kernel always ends.
//
// The CTA has 512 threads (16 warps; every item routine fits 128 registers).
// Items run the same device routines as the per-stage kernels: z tiles of 16
// warps (pipelined where the double buffer fits), transverse planes with the
// cyclic-layout routine of the (1 CTA, 512 threads) plan; single solves with
// that transverse plan give the same bits.
//
// The solves left outside the persistent launch run as their own launches,
// on the caller's stream or dealt to side streams.  FP32 mode-space solves of
// one shape and one y-mode table among them can run as a group: one launch
// per stage (projection, z convolution, back-projection) for up to 64 solves,
// each CTA finding its solve from its block index.  A stage of many solves is
// a grid of many waves, so the reduction phase of some CTAs overlaps the
// field streams of others.  The tuner times the persistent/outside split, the
// work-list order, the side streams and the grouping, and keeps the fastest.
#include <cuda_runtime.h>

#include <cstring>
#include <new>
#include <algorithm>
#include <vector>

#include "../../include/pipe_poisson.h"
#include "handle.cuh"
#include "modes.cuh"
#include "modes_impl.cuh"
#include "tdst_impl.cuh"
#include "tsym_impl.cuh"
#include "zfft_impl.cuh"

namespace pp {

constexpr int kMaxBatch = 128;
constexpr int kBatchThreads = 512;   // 16 warps: every item routine fits 128 registers
constexpr int kBatchZWarps = 16;

template <typename T>
struct BatchParams {
  const SolveArgs<T>* solves;   // [n], rho/phi taken from the arrays below
  const int2* items;            // [total]: (solve, stage << 24 | index)
  const int2* need;             // [n]: (z-forward items, transverse items) of each solve
  const int2* per;              // [n]: (tiles per z item, planes per transverse item)
  int* done;                    // [n][2]: completed z-forward tiles, planes
  int* counter;                 // next item
  int* status;                  // PIPE_OK or PIPE_ETIMEOUT
  int total;
  int n;
  long long spin_limit;
  int drop_stage;               // test hook: items of this stage are skipped (-1: none)
  const T* rho[kMaxBatch];
  T* phi[kMaxBatch];
};

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// a z item is `per` consecutive tiles
template <typename T, int NZ>
constexpr bool z_pipe_fits() {
  using Cfg = ZCfg<T, NZ, kBatchZWarps>;
  return Cfg::fwd_pipe_smem() <= kMaxSmem && Cfg::inv_pipe_smem() <= kMaxSmem;
}

template <typename T, int NZ>
__device__ __noinline__ void z_item(bool forward, const SolveArgs<T>& a, int item, int per,
                                    unsigned char* smem) {
  const int ntiles = a.nx * a.ny / ZCfg<T, NZ, kBatchZWarps>::COLS;
  const int first = item * per;
  const int count = (ntiles - first) < per ? (ntiles - first) : per;
  if constexpr (z_pipe_fits<T, NZ>()) {          // the pipelined multi-tile routine
    if (forward) zfwd_tiles_pipe<T, NZ, kBatchZWarps, false>(a, first, 1, count, smem);
    else zinv_tiles_pipe<T, NZ, kBatchZWarps, false>(a, first, 1, count, smem);
  } else {
    for (int k = 0; k < count; ++k) {
      if (k) __syncthreads();
      if (forward) zfwd_tile<T, NZ, kBatchZWarps, false>(a, first + k, smem);
      else zinv_tile<T, NZ, kBatchZWarps, false>(a, first + k, smem);
    }
  }
}

// a transverse item is `per` consecutive kz planes
template <typename T, int N>
__device__ __noinline__ void t_item(const SolveArgs<T>& a, int item, int per, unsigned char* smem) {
  for (int k = 0; k < per; ++k) {
    const int kz = item * per + k;
    if (kz > a.nz) break;
    if (k) __syncthreads();
    if constexpr (TDstCfg<T, N, kBatchThreads>::smem_bytes() <= kMaxSmem) {
      if (a.sx == 1 && a.sy == 1) {                // cell-centred: the n-point routine
        tdst_plane<T, N, kBatchThreads, false>(a, kz, smem);
        continue;
      }
    }
    tsym_cyc_plane<T, N, kBatchThreads, false>(a, kz, smem);
  }
}

template <typename T>
__device__ void run_item(int stage, const SolveArgs<T>& a, int idx, int per, unsigned char* smem) {
  if (stage == 1) {
    switch (a.nx) {
      case 16: t_item<T, 16>(a, idx, per, smem); break;
      case 32: t_item<T, 32>(a, idx, per, smem); break;
      case 64: t_item<T, 64>(a, idx, per, smem); break;
      case 128: t_item<T, 128>(a, idx, per, smem); break;
      default: break;
    }
    return;
  }
  const bool fwd = (stage == 0);
  switch (a.nz) {
    case 32: z_item<T, 32>(fwd, a, idx, per, smem); break;
    case 64: z_item<T, 64>(fwd, a, idx, per, smem); break;
    case 128: z_item<T, 128>(fwd, a, idx, per, smem); break;
    case 256: z_item<T, 256>(fwd, a, idx, per, smem); break;
    case 512: z_item<T, 512>(fwd, a, idx, per, smem); break;
    case 1024: z_item<T, 1024>(fwd, a, idx, per, smem); break;
    default: break;
  }
}

template <typename T>
__global__ void __launch_bounds__(kBatchThreads, 1) batched_kernel(BatchParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_item;
  __shared__ int s_ok;
  __shared__ int s_next;
  __shared__ int2 s_desc, s_next_desc;
  if (threadIdx.x == 0) {
    s_item = atomicAdd(p.counter, 1);
    if (s_item < p.total) s_desc = p.items[s_item];
  }
  __syncthreads();
  for (;;) {
    const int it = s_item;
    if (it >= p.total) return;
    const int2 d = s_desc;
    // claim the next item (and fetch its descriptor) now: the latency of the
    // atomic and of the load overlaps this item's work
    if (threadIdx.x == 0) {
      const int nx = atomicAdd(p.counter, 1);
      s_next = nx;
      if (nx < p.total) s_next_desc = p.items[nx];
    }
    const int s = d.x, stage = d.y >> 24, idx = d.y & 0xffffff;
    if (threadIdx.x == 0) {
      int ok = (stage != p.drop_stage);
      if (ok && stage > 0) {
        const int need = (stage == 1) ? p.need[s].x : p.need[s].y;
        const int* flag = &p.done[2 * s + stage - 1];
        long long polls = 0;
        while (ld_acquire(flag) < need) {
          if (ld_acquire(p.status) != PIPE_OK || ++polls > p.spin_limit) {
            atomicCAS(p.status, PIPE_OK, PIPE_ETIMEOUT);
            ok = 0;
            break;
          }
          __nanosleep(200);
        }
      }
      s_ok = ok;
    }
    __syncthreads();
    if (s_ok) {
      SolveArgs<T> a = p.solves[s];
      a.rho = p.rho[s];
      a.phi = p.phi[s];
      run_item<T>(stage, a, idx, stage == 1 ? p.per[s].y : p.per[s].x, smem_raw);
      __syncthreads();
      if (threadIdx.x == 0 && stage < 2) {
        __threadfence();
        atomicAdd(&p.done[2 * s + stage], 1);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      s_item = s_next;
      s_desc = s_next_desc;
    }
    __syncthreads();
  }
}

// shared memory of the persistent CTA: the largest item routine of the batch
template <typename T>
size_t item_smem(int nx, int nz) {
  size_t z = 0, t = 0;
  auto zs = [](auto cfg, bool pipe) {
    using C = decltype(cfg);
    if (!pipe) return C::smem_bytes();
    return C::fwd_pipe_smem() > C::inv_pipe_smem() ? C::fwd_pipe_smem() : C::inv_pipe_smem();
  };
  switch (nz) {
    case 32: z = zs(ZCfg<T, 32, kBatchZWarps>{}, z_pipe_fits<T, 32>()); break;
    case 64: z = zs(ZCfg<T, 64, kBatchZWarps>{}, z_pipe_fits<T, 64>()); break;
    case 128: z = zs(ZCfg<T, 128, kBatchZWarps>{}, z_pipe_fits<T, 128>()); break;
    case 256: z = zs(ZCfg<T, 256, kBatchZWarps>{}, z_pipe_fits<T, 256>()); break;
    case 512: z = zs(ZCfg<T, 512, kBatchZWarps>{}, z_pipe_fits<T, 512>()); break;
    case 1024: z = zs(ZCfg<T, 1024, kBatchZWarps>{}, z_pipe_fits<T, 1024>()); break;
  }
  auto ts = [](auto cyc, auto dst) {
    using C = decltype(cyc);
    using D = decltype(dst);
    const size_t d = D::smem_bytes() <= kMaxSmem ? D::smem_bytes() : 0;
    return C::smem_bytes() > d ? C::smem_bytes() : d;
  };
  switch (nx) {
    case 16: t = ts(TCycCfg<T, 16, kBatchThreads>{}, TDstCfg<T, 16, kBatchThreads>{}); break;
    case 32: t = ts(TCycCfg<T, 32, kBatchThreads>{}, TDstCfg<T, 32, kBatchThreads>{}); break;
    case 64: t = ts(TCycCfg<T, 64, kBatchThreads>{}, TDstCfg<T, 64, kBatchThreads>{}); break;
    case 128: t = ts(TCycCfg<T, 128, kBatchThreads>{}, TDstCfg<T, 128, kBatchThreads>{}); break;
  }
  return z > t ? z : t;
}

template <typename T>
int z_cols(int nz) {
  switch (nz) {
    case 32: return ZCfg<T, 32, kBatchZWarps>::COLS;
    case 64: return ZCfg<T, 64, kBatchZWarps>::COLS;
    case 128: return ZCfg<T, 128, kBatchZWarps>::COLS;
    case 256: return ZCfg<T, 256, kBatchZWarps>::COLS;
    case 512: return ZCfg<T, 512, kBatchZWarps>::COLS;
    case 1024: return ZCfg<T, 1024, kBatchZWarps>::COLS;
  }
  return 0;
}

// FP32 mode-form solves outside the persistent launch that share a shape and
// a y-mode table: one launch per stage for all of them (ModeGroup), the same
// kernels and arithmetic per solve as their single-solve launches
struct MGroup {
  std::vector<int> members;            // indices into the handle set
  ModeArgs<float>* dargs = nullptr;    // [members] in device memory: tables and scratch
  ModeArgs<float> a0{};                // the shape (members[0]'s arguments)
  int myp = 0;
  int zgroups = 0;                     // partial projections the z stage sums
  const float* sy = nullptr;           // the shared y-mode table (host copy)
};

// One way of running a handle set: the solves in the persistent launch
// ("members", with their work lists) and the solves left to their own
// single-solve launches ("outside").
struct BatchVariant {
  std::vector<int> members;
  std::vector<int> outside;
  int n = 0;                 // members.size()
  void* solves = nullptr;    // SolveArgs<T>[n]
  int2* lists[3] = {nullptr, nullptr, nullptr};   // candidate work lists
  int2* items = nullptr;     // the chosen one
  int2* need = nullptr;
  int2* per = nullptr;
  int* words = nullptr;      // done[2n], counter, status
  int total = 0;
  size_t smem = 0;
  int grid = 0;
  int order = 0;
  std::vector<MGroup> mgroups;   // groups among `outside` (two or more solves each)
};

// Built and timed on the first call for a handle set, kept by handles[0].
struct BatchPlan {
  int n = 0;
  int dtype = 0;
  pipe_handle* handles[kMaxBatch] = {};
  // variant k: the solves whose z spectrum is smaller than the k-th largest
  // spectrum size in the set run persistent, the others outside (k = 0: all
  // persistent; the last variant may have none persistent)
  static constexpr int kMaxVar = 5;
  BatchVariant var[kMaxVar];
  int nvar = 0;
  int chosen = 0;
  int last = 0;              // variant of the last call (its status word is read back)
  bool tuned = false;
  int drop_stage = -1;          // fault injection for the next launch only
  long long spin_limit = 1ll << 22;
  // the outside solves on nside (2 or 3) side streams, forked from and joined
  // back to the caller's stream by events (parallel branches when captured in
  // a graph); nside = 0 runs them in order on the caller's stream
  static constexpr int kSide = 3;
  cudaStream_t side[kSide] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kSide] = {};
  int nside = 0;
  int group = 0;                // the mode-form groups launched together (1) or solve by solve (0)
};

// the side streams and their events, created on first use
int side_streams(BatchPlan* b) {
  if (b->fork) return PIPE_OK;
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) return PIPE_ECUDA;
  for (int i = 0; i < BatchPlan::kSide; ++i) {
    if (cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking) != cudaSuccess) return PIPE_ECUDA;
    if (cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) != cudaSuccess) return PIPE_ECUDA;
  }
  return PIPE_OK;
}

void variant_release(BatchVariant& v) {
  for (MGroup& g : v.mgroups) cudaFree(g.dargs);
  cudaFree(v.solves);
  for (int k = 0; k < 3; ++k) cudaFree(v.lists[k]);
  cudaFree(v.need);
  cudaFree(v.per);
  cudaFree(v.words);
  v = BatchVariant();
}

void batch_release(pipe_handle* h) {
  if (!h || !h->batch) return;
  BatchPlan* b = static_cast<BatchPlan*>(h->batch);
  for (int k = 0; k < BatchPlan::kMaxVar; ++k) variant_release(b->var[k]);
  for (int i = 0; i < BatchPlan::kSide; ++i) {
    if (b->side[i]) cudaStreamDestroy(b->side[i]);
    if (b->join[i]) cudaEventDestroy(b->join[i]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
  h->batch = nullptr;
}

template <typename T>
SolveArgs<T> batch_args(pipe_handle* h);
template <>
SolveArgs<float> batch_args<float>(pipe_handle* h) {
  SolveArgs<float> a{};
  a.work = static_cast<float2*>(h->work); a.green = h->green32;
  a.tw_t = h->tw_t32; a.w2_t = h->w2_t32; a.tw_z = h->tw_z32; a.w2_z = h->w2_z32; a.tw_t2 = h->tw_t2_32;
  a.tw_t2c = h->tw_t2c_32;
  a.nx = h->grid.nx; a.ny = h->grid.ny; a.nz = h->grid.nz;
  a.sx = h->sx; a.sy = h->sy; a.images = h->images;
  return a;
}
template <>
SolveArgs<double> batch_args<double>(pipe_handle* h) {
  SolveArgs<double> a{};
  a.work = static_cast<double2*>(h->work); a.green = h->green64;
  a.tw_t = h->tw_t64; a.w2_t = h->w2_t64; a.tw_z = h->tw_z64; a.w2_z = h->w2_z64; a.tw_t2 = h->tw_t2_64;
  a.tw_t2c = h->tw_t2c_64;
  a.tbuf = static_cast<double2*>(h->tbuf);
  a.nx = h->grid.nx; a.ny = h->grid.ny; a.nz = h->grid.nz;
  a.sx = h->sx; a.sy = h->sy; a.images = h->images;
  return a;
}

// Work lists.  z items group tiles so that a solve has at most about 256 of
// them; transverse items group small planes.  Three orders are built and
// the first launch times each and keeps the fastest (the autotuner's choice
// for this handle set):
//   0 stage-major: every z-forward item, then every transverse item, then
//     every z-inverse item (solves largest first within a stage);
//   1 pipelined: wave w holds the z-forward items of solve w, the transverse
//     items of solve w-2 and the z-inverse items of solve w-4, so that
//     memory-bound and compute-bound items run at the same time;
//   2 L2-local: solves whose z spectrum is a sizeable part of L2 run stage
//     after stage, one at a time, so the spectrum stays in L2 between
//     stages; the small solves (pipelined among themselves) fill the gaps.
// In every order an item appears after all items it waits for.
template <typename T>
int build_variant(pipe_handle* const* all, BatchVariant* b) {
  const int n = b->n;
  std::vector<pipe_handle*> hs(n);
  for (int s = 0; s < n; ++s) hs[s] = all[b->members[s]];
  std::vector<SolveArgs<T>> solves(n);
  std::vector<int2> need(n);
  std::vector<int2> per(n);
  std::vector<int> order(n);
  size_t smem = 0;
  for (int s = 0; s < n; ++s) {
    solves[s] = batch_args<T>(hs[s]);
    const int nt = hs[s]->grid.nx * hs[s]->grid.ny / z_cols<T>(hs[s]->grid.nz);
    const int nx = hs[s]->grid.nx, planes = hs[s]->grid.nz + 1;
    const int pz = nt > 256 ? nt / 256 : 1;
    const int pt = nx >= 128 ? 1 : (nx >= 64 ? 2 : 8);   // about the work of a 128^2 plane
    per[s] = make_int2(pz, pt);
    need[s] = make_int2((nt + pz - 1) / pz, (planes + pt - 1) / pt);
    const size_t m = item_smem<T>(hs[s]->grid.nx, hs[s]->grid.nz);
    smem = m > smem ? m : smem;
    order[s] = s;
  }
  auto cost = [&](int s) {
    return double(hs[s]->grid.nx) * hs[s]->grid.ny * hs[s]->grid.nz;
  };
  for (int i = 1; i < n; ++i)            // largest first (stable)
    for (int j = i; j > 0 && cost(order[j]) > cost(order[j - 1]); --j) std::swap(order[j], order[j - 1]);
  auto append = [&](std::vector<int2>& dst, int s, int stage) {
    const int cnt = (stage == 1) ? need[s].y : need[s].x;
    for (int i = 0; i < cnt; ++i) dst.push_back(make_int2(s, (stage << 24) | i));
  };
  auto pipelined = [&](const std::vector<int>& list, std::vector<int2>& dst) {
    constexpr int LAG = 2;
    const int m = int(list.size());
    for (int w = 0; w < m + 2 * LAG; ++w)
      for (int stage = 0; stage < 3; ++stage) {
        const int k = w - LAG * stage;
        if (k >= 0 && k < m) append(dst, list[k], stage);
      }
  };
  std::vector<int2> lists[3];
  for (int stage = 0; stage < 3; ++stage)
    for (int k = 0; k < n; ++k) append(lists[0], order[k], stage);
  pipelined(order, lists[1]);
  {
    const double l2_share = 16.0 * 1024 * 1024;
    std::vector<int> large, small;
    for (int k = 0; k < n; ++k) {
      const int s = order[k];
      const double bytes = double(hs[s]->grid.nx) * hs[s]->grid.ny * (hs[s]->grid.nz + 1) * 2 * sizeof(T);
      (bytes > l2_share ? large : small).push_back(s);
    }
    std::vector<int2> fill;
    pipelined(small, fill);
    const int slots = 3 * int(large.size());
    size_t f = 0;
    for (int k = 0; k < int(large.size()); ++k)
      for (int stage = 0; stage < 3; ++stage) {
        append(lists[2], large[k], stage);
        const size_t until = fill.size() * size_t(3 * k + stage + 1) / size_t(slots);
        for (; f < until; ++f) lists[2].push_back(fill[f]);
      }
    for (; f < fill.size(); ++f) lists[2].push_back(fill[f]);
  }
  std::vector<int2>& items = lists[0];
  b->total = int(items.size());
  b->smem = smem;
  cudaError_t e;
  if ((e = cudaMalloc(&b->solves, sizeof(SolveArgs<T>) * n)) != cudaSuccess) return PIPE_ENOMEM;
  for (int k = 0; k < 3; ++k) {
    if ((e = cudaMalloc(&b->lists[k], sizeof(int2) * items.size())) != cudaSuccess) return PIPE_ENOMEM;
    if (cudaMemcpy(b->lists[k], lists[k].data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return PIPE_ECUDA;
  }
  b->items = b->lists[0];
  if ((e = cudaMalloc(&b->need, sizeof(int2) * n)) != cudaSuccess) return PIPE_ENOMEM;
  if ((e = cudaMalloc(&b->per, sizeof(int2) * n)) != cudaSuccess) return PIPE_ENOMEM;
  if ((e = cudaMalloc(&b->words, sizeof(int) * (2 * n + 2))) != cudaSuccess) return PIPE_ENOMEM;
  if (cudaMemcpy(b->solves, solves.data(), sizeof(SolveArgs<T>) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->need, need.data(), sizeof(int2) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->per, per.data(), sizeof(int2) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(b->words, 0, sizeof(int) * (2 * n + 2)) != cudaSuccess)
    return PIPE_ECUDA;
  if (smem > kMaxSmem) return PIPE_EUNSUPPORTED;
  // the attribute belongs to the kernel, shared by every plan: only raise it
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, batched_kernel<T>) != cudaSuccess) return PIPE_ECUDA;
  if (int(smem) > fa.maxDynamicSharedSizeBytes &&
      cudaFuncSetAttribute(batched_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) !=
          cudaSuccess)
    return PIPE_ECUDA;
  int per_sm = 0, sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_kernel<T>, kBatchThreads, smem) !=
          cudaSuccess || per_sm < 1)
    return PIPE_ECUDA;
  b->grid = sms * per_sm;
  return PIPE_OK;
}

template <typename T>
int launch_variant(BatchVariant* b, const void* const* rho, void* const* phi, int drop_stage,
                   long long spin_limit, cudaStream_t st) {
  BatchParams<T> p;
  p.solves = static_cast<const SolveArgs<T>*>(b->solves);
  p.items = b->items;
  p.need = b->need;
  p.per = b->per;
  p.done = b->words;
  p.counter = b->words + 2 * b->n;
  p.status = b->words + 2 * b->n + 1;
  p.total = b->total;
  p.n = b->n;
  p.spin_limit = spin_limit;         // default 2^22 polls of >= 200 ns: about a second
  p.drop_stage = drop_stage;
  for (int s = 0; s < b->n; ++s) {
    p.rho[s] = static_cast<const T*>(rho[b->members[s]]);
    p.phi[s] = static_cast<T*>(phi[b->members[s]]);
  }
  for (int s = b->n; s < kMaxBatch; ++s) {
    p.rho[s] = nullptr;
    p.phi[s] = nullptr;
  }
  if (b->n > 0) {
    if (cudaMemsetAsync(b->words, 0, sizeof(int) * (2 * b->n + 2), st) != cudaSuccess) return PIPE_ECUDA;
    batched_kernel<T><<<b->grid, kBatchThreads, b->smem, st>>>(p);
    if (cudaGetLastError() != cudaSuccess) return PIPE_ECUDA;
  }
  return PIPE_OK;
}

// spectrum bytes of a solve (the "large" solves are those whose spectrum is a
// sizeable part of L2; candidates for their own launches)
static double spectrum_bytes(const pipe_handle* h) {
  return double(h->grid.nx) * h->grid.ny * (h->grid.nz + 1) * (h->grid.dtype == PIPE_F64 ? 16 : 8);
}

// the groups of a variant's outside solves: FP32 mode-form solves with the
// occupancy-laid-out kernels, of one shape and one y-mode table, up to
// kMaxModeGroup each; only groups of two or more are kept
static bool mode_groupable(const pipe_handle* h) {
  return h->grid.dtype == PIPE_F32 && h->use_modes && h->mfast && h->banded < 0 && h->msy_host;
}
static bool same_mode_shape(const pipe_handle* a, const pipe_handle* b) {
  if (a->grid.nx != b->grid.nx || a->grid.ny != b->grid.ny || a->grid.nz != b->grid.nz ||
      a->geom.modes_m != b->geom.modes_m || a->mxp != b->mxp || a->myp != b->myp || a->fy != b->fy)
    return false;
  const size_t nsy = size_t(a->grid.ny / 2) * a->myp;
  return std::memcmp(a->msy_host, b->msy_host, nsy * sizeof(float)) == 0;
}
static int build_mode_groups(pipe_handle* const* hs, BatchVariant* v) {
  std::vector<MGroup> gs;
  for (int s : v->outside) {
    if (!mode_groupable(hs[s])) continue;
    MGroup* into = nullptr;
    for (MGroup& g : gs)
      if (int(g.members.size()) < kMaxModeGroup && same_mode_shape(hs[g.members[0]], hs[s])) { into = &g; break; }
    if (!into) {
      gs.emplace_back();
      into = &gs.back();
    }
    into->members.push_back(s);
  }
  for (MGroup& g : gs) {
    if (g.members.size() < 2) continue;
    const pipe_handle* h0 = hs[g.members[0]];
    std::vector<ModeArgs<float>> args;
    for (int s : g.members) args.push_back(mode_args_f32(hs[s]));
    g.a0 = args[0];
    g.myp = h0->myp;
    g.zgroups = mode_xblocks(h0);
    g.sy = h0->msy_host;
    if (cudaMalloc(&g.dargs, sizeof(ModeArgs<float>) * args.size()) != cudaSuccess) return PIPE_ENOMEM;
    if (cudaMemcpy(g.dargs, args.data(), sizeof(ModeArgs<float>) * args.size(), cudaMemcpyHostToDevice) !=
        cudaSuccess) {
      cudaFree(g.dargs);
      return PIPE_ECUDA;
    }
    v->mgroups.push_back(g);
  }
  return PIPE_OK;
}

// the three stages of one mode group on stream st
static int run_mode_group(const MGroup& g, const void* const* rho, void* const* phi, cudaStream_t st) {
  ModeGroup p{};
  p.args = g.dargs;
  p.n = int(g.members.size());
  p.nz = g.a0.nz;
  for (int i = 0; i < p.n; ++i) {
    p.rho[i] = static_cast<const float*>(rho[g.members[i]]);
    p.phi[i] = static_cast<float*>(phi[g.members[i]]);
  }
  cudaError_t e = launch_mode_fast_group(0, g.myp, g.a0, p, g.sy, st);
  if (e == cudaSuccess) e = launch_mode_z_warp_group(g.a0, g.zgroups, p, st);
  if (e == cudaSuccess) e = launch_mode_fast_group(2, g.myp, g.a0, p, g.sy, st);
  return e == cudaSuccess ? PIPE_OK : PIPE_ECUDA;
}

template <typename T>
static int build_plan(pipe_handle* const* hs, int n, BatchPlan* b) {
  std::vector<double> sizes;
  for (int s = 0; s < n; ++s) sizes.push_back(spectrum_bytes(hs[s]));
  std::sort(sizes.begin(), sizes.end(), [](double x, double y) { return x > y; });
  sizes.erase(std::unique(sizes.begin(), sizes.end()), sizes.end());
  // cut-offs: none, then each distinct size from the largest down
  const int ncut = std::min(int(sizes.size()) + 1, BatchPlan::kMaxVar);
  for (int k = 0; k < ncut; ++k) {
    BatchVariant& v = b->var[k];
    for (int s = 0; s < n; ++s)
      (k > 0 && spectrum_bytes(hs[s]) >= sizes[k - 1] ? v.outside : v.members).push_back(s);
    v.n = int(v.members.size());
    if (v.n > 0) {
      const int st = build_variant<T>(hs, &v);
      if (st != PIPE_OK) return st;
    }
    if (sizeof(T) == 4) {
      const int st = build_mode_groups(hs, &v);
      if (st != PIPE_OK) return st;
    }
    b->nvar = k + 1;
  }
  return PIPE_OK;
}

// one batched call with variant v: the persistent launch and the solves
// outside it.  nside = 0: all in order on stream st.  Otherwise the side
// streams fork from st, the persistent launch takes side stream 0 and the
// outside solves are dealt round-robin to the side streams after it, so that
// they run beside it; the side streams rejoin st.  (A persistent item waits
// only for items handed out before it, which running CTAs hold, so kernels
// beside it cannot stall it.)  With grp, each mode group's three launches
// take one slot of that order.
static int run_variant(BatchPlan* b, int v, int nside, int grp, pipe_handle* const* hs, const void* const* rho,
                       void* const* phi, cudaStream_t st) {
  BatchVariant& x = b->var[v];
  auto persistent = [&](cudaStream_t s) {
    return b->dtype == PIPE_F64 ? launch_variant<double>(&x, rho, phi, b->drop_stage, b->spin_limit, s)
                                : launch_variant<float>(&x, rho, phi, b->drop_stage, b->spin_limit, s);
  };
  int r = PIPE_OK;
  if (nside == 0 || x.outside.empty()) {
    r = persistent(st);
    if (r != PIPE_OK || x.outside.empty()) return r;
  }
  std::vector<char> grouped(b->n, 0);
  if (grp)
    for (const MGroup& g : x.mgroups)
      for (int s : g.members) grouped[s] = 1;
  if (nside == 0) {
    if (grp)
      for (size_t k = 0; r == PIPE_OK && k < x.mgroups.size(); ++k) r = run_mode_group(x.mgroups[k], rho, phi, st);
    for (size_t k = 0; r == PIPE_OK && k < x.outside.size(); ++k) {
      const int s = x.outside[k];
      if (!grouped[s]) r = handle_solve(hs[s], rho[s], phi[s], false, st);
    }
    return r;
  }
  if ((r = side_streams(b)) != PIPE_OK) return r;
  if (cudaEventRecord(b->fork, st) != cudaSuccess) return PIPE_ECUDA;
  for (int i = 0; i < nside; ++i)
    if (cudaStreamWaitEvent(b->side[i], b->fork, 0) != cudaSuccess) return PIPE_ECUDA;
  size_t slot = 0;
  if (x.n > 0) {
    r = persistent(b->side[0]);
    slot = 1;
  }
  if (grp)
    for (size_t k = 0; r == PIPE_OK && k < x.mgroups.size(); ++k)
      r = run_mode_group(x.mgroups[k], rho, phi, b->side[slot++ % nside]);
  for (size_t k = 0; r == PIPE_OK && k < x.outside.size(); ++k) {
    const int s = x.outside[k];
    if (!grouped[s]) r = handle_solve(hs[s], rho[s], phi[s], false, b->side[slot++ % nside]);
  }
  // rejoin even after an error, so that a capture is never left unjoined
  for (int i = 0; i < nside; ++i) {
    if (cudaEventRecord(b->join[i], b->side[i]) != cudaSuccess) return PIPE_ECUDA;
    if (cudaStreamWaitEvent(st, b->join[i], 0) != cudaSuccess) return PIPE_ECUDA;
  }
  return r;
}

}  // namespace pp

using namespace pp;

extern "C" int pipe_poisson_solve_batched(pipe_handle* const* handles, const void* const* rho,
                                          void* const* phi, int n, void* stream) {
  if (!handles || !rho || !phi || n < 1) return PIPE_EINVAL;
  if (n > kMaxBatch) return PIPE_EUNSUPPORTED;
  for (int s = 0; s < n; ++s) {
    if (!handles[s] || !rho[s] || !phi[s]) return PIPE_EINVAL;
    if ((reinterpret_cast<uintptr_t>(rho[s]) | reinterpret_cast<uintptr_t>(phi[s])) % 16) return PIPE_EINVAL;
    if (handles[s]->grid.dtype != handles[0]->grid.dtype || handles[s]->device != handles[0]->device ||
        !handles[s]->images || handles[s]->banded >= 0 || handles[s]->general || !handles[s]->fft_ok ||
        handles[s]->grid.dtype == PIPE_F32_C16)
      return PIPE_EUNSUPPORTED;
    for (int r = 0; r < s; ++r)
      if (handles[r] == handles[s]) return PIPE_EINVAL;      // workspaces would collide
  }
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != handles[0]->device) cudaSetDevice(handles[0]->device);
  BatchPlan* b = static_cast<BatchPlan*>(handles[0]->batch);
  bool same = b && b->n == n;
  for (int s = 0; same && s < n; ++s) same = (b->handles[s] == handles[s]);
  int st = PIPE_OK;
  if (!same) {
    batch_release(handles[0]);
    b = new (std::nothrow) BatchPlan();
    if (!b) st = PIPE_ENOMEM;
    if (st == PIPE_OK) {
      b->n = n;
      b->dtype = handles[0]->grid.dtype;
      for (int s = 0; s < n; ++s) b->handles[s] = handles[s];
      handles[0]->batch = b;
      st = b->dtype == PIPE_F64 ? build_plan<double>(handles, n, b) : build_plan<float>(handles, n, b);
      // the side streams exist before any later call can be captured
      if (st == PIPE_OK) st = side_streams(b);
      if (st != PIPE_OK) batch_release(handles[0]);
    }
  }
  if (st == PIPE_OK) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!b->tuned) {
      // time every (variant, work-list order) once after a warm-up run and
      // keep the fastest; these runs are valid solves
      float best = 1e30f;
      int pick_v = 0, pick_o = 0, pick_s = 0, pick_g = 0;
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      for (int v = 0; v < b->nvar && st == PIPE_OK; ++v)
        for (int k = 0; k < (b->var[v].n > 0 ? 3 : 1) && st == PIPE_OK; ++k)
          for (int ns : {0, 2, 3})
            for (int grp = 0; grp < (b->var[v].mgroups.empty() ? 1 : 2); ++grp) {
              if (ns > 0 && b->var[v].outside.size() < size_t(ns)) continue;
              if (st != PIPE_OK) break;
              b->var[v].items = b->var[v].lists[k];
              st = run_variant(b, v, ns, grp, handles, rho, phi, s);
              cudaEventRecord(e0, s);
              if (st == PIPE_OK) st = run_variant(b, v, ns, grp, handles, rho, phi, s);
              cudaEventRecord(e1, s);
              cudaEventSynchronize(e1);
              float ms = 0.f;
              cudaEventElapsedTime(&ms, e0, e1);
              if (st == PIPE_OK && ms < best) { best = ms; pick_v = v; pick_o = k; pick_s = ns; pick_g = grp; }
            }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      for (int v = 0; v < b->nvar; ++v) {
        b->var[v].order = (v == pick_v) ? pick_o : 0;
        b->var[v].items = b->var[v].lists[b->var[v].order];
      }
      b->chosen = pick_v;
      b->nside = pick_s;
      b->group = pick_g;
      b->tuned = true;
    }
    // an injected fault is meant for the persistent launch: run every solve there
    const int v = b->drop_stage >= 0 ? 0 : b->chosen;
    if (st == PIPE_OK) st = run_variant(b, v, b->nside, b->group, handles, rho, phi, s);
    b->last = v;
    b->drop_stage = -1;
    b->spin_limit = 1ll << 22;
  }
  if (cur >= 0 && cur != handles[0]->device) cudaSetDevice(cur);
  return st;
}

extern "C" int pipe_batch_status(pipe_handle* const* handles, int n) {
  if (!handles || n < 1 || !handles[0]) return PIPE_EINVAL;
  BatchPlan* b = static_cast<BatchPlan*>(handles[0]->batch);
  if (!b || b->n != n) return PIPE_EINVAL;
  const BatchVariant& x = b->var[b->last];
  if (x.n == 0) return PIPE_OK;
  int status = PIPE_OK;
  if (cudaMemcpy(&status, x.words + 2 * x.n + 1, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return PIPE_ECUDA;
  return status;
}

extern "C" int pipe_batch_inject_fault(pipe_handle* const* handles, int n, int drop_stage,
                                       long long spin_limit) {
  if (!handles || n < 1 || !handles[0] || drop_stage < 0 || drop_stage > 2 || spin_limit < 0)
    return PIPE_EINVAL;
  BatchPlan* b = static_cast<BatchPlan*>(handles[0]->batch);
  if (!b || b->n != n || !b->tuned) return PIPE_EINVAL;
  for (int s = 0; s < n; ++s)
    if (b->handles[s] != handles[s]) return PIPE_EINVAL;
  b->drop_stage = drop_stage;
  b->spin_limit = spin_limit;
  return PIPE_OK;
}

extern "C" int pipe_batch_plan_info(pipe_handle* const* handles, int n, int* persistent, int* order) {
  if (!handles || n < 1 || !handles[0] || !persistent || !order) return PIPE_EINVAL;
  BatchPlan* b = static_cast<BatchPlan*>(handles[0]->batch);
  if (!b || b->n != n || !b->tuned) return PIPE_EINVAL;
  for (int s = 0; s < n; ++s)
    if (b->handles[s] != handles[s]) return PIPE_EINVAL;
  *persistent = b->var[b->chosen].n;
  *order = b->var[b->chosen].order;
  return PIPE_OK;
}

extern "C" int pipe_batch_side_streams(pipe_handle* const* handles, int n, int* nside) {
  if (!handles || n < 1 || !handles[0] || !nside) return PIPE_EINVAL;
  BatchPlan* b = static_cast<BatchPlan*>(handles[0]->batch);
  if (!b || b->n != n || !b->tuned) return PIPE_EINVAL;
  for (int s = 0; s < n; ++s)
    if (b->handles[s] != handles[s]) return PIPE_EINVAL;
  *nside = b->nside;
  return PIPE_OK;
}

extern "C" int pipe_batch_select_streams(pipe_handle* const* handles, int n, int nside) {
  if (!handles || n < 1 || !handles[0] || (nside != 0 && nside != 2 && nside != 3)) return PIPE_EINVAL;
  BatchPlan* b = static_cast<BatchPlan*>(handles[0]->batch);
  if (!b || b->n != n || !b->tuned) return PIPE_EINVAL;
  for (int s = 0; s < n; ++s)
    if (b->handles[s] != handles[s]) return PIPE_EINVAL;
  b->nside = nside;
  return PIPE_OK;
}

extern "C" int pipe_batch_grouped(pipe_handle* const* handles, int n, int* grouped, int* groups) {
  if (!handles || n < 1 || !handles[0] || !grouped) return PIPE_EINVAL;
  BatchPlan* b = static_cast<BatchPlan*>(handles[0]->batch);
  if (!b || b->n != n || !b->tuned) return PIPE_EINVAL;
  for (int s = 0; s < n; ++s)
    if (b->handles[s] != handles[s]) return PIPE_EINVAL;
  int k = 0, ng = 0;
  if (b->group)
    for (const MGroup& g : b->var[b->chosen].mgroups) {
      k += int(g.members.size());
      ++ng;
    }
  *grouped = k;
  if (groups) *groups = ng;
  return PIPE_OK;
}

extern "C" int pipe_batch_select_groups(pipe_handle* const* handles, int n, int on) {
  if (!handles || n < 1 || !handles[0] || (on != 0 && on != 1)) return PIPE_EINVAL;
  BatchPlan* b = static_cast<BatchPlan*>(handles[0]->batch);
  if (!b || b->n != n || !b->tuned) return PIPE_EINVAL;
  for (int s = 0; s < n; ++s)
    if (b->handles[s] != handles[s]) return PIPE_EINVAL;
  b->group = on;
  return PIPE_OK;
}

extern "C" int pipe_batch_select(pipe_handle* const* handles, int n, int variant, int order) {
  if (!handles || n < 1 || !handles[0]) return PIPE_EINVAL;
  BatchPlan* b = static_cast<BatchPlan*>(handles[0]->batch);
  if (!b || b->n != n || !b->tuned) return PIPE_EINVAL;
  for (int s = 0; s < n; ++s)
    if (b->handles[s] != handles[s]) return PIPE_EINVAL;
  if (variant < 0 || variant >= b->nvar || order < 0 || order > 2) return PIPE_EINVAL;
  BatchVariant& v = b->var[variant];
  if (v.n == 0 && order != 0) return PIPE_EINVAL;
  v.order = order;
  if (v.n > 0) v.items = v.lists[order];
  b->chosen = variant;
  return PIPE_OK;
}
