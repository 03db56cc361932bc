// Banded z reduction of the pipe solve (Sec. 5, Eq. 17-18): when the Green
// function falls off within n_nb z planes, each output plane k is the sum over
// d = -n_nb..n_nb of a 2-D mixed convolution/correlation of source plane k-d
// with the R table at z-offset d*hz.  No transform along z is taken.
//
// Cell-centred meshes (s = 2 x0 / h = 1).  In the n-point sine form of the
// transverse stage (tdst_impl.cuh) the 2-D operator of offset d is diagonal:
// a real plane x has transverse coefficients U(kx,ky) = c(kx) c(ky) D(kx,ky)
// with D real and c(q) = 2i e^{i pi q / 2N}, and the operator multiplies by
// the real 2-D spectrum g_d(kx,ky) (the octant of the offset-d table, scaled
// by hx hy hz / (4 nx ny)).  So
//     pair_transpose: rho [nx*ny][nz] viewed as pairs (rho_2m, rho_2m+1) ->
//       pair-major planes C[m][i][j] (one complex value per node), so that
//       the transverse passes read and write whole contiguous planes;
//     banded_fwd_kernel: plane m of C (rho_2m + i rho_2m+1), rows along y,
//       columns along x, divided by c(kx) c(ky): the packed real coefficients
//       D_2m + i D_2m+1, stored [m][ky-1][kx slot];
//     banded_inv_kernel: for output planes 2m, 2m+1 the stencil
//       E_k = sum_d g_|d| D_{k-d} (source planes inside 0..nz-1), multiplied
//       by c(kx) c(ky), inverse along x, inverse along y: phi_2m + i phi_2m+1
//       into plane m of C, transposed back into phi.
// Workspace: D in the first nz/2 planes of `work`, C in the next nz/2.
// The banded operator is symmetric (G even in z and reciprocal), so the
// adjoint is the same computation.
#include "tdst_impl.cuh"

namespace pp {

namespace {

// c(q) for the kx / ky slots (slot 0 carries q = N)
template <typename T, int N, int THREADS>
__device__ __forceinline__ void load_phase(C2<T>* ctab) {
  for (int s = threadIdx.x; s < N; s += THREADS) {
    const int q = s == 0 ? N : s;
    T sn, cs;
    if constexpr (sizeof(T) == 8) sincospi(double(q) / double(2 * N), &sn, &cs);
    else sincospif(float(q) / float(2 * N), &sn, &cs);
    ctab[s] = mk<C2<T>>(T(-2) * sn, T(2) * cs);                // 2i (cos + i sin)
  }
}

// out[c][r] = in[r][c] for a rows x cols matrix of complex values (32 x 32
// tiles through shared memory, both sides coalesced)
template <typename V>
__global__ void __launch_bounds__(256) pair_transpose(const V* __restrict__ in, V* __restrict__ out,
                                                      int rows, int cols) {
  __shared__ V tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
  for (int k = ty; k < 32; k += 8) {
    const int r = r0 + k, c = c0 + tx;
    if (r < rows && c < cols) tile[k][tx] = in[size_t(r) * cols + c];
  }
  __syncthreads();
#pragma unroll
  for (int k = ty; k < 32; k += 8) {
    const int c = c0 + k, r = r0 + tx;
    if (c < cols && r < rows) out[size_t(c) * rows + r] = tile[tx][k];
  }
}

template <typename T, int N, int THREADS>
constexpr size_t banded_smem() {
  return TDstCfg<T, N, THREADS>::smem_bytes() + sizeof(C2<T>) * N;
}

template <typename T, int N, int THREADS>
__global__ void __launch_bounds__(THREADS, 1) banded_fwd_kernel(SolveArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using R = TDst<T, N, THREADS, false>;
  using V = C2<T>;
  constexpr int G = R::G, E = R::E, H = R::H, GPC = R::GPC, MASK = R::MASK, SGN = R::SGN;
  R r(a, smem_raw);
  V* ctab = reinterpret_cast<V*>(smem_raw + TDstCfg<T, N, THREADS>::smem_bytes());
  const int m = blockIdx.x;                                    // planes 2m, 2m+1
  const int nz = a.nz;
  r.load_tables(a);
  load_phase<T, N, THREADS>(ctab);
  __syncthreads();

  // rows i along y: the packed pair (rho_2m + i rho_2m+1) of plane m of C
  const V* cplane = a.work + (size_t(nz / 2) + m) * N * N;
#pragma unroll 1
  for (int r0 = 0; r0 < N; r0 += GPC) {
    const int il = r0 + r.line;
    V v[E];
    r.load_row(cplane, il, v);
    group_fft<N, false>(v, r.scratch, r.tw, r.t);
    V mm[E];
    mirror_fetch<N>(v, mm, r.t, 0, r.lane - r.t);
    if (il < N) {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int q = r.t + G * e;
        if (q == 0) r.ybuf[R::tile(N, il)] = mk<V>(v[e].x + v[e].x, v[e].y + v[e].y);
        else r.ybuf[R::tile(q, il)] = cfms(v[e], r.sw2[(SGN * q) & MASK], mm[e]);
      }
    }
  }
  __syncthreads();

  // columns ky along x, then divide by c(kx) c(ky): D_2m + i D_2m+1
#pragma unroll 1
  for (int c0 = 0; c0 < N; c0 += GPC) {
    const int cl = c0 + r.line;
    const bool act = cl < N;
    const int ky = 1 + (act ? cl : 0);
    V u[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int n = r.t + G * e;
      if (e < H) {
        u[e] = r.ybuf[R::tile(ky, 2 * n)];
      } else {
        const V x = r.ybuf[R::tile(ky, 2 * N - 1 - 2 * n)];
        u[e] = mk<V>(-x.x, -x.y);
      }
    }
    group_fft<N, false>(u, r.scratch, r.tw, r.t);
    V mm[E];
    mirror_fetch<N>(u, mm, r.t, 0, r.lane - r.t);
    const V cy = ctab[ky == N ? 0 : ky];
    V* dst = a.work + (size_t(m) * N + (ky - 1)) * N;
    if (act) {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int s = r.t + G * e;
        const V w = (s == 0) ? mk<V>(u[e].x + u[e].x, u[e].y + u[e].y)
                             : cfms(u[e], r.sw2[(SGN * s) & MASK], mm[e]);
        const V cc = cmul(ctab[s], cy);                        // c(kx) c(ky)
        // w / (c c) = w conj(c c) / |c c|^2, |c c|^2 = 16
        const V d = mk<V>(w.x * cc.x + w.y * cc.y, w.y * cc.x - w.x * cc.y);
        dst[s] = mk<V>(d.x * T(0.0625), d.y * T(0.0625));
      }
    }
  }
}

template <typename T, int N, int THREADS>
__global__ void __launch_bounds__(THREADS, 1) banded_inv_kernel(SolveArgs<T> a, int n_nb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using R = TDst<T, N, THREADS, false>;
  using V = C2<T>;
  constexpr int G = R::G, E = R::E, H = R::H, GPC = R::GPC, MASK = R::MASK, SGN = R::SGN;
  R r(a, smem_raw);
  V* ctab = reinterpret_cast<V*>(smem_raw + TDstCfg<T, N, THREADS>::smem_bytes());
  const int m = blockIdx.x;                                    // output planes 2m, 2m+1
  const int nz = a.nz;
  r.load_tables(a);
  load_phase<T, N, THREADS>(ctab);
  __syncthreads();

  // columns ky: stencil, times c(kx) c(ky), inverse along x
#pragma unroll 1
  for (int c0 = 0; c0 < N; c0 += GPC) {
    const int cl = c0 + r.line;
    const bool act = cl < N;
    const int ky = 1 + (act ? cl : 0);
    const V cy = ctab[ky == N ? 0 : ky];
    T e0[E], e1[E];
#pragma unroll
    for (int e = 0; e < E; ++e) e0[e] = e1[e] = T(0);
    if (act) {
      const T* g0 = a.green + size_t(ky) * (N + 1);
#pragma unroll 1
      for (int d = -n_nb; d <= n_nb; ++d) {
        // source planes k0 = 2m - d (for output 2m) and k0 + 1 (for 2m + 1)
        const int k0 = 2 * m - d;
        const T* grow = g0 + size_t(d < 0 ? -d : d) * (N + 1) * (N + 1);
        if ((k0 & 1) == 0) {                                   // one packed plane holds both
          if (k0 < 0 || k0 >= nz) continue;
          const V* src = a.work + (size_t(k0 >> 1) * N + (ky - 1)) * N;
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int s = r.t + G * e;
            const T g = __ldg(&grow[s == 0 ? N : s]);
            const V dv = src[s];
            e0[e] += g * dv.x;
            e1[e] += g * dv.y;
          }
        } else {                                               // D_k0 = .y of one, D_k0+1 = .x of the next
          const bool v0 = k0 >= 0 && k0 < nz, v1 = k0 + 1 >= 0 && k0 + 1 < nz;
          // (clamped planes are never read: v0 / v1 guard every access)
          const V* s0 = a.work + (size_t(min(max(k0, 0), nz - 1) >> 1) * N + (ky - 1)) * N;
          const V* s1 = a.work + (size_t(min(max(k0 + 1, 0), nz - 1) >> 1) * N + (ky - 1)) * N;
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int s = r.t + G * e;
            const T g = __ldg(&grow[s == 0 ? N : s]);
            if (v0) e0[e] += g * s0[s].y;
            if (v1) e1[e] += g * s1[s].x;
          }
        }
      }
    }
    V u[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const V cc = cmul(ctab[r.t + G * e], cy);
      u[e] = mk<V>(e0[e] * cc.x - e1[e] * cc.y, e0[e] * cc.y + e1[e] * cc.x);   // c c (E_2m + i E_2m+1)
    }
    V mm[E];
    mirror_fetch<N>(u, mm, r.t, 0, r.lane - r.t);              // P(N - kx)
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int q = r.t + G * e;
      if (q != 0) u[e] = cfma_(u[e], r.sw2[(SGN * q) & MASK], mm[e]);
    }
    group_fft<N, true>(u, r.scratch, r.tw, r.t);
    if (act) {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int n = r.t + G * e;
        if (e < H) r.ybuf[R::tile(ky, 2 * n)] = u[e];
        else r.ybuf[R::tile(ky, 2 * N - 1 - 2 * n)] = mk<V>(-u[e].x, -u[e].y);
      }
    }
  }
  __syncthreads();

  // rows i, back along y: (phi[i][j][2m], phi[i][j][2m+1])
#pragma unroll 1
  for (int r0 = 0; r0 < N; r0 += GPC) {
    const int il = r0 + r.line;
    const int i = il < N ? il : 0;
    V u[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int q = r.t + G * e;
      if (q == 0) {
        u[e] = r.ybuf[R::tile(N, i)];
      } else {
        const V p = r.ybuf[R::tile(q, i)];
        const V pm = r.ybuf[R::tile(N - q, i)];
        u[e] = cfma_(p, r.sw2[(SGN * q) & MASK], pm);
      }
    }
    group_fft<N, true>(u, r.scratch, r.tw, r.t);
    if (il < N) {
      V* out = a.work + (size_t(nz / 2) + m) * N * N + size_t(i) * N;   // plane m of C
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int n = r.t + G * e;
        if (e < H) out[2 * n] = u[e];
        else out[2 * N - 1 - 2 * n] = mk<V>(-u[e].x, -u[e].y);
      }
    }
  }
}

template <typename T, int N, int THREADS>
cudaError_t blaunch(const SolveArgs<T>& a, int n_nb, cudaStream_t st) {
  constexpr size_t smem = banded_smem<T, N, THREADS>();
  if constexpr (smem > kMaxSmem) {
    return cudaErrorInvalidConfiguration;
  } else {
    void (*kf)(SolveArgs<T>) = banded_fwd_kernel<T, N, THREADS>;
    void (*ki)(SolveArgs<T>, int) = banded_inv_kernel<T, N, THREADS>;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem))) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(ki, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem))) != cudaSuccess)
      return e;
    using V = C2<T>;
    const int pairs = a.nz / 2, nodes = a.nx * a.ny;
    V* cbuf = a.work + size_t(pairs) * nodes;
    // rho [nodes][pairs] -> C [pairs][nodes]
    pair_transpose<V><<<dim3((pairs + 31) / 32, (nodes + 31) / 32), 256, 0, st>>>(
        reinterpret_cast<const V*>(a.rho), cbuf, nodes, pairs);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    kf<<<pairs, THREADS, smem, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ki<<<pairs, THREADS, smem, st>>>(a, n_nb);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // C [pairs][nodes] -> phi [nodes][pairs]
    pair_transpose<V><<<dim3((nodes + 31) / 32, (pairs + 31) / 32), 256, 0, st>>>(
        cbuf, reinterpret_cast<V*>(a.phi), pairs, nodes);
    return cudaGetLastError();
  }
}

template <typename T, int N>
cudaError_t blaunch2(int threads, const SolveArgs<T>& a, int n_nb, cudaStream_t st) {
  switch (threads) {
    case 128: return blaunch<T, N, 128>(a, n_nb, st);
    case 256: return blaunch<T, N, 256>(a, n_nb, st);
    case 512: return blaunch<T, N, 512>(a, n_nb, st);
    default: return cudaErrorInvalidConfiguration;
  }
}

template <typename T>
cudaError_t launch_banded_t(int threads, const SolveArgs<T>& a, int n_nb, cudaStream_t st) {
  if (a.nx != a.ny || a.sx != 1 || a.sy != 1 || (a.nz & 1) || n_nb < 0 || n_nb >= a.nz)
    return cudaErrorInvalidValue;
  switch (a.nx) {
    case 16: return blaunch2<T, 16>(threads, a, n_nb, st);
    case 32: return blaunch2<T, 32>(threads, a, n_nb, st);
    case 64: return blaunch2<T, 64>(threads, a, n_nb, st);
    case 128: return blaunch2<T, 128>(threads, a, n_nb, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

template <>
cudaError_t launch_banded<float>(int threads, const SolveArgs<float>& a, int n_nb, cudaStream_t st) {
  return launch_banded_t<float>(threads, a, n_nb, st);
}
template <>
cudaError_t launch_banded<double>(int threads, const SolveArgs<double>& a, int n_nb, cudaStream_t st) {
  return launch_banded_t<double>(threads, a, n_nb, st);
}

}  // namespace pp
