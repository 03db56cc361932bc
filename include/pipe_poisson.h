/*
 * pipe_poisson.h -- C ABI of the GB300 open-rectangular-pipe Poisson solver.
 *
 * The solver computes, on a mesh x_i = x0 + i*hx, y_j = y0 + j*hy, z_k = k*hz
 * (i < nx, j < ny, k < nz) inside the pipe (0,a) x (0,b), open in z:
 *
 *     phi_ijk = hx*hy*hz * sum_{i'j'k'} rho_{i'j'k'} G(x_i, x_i', y_j, y_j', z_k - z_k')
 *
 * (the discretised Green-function integral, Sec. 1 Eq. 1 and Eq. 4), with G
 * the pipe Green function of Sec. 2 Eq. 7-9 (ordinary point Green function) or
 * its longitudinally integrated form of Sec. 3 Eq. 15-16 (IGF).  The mode
 * series is truncated at m <= modes_m, n <= modes_n (Sec. 4 uses 20).  G is
 * normalised so that G -> 1/r near the source (series prefactor 8*pi/(a*b) for
 * the sine form, 2*pi/(a*b) for the cosine form R); multiply phi by
 * 1/(4*pi*eps0) for SI units.  A free-space handle (Eq. 3, Eq. 5, the Hockney
 * method) is also provided for comparison.
 *
 * Method (Sec. 2 Eq. 10, Appendix A): zero-padding to (2nx, 2ny, 2nz), FFTs
 * whose direction is chosen per dimension so that x and y realise convolution
 * (x - x') or correlation (x + x'), a pointwise product with the transformed
 * Green function computed once at setup (Sec. 5), an inverse transform, crop.
 *
 * Conventions common to every entry point
 *  - Returns a status code (PIPE_OK = 0).  No C++ exception crosses the ABI.
 *  - Densities and potentials are device arrays in C order [nx][ny][nz]
 *    (z contiguous), of the handle's dtype, 16-byte aligned.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    asynchronous and stream-ordered unless stated otherwise.
 *  - A handle owns device memory (Green spectrum, workspace, tables) on the
 *    device that was current at setup; it must not be used on two streams at
 *    the same time (the workspace is shared).
 */
#ifndef PIPE_POISSON_H
#define PIPE_POISSON_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define PIPE_OK           0
#define PIPE_EINVAL       1  /* bad argument: sizes, spacings, geometry, null or misaligned pointer */
#define PIPE_ENOMEM       2  /* device or host allocation failed */
#define PIPE_EUNSUPPORTED 3  /* valid request outside what this library implements */
#define PIPE_ECUDA        4  /* a CUDA call or kernel launch failed */
#define PIPE_ETIMEOUT     5  /* a bounded device-side wait gave up (batched launch, staged transverse kernel) */
#define PIPE_ENODEVICE    6  /* no CUDA device / driver available */

/* dtypes */
#define PIPE_F32 0
#define PIPE_F64 1
/* FP32 arithmetic with the z half-spectrum stored between the kernels as
 * complex FP16 (2 x 16 bits per value) with per-slab FP32 scale factors: one
 * per z-transform tile of columns after the forward z transform, one per
 * transverse row after the transverse stage; the Green product is taken in
 * FP16 on operands scaled per transverse column.  An optional variant whose
 * error (1e-4 to 4e-4 relative against the FP64 solve, below 8 FP16 rounding
 * units 2^-11) is above the FP32 path's 1e-5: for uses whose error budget
 * allows it.  Cell-centred meshes only;
 * solves, adjoints and host solves; not the stage, no-alloc, batched or
 * banded entry points (PIPE_EUNSUPPORTED).  Fields are FP32 tensors. */
#define PIPE_F32_C16 2

/* Green function kinds for pipe_green_setup's `igf` argument */
#define PIPE_GREEN_ORDINARY 0   /* Eq. 9: exp(-kappa |w|) */
#define PIPE_GREEN_IGF      1   /* Eq. 16: g_z(w) of Eq. 15 */

/* Pipe cross-section (0,a) x (0,b) (Sec. 2) and the mesh origin.
 * x0, y0: coordinates of mesh node (0,0).  modes_m, modes_n: series truncation. */
typedef struct {
  double a, b;
  double x0, y0;
  int modes_m, modes_n;
} pipe_geometry;

/* Physical mesh nx x ny x nz with spacings hx, hy, hz, and the arithmetic type
 * of the solve (PIPE_F32, PIPE_F64 or PIPE_F32_C16).  The Green function is always tabulated
 * and transformed in FP64; the F32 path uses an FP32 copy of its spectrum. */
typedef struct {
  int nx, ny, nz;
  double hx, hy, hz;
  int dtype;
} pipe_grid;

typedef struct pipe_handle pipe_handle;

/* Tabulate the pipe Green function R (Eq. 9, or R_int of Eq. 16 when igf = 1)
 * on the doubled grid and transform it (Sec. 2, after Eq. 10; Sec. 5: computed
 * once, stored, reused).  Allocates every device buffer the solves need.
 *
 * Two forms of the same operator, chosen per handle (pipe_get_plan's t_kind
 * reports which; pipe_set_plan and pipe_autotune can change it):
 *  - the padded transforms of Eq. 10: nx == ny in {16, 32, 64, 128}; nz in
 *    {32, 64, 128, 256, 512, 1024}; 1 <= modes <= 4096.  Meshes that span
 *    the pipe (nx*hx == a, ny*hy == b to 1e-12 relative) with 2*x0/hx and
 *    2*y0/hy integers (cell-centred x0 = hx/2, or a node on the wall x0 = 0)
 *    store one real octant of the spectrum; any other mesh inside the pipe
 *    (a transverse window, Sec. 5: smaller than the cross-section, at any
 *    origin) uses the general form of Eq. 10 with the four transformed
 *    tables stored in full, for nx == ny <= 64.
 *  - the mode-space form (t_kind 3): the same sum with the transverse
 *    transforms pruned to the modes of the truncated series (Eq. 7), where
 *    the transformed Green function is nonzero: a projection of rho onto the
 *    modes_m x modes_n sine modes, the zero-padded z convolution of each
 *    mode's column by FFT (Appendix A), and the back-projection.  Any mesh
 *    inside the pipe with nx and ny multiples of 16 (nx != ny allowed, up to
 *    4096 each), nz in {32, ..., 1024} as above, modes_m, modes_n <= 32;
 *    PIPE_F32 or PIPE_F64; not banded; and its kernels' shared memory within
 *    the device's 227 KB per CTA (it grows with ny and the modes: FP32 with
 *    20 x 20 modes takes ny up to about 1400, FP64 about 700; FP64 takes at
 *    most about 880 mode pairs, e.g. 32 x 24 but not 32 x 32).  Its tables
 *    (FP64, with FP32 copies) take (nx*mxp + ny*myp + mxp*myp*(nz+1))*12
 *    bytes and its scratch (xblocks + 1)*mxp*myp*nz values of the dtype (the
 *    sizes of pipe_mode_layout).
 *    The default where the modes are at most half the transverse mesh
 *    (2*max(ceil4(modes_m), slots) <= min(nx, ny)) or the padded transforms
 *    cannot take the mesh.
 * A mesh that neither form takes gives PIPE_EUNSUPPORTED.
 * Errors: PIPE_EINVAL (non-positive sizes or spacings, mesh not inside the
 * pipe, bad dtype / igf, out == NULL), PIPE_EUNSUPPORTED (other sizes or
 * meshes), PIPE_ENOMEM, PIPE_ECUDA.  On error *out is set to NULL.
 * Synchronous (returns once the spectrum is ready). */
int pipe_green_setup(const pipe_geometry* geometry, const pipe_grid* grid, int igf,
                     pipe_handle** out);

/* The banded reduction of Sec. 5 (Eq. 17-18): a handle whose solve computes,
 * for every z plane k, only the source planes k' with |k - k'| <= n_neighbors:
 *     phi_ijk = hx hy hz sum_{|k-k'| <= n_neighbors} sum_{i'j'} rho_{i'j'k'} G(..., (k-k') hz)
 * (n_neighbors = 0 is Eq. 17: one 2-D mixed convolution/correlation per
 * plane).  Accurate when the Green function (usually the IGF on a z mesh
 * coarse against the pipe width) is negligible beyond n_neighbors planes;
 * n_neighbors = nz - 1 reproduces the full solve.  No transform along z is
 * taken.  Two forms, chosen like the full solve's (pipe_get_plan t_kind 3 or
 * not):
 *   mode space (any mesh the mode-space form of pipe_green_setup takes): the
 *     projection onto the modes, a (2 n_neighbors + 1)-tap stencil along z on
 *     each mode column with the real-space kernel K_mn(d hz), d <= n_neighbors
 *     (FP64 tables, FP32 copy), and the back-projection; pipe_stage_modes
 *     stage 1 runs the stencil;
 *   transforms (cell-centred meshes, 2*x0/hx == 2*y0/hy == 1, with an nx*ny
 *     complex plane of at most 200 KB: FP32 up to 128^2, FP64 up to 64^2):
 *     the 2-D spectra of the tables at offsets 0..n_neighbors, computed once
 *     (FP64), and two kernels over pairs of z planes; pipe_green_spectrum
 *     returns its (nx+1)*(ny+1)*(n_neighbors+1) planes [d][ky][kx], scaled
 *     by hx*hy*hz/(4*nx*ny).
 * pipe_poisson_solve and pipe_poisson_adjoint (the same operator: it is
 * symmetric) and pipe_poisson_solve_host accept the handle; the transform
 * stage, no-alloc and batched entry points return PIPE_EUNSUPPORTED for it.
 * Errors: as pipe_green_setup (PIPE_EUNSUPPORTED when neither form takes the
 * mesh), plus PIPE_EINVAL for n_neighbors < 0 or >= nz. */
int pipe_banded_setup(const pipe_geometry* geometry, const pipe_grid* grid, int igf, int n_neighbors,
                      pipe_handle** out);

/* Free-space (Hockney) comparison handle: Eq. 5 with G = 1/r (Eq. 3) tabulated
 * on the doubled grid with convolution offsets in x, y and z.  The paper does
 * not give G(0,0,0); `self_value` supplies it (<= 0 selects 1/min(hx,hy,hz)).
 * Same size limits and errors as pipe_green_setup (no geometry needed). */
int pipe_free_space_setup(const pipe_grid* grid, double self_value, pipe_handle** out);

/* phi = A rho (the forward solve of Eq. 10).  rho, phi: device [nx][ny][nz]
 * arrays of the handle's dtype; phi may alias rho (in-place).  Errors:
 * PIPE_EINVAL (null handle or pointer, misaligned pointer), PIPE_ECUDA. */
int pipe_poisson_solve(pipe_handle* h, const void* rho, void* phi, void* stream);

/* drho = A^T dphi: the transposed operator, applied as the transposed chain of
 * Eq. 10 (the final-direction transforms of each term first, the product with
 * the same Green spectra, then the forward transform, crop).  Because
 * G(r, r') = G(r', r) (Eq. 7), A^T = A; this entry point is what gradients
 * (dW/drho, backward passes) call.  Same arguments and errors as the solve. */
int pipe_poisson_adjoint(pipe_handle* h, const void* dphi, void* drho, void* stream);

/* pipe_poisson_solve without any device allocation by the library: the
 * solve's working buffer is a fixed 64 MiB device array that belongs to the
 * library instead of device memory owned by the handle -- for the
 * padded-transform form the z half-spectrum, (nz+1)*nx*ny complex values of
 * the dtype; for the mode-space form (plan t_kind 3) the projections and the
 * convolved mode columns, (xblocks+1)*mxp*myp*nz values (pipe_mode_layout).
 * The handle's current form runs, so the result is bit for bit that of
 * pipe_poisson_solve.  Meant for programs that must not let a library
 * allocate device memory while they run (a host that keeps the GPU's memory
 * in its own pool, a loop that cannot risk an allocation stalling or
 * failing): they create the handle during initialisation and call this
 * afterwards.  The paper has no counterpart; it is an interface convenience.
 * The array is reserved on a device when a handle is set up there (the setup
 * looks up its device address, with that device current; a failure there is
 * reported by the first call of this entry point, which tries again), and it
 * stays reserved until the process exits.  The first launch of each kernel
 * on a device also loads that kernel's code (the CUDA runtime's lazy
 * loading): a program that must not see that memory taken later makes one
 * call during initialisation or sets CUDA_MODULE_LOADING=EAGER.  After
 * cudaDeviceReset every handle on that device is invalid; a handle set up
 * afterwards looks the address up again.  All calls share the array: calls
 * whose kernels overlap on the GPU (other streams or handles at the same
 * time) race and corrupt each other's results.  Nothing needs clearing
 * between calls.  Same arguments as pipe_poisson_solve.  Errors: PIPE_EINVAL
 * (null or misaligned pointers), PIPE_EUNSUPPORTED when the buffer exceeds
 * 64 MiB (e.g. 128x128x256 FP32 in the transform form fits, 128x128x512 does
 * not; the mode-space form of 128x128x1024 FP32 with 20 x 20 modes takes
 * 4.9 MB), or for banded, complex-FP16 or window (transform form) handles,
 * PIPE_ECUDA. */
int pipe_poisson_solve_noalloc(pipe_handle* h, const void* rho, void* phi, void* stream);

/* Same as pipe_poisson_solve but rho_host / phi_host are HOST arrays: the
 * library copies rho to the device, solves and copies phi back on `stream`,
 * then synchronises the stream.  Device staging buffers are allocated on the
 * first call and owned by the handle.  Host memory should be pinned for full
 * copy bandwidth (pageable memory works, slower). */
int pipe_poisson_solve_host(pipe_handle* h, const void* rho_host, void* phi_host, void* stream);

/* `count` solves from HOST memory, with the transfers overlapped: solve k runs
 * on `stream` while the input of solve k+1 is copied in and the result of
 * solve k-1 is copied out (two further streams, two device staging buffers
 * per direction, all owned by the handle and created on the first call).
 * rho_host[k] / phi_host[k]: host arrays of nx*ny*nz values of the handle's
 * dtype (pinned memory for overlapped copies).  Synchronous: returns when every
 * result is in host memory.  Same operator as pipe_poisson_solve.
 * Errors: PIPE_EINVAL (null arrays or entries, count < 1), PIPE_ENOMEM,
 * PIPE_ECUDA, and the errors of pipe_poisson_solve. */
int pipe_poisson_solve_host_stream(pipe_handle* h, const void* const* rho_host, void* const* phi_host,
                                   int count, void* stream);

/* n independent solves (different grids and geometries) in one persistent
 * kernel launch that walks a work list of (solve, stage, tile) items; each
 * stage of a solve waits, with a bounded spin, for the previous stage of the
 * same solve.  All handles must share one dtype and device, and must not be
 * used concurrently elsewhere.  A wait that gives up records PIPE_ETIMEOUT in
 * the batch status (read with pipe_batch_status after the stream completes).
 * The first call with a handle set builds the work lists and times the ways
 * of splitting the set between the persistent launch and single-solve launches
 * issued after it on the same stream (cut-offs: none, then each distinct z
 * spectrum size from the largest down, at most five; the solves at or above
 * the cut-off go to single-solve launches) and three work-list orders, keeping
 * the fastest; those timing runs are valid solves, and the first call
 * synchronises the stream.  Later calls with the same set reuse the
 * choice and are capturable in a CUDA graph.  Results equal those of
 * pipe_poisson_solve up to rounding, and bitwise for FP32 handles whose plan is
 * z_warps = 16, z_pipe = 0, t_h = 1, t_threads = 512, and t_kind = 1 on
 * cell-centred meshes, 0 on others (the persistent kernel's shapes).
 * Errors: PIPE_EINVAL (n < 1, null arrays), PIPE_EUNSUPPORTED (mixed dtypes
 * or devices), PIPE_ENOMEM, PIPE_ECUDA. */
int pipe_poisson_solve_batched(pipe_handle* const* handles, const void* const* rho,
                               void* const* phi, int n, void* stream);

/* Device-side status of the last batched launch that used `handles[0]`'s
 * batch plan: PIPE_OK or PIPE_ETIMEOUT.  Synchronous (copies one word). */
int pipe_batch_status(pipe_handle* const* handles, int n);

/* The choice the first batched call made for this exact handle set: how many
 * solves run in the persistent launch (the rest as single-solve launches) and
 * the work-list order (0 stage-major, 1 pipelined, 2 L2-local).  Errors:
 * PIPE_EINVAL (null pointers, or no tuned plan for this set). */
int pipe_batch_plan_info(pipe_handle* const* handles, int n, int* persistent, int* order);

/* The number of side streams (0, 2 or 3) that the first batched call chose
 * for this exact handle set's single-solve launches: 0 runs them in order on
 * the caller's stream; otherwise they are dealt round-robin to side streams
 * that start after the persistent launch and rejoin the caller's stream
 * through events, so that the solves overlap (parallel branches when the call
 * is captured in a CUDA graph).  Not in the paper: a GB300 scheduling choice.
 * Errors: PIPE_EINVAL (null pointers, or no tuned plan for this set). */
int pipe_batch_side_streams(pipe_handle* const* handles, int n, int* nside);
/* Override that choice (nside 0, 2 or 3) for the later calls with this set,
 * for tests and experiments.  Errors: PIPE_EINVAL (other values, null
 * pointers, or no tuned plan for this set). */
int pipe_batch_select_streams(pipe_handle* const* handles, int n, int nside);

/* Mode-form groups of the batched call: FP32 solves outside the persistent
 * launch that run the mode-space form with the occupancy-laid-out kernels
 * (pipe_get_plan t_kind 3 on a mesh symmetric in y, ny/2 in {16, 32, 64, 128})
 * and share nx, ny, nz, the mode counts and the y-mode table run together:
 * one launch per stage for up to 64 solves, with the same kernels and the
 * same results, bit for bit, as their single-solve launches.  The tuner
 * times the call with and without them.  pipe_batch_grouped reports how
 * many solves the tuned plan runs that way (0: none) and, if `groups` is not
 * null, in how many groups; pipe_batch_select_groups
 * sets it on (1) or off (0) for later calls, for tests and experiments.
 * Errors: PIPE_EINVAL as pipe_batch_side_streams. */
int pipe_batch_grouped(pipe_handle* const* handles, int n, int* grouped, int* groups);
int pipe_batch_select_groups(pipe_handle* const* handles, int n, int on);

/* Override that choice for later calls with this exact handle set: `variant`
 * k runs persistent the solves whose z spectrum is smaller than the k-th
 * largest distinct spectrum size of the set (k = 0: every solve), `order` as
 * above.  For tests and experiments.  Errors: PIPE_EINVAL (no tuned plan for
 * this set, k beyond the cut-offs built, order outside 0..2, or order != 0
 * for a variant with no persistent solve). */
int pipe_batch_select(pipe_handle* const* handles, int n, int variant, int order);

/* Failure-detection test hook for the batched launch: the NEXT
 * pipe_poisson_solve_batched call with this exact handle set (whose work list
 * must already exist, i.e. after one normal call) skips every item of stage
 * `drop_stage` (0 z-forward, 1 transverse, 2 z-inverse) without counting it
 * and polls at most `spin_limit` times per wait, so the dependent waits give
 * up and the batch status becomes PIPE_ETIMEOUT while the kernel still ends.
 * That call runs every solve of the set in the persistent launch.
 * The results of that call are undefined.  Errors: PIPE_EINVAL. */
int pipe_batch_inject_fault(pipe_handle* const* handles, int n, int drop_stage, long long spin_limit);

/* Copy the handle's FP64 Green spectrum to host memory `out` of `count`
 * doubles.  Spanning meshes: the real octant g[kz][ky][kx], kz <= nz,
 * ky <= ny, kx <= nx, already multiplied by hx*hy*hz/(8*nx*ny*nz); count
 * (nx+1)*(ny+1)*(nz+1).  Window meshes: the four transformed tables
 * [cc, cr, rc, rr][kz <= nz][ky < 2ny][kx < 2nx] as interleaved complex
 * (re, im), same scale; count 8*(nz+1)*(2ny)*(2nx).  Banded handles: see
 * pipe_banded_setup.  Synchronous.  For inspection and tests. */
int pipe_green_spectrum(pipe_handle* h, double* out, size_t count);

/* Stages of the solve, exposed for inspection and per-kernel tests.  `spec`
 * is a caller-owned device array of (nz+1)*nx*ny complex values of the
 * handle's dtype (interleaved re, im), laid out [kz][i][j].
 *   z_forward : spec = the (2nz)-point DFT along z of the zero-padded rho,
 *               kz = 0..nz (direction e^{-}, or e^{+} when adjoint != 0)
 *   transverse: in place on spec -- padded x,y transforms, Green product,
 *               cropped inverse x,y transforms (adjoint: transposed chain)
 *   z_inverse : phi = the unnormalised (2nz)-point inverse along z of the
 *               Hermitian half spectrum, first nz outputs */
int pipe_stage_z_forward(pipe_handle* h, const void* rho, void* spec, int adjoint, void* stream);
int pipe_stage_transverse(pipe_handle* h, void* spec, int adjoint, void* stream);
int pipe_stage_z_inverse(pipe_handle* h, const void* spec, void* phi, int adjoint, void* stream);
/* (The three stages above exist on handles of the padded-transform form;
 * PIPE_EUNSUPPORTED on a handle that only the mode-space form takes.) */

/* Layout of the mode-space form (Sec. 2 Eq. 7: the sine modes of the
 * truncated series).  mx = modes_m; mxp = mx rounded up to a multiple of 4;
 * myp = the y-mode slots: when the mesh is symmetric about the pipe's
 * mid-plane in y (2*y0 + (ny-1)*hy == b, e.g. cell-centred), *fold = 1 and
 * slot s < myp/2 holds mode n = 2s+1, slot s >= myp/2 mode n = 2(s - myp/2)+2;
 * otherwise *fold = 0 and slot s holds n = s+1 (slots beyond modes_n are
 * zero).  Mode column c = (m-1)*myp + slot.  xblocks: the groups of x rows
 * whose projections the first stage writes separately (the kernel works on
 * blocks of 16 rows in FP32, 8 in FP64, and sums up to 4 neighbouring blocks
 * in a thread-block cluster; xblocks = blocks / that cluster size, 2 for
 * FP32 nx = 128).  Errors: PIPE_EINVAL (null pointers), PIPE_EUNSUPPORTED
 * (the mode-space form cannot take the handle). */
int pipe_mode_layout(pipe_handle* h, int* mx, int* mxp, int* myp, int* fold, int* xblocks);

/* The FP64 kernel spectra of the mode-space form, [c][kz] for the mxp*myp
 * mode columns and kz = 0..nz: the DCT-I of the doubled z table of
 *     K_mn(d) = hx*hy*hz * (8*pi/(a*b)) * f_mn(d*hz) / kappa_mn
 * (f = exp(-kappa |w|) of Eq. 9, or the IGF g_z of Eq. 15), with the free
 * slot d = nz filled by the formula, divided by 2*nz; zero for padded
 * columns.  count must be mxp*myp*(nz+1).  Synchronous.  For inspection and
 * tests.  Errors: PIPE_EINVAL, PIPE_EUNSUPPORTED as pipe_mode_layout. */
int pipe_mode_spectrum(pipe_handle* h, double* out, size_t count);

/* Stages of the mode-space form, for inspection and per-kernel tests (device
 * arrays of the handle's dtype, caller-owned, 16-byte aligned; asynchronous):
 *   stage 0: in = rho [nx][ny][nz] -> out = part [xblocks][mxp*myp][nz], the
 *            projection of each block of x rows (block b: rows b*nx/xblocks ..)
 *            part[b][c][k] = sum_{i in block b} sum_j sin(m pi x_i/a) *
 *                            sin(n pi y_j/b) rho[i][j][k]
 *   stage 1: in = part -> out = psi [mxp*myp][nz]: the blocks summed, each
 *            column convolved along z with its kernel (zero-padded 2nz-point
 *            transforms, the spectrum of pipe_mode_spectrum), first nz values;
 *            for a banded handle (pipe_banded_setup) the sum over
 *            |d| <= n_neighbors of K_c(|d| hz) part[c][k - d] instead
 *   stage 2: in = psi -> out = phi [nx][ny][nz]:
 *            phi[i][j][k] = sum_{m,n} sin(m pi x_i/a) sin(n pi y_j/b) psi[c][k]
 * The three in a row are the solve of this form (pipe_poisson_solve with plan
 * t_kind 3); it is symmetric, so the adjoint is the same chain.
 * Errors: PIPE_EINVAL (stage outside 0..2, null or misaligned pointers),
 * PIPE_EUNSUPPORTED as pipe_mode_layout, PIPE_ECUDA. */
int pipe_stage_modes(pipe_handle* h, int stage, const void* in, void* out, void* stream);

/* Time the kernel variants available for this handle's sizes on `stream` and
 * keep the fastest (per size and dtype, shared by all handles of that shape in
 * this process).  Synchronous; uses the handle's workspace as scratch.  If the
 * environment variable PIPE_TUNE_CACHE names a file, results are read from and
 * appended to it. */
int pipe_autotune(pipe_handle* h, void* stream);

/* Read or pin the kernel variants a handle uses: z_warps in {4, 8, 16} (CTA
 * size of the z transforms; 4 and 16 apply at nz >= 512, smaller nz run 8),
 * z_pipe in {0, 1} (1: each z CTA walks several tiles and streams the next
 * tile's input while transforming the current one), t_h in
 * {1, 2, 4} (the transverse stage runs t_h CTAs per kz plane, each holding
 * nx/t_h rows), t_threads in {128, 256, 512}, t_kind in {0, 1, 2}: 0 computes
 * each transverse line with the padded 2n-point transforms of Eq. 10 (any
 * supported mesh); 1 computes the same combinations with n-point transforms,
 * for cell-centred meshes only (2*x0/hx == 2*y0/hy == 1) and t_h == 1; its
 * plane buffer is in shared memory, or for FP64 128^2 planes in global
 * scratch planes that the setup allocates ((nz+1)*nx*ny complex).  2 is the
 * same arithmetic as 1 in a persistent launch (one CTA per SM looping over
 * kz planes) whose input rows arrive by bulk asynchronous copies into shared
 * memory, the next plane's first rows while the current plane is still being
 * transformed; same meshes as 1, plane buffer in shared memory only (not
 * FP64 128^2).  t_kind 3 selects the mode-space form of pipe_green_setup
 * (the other fields then keep the transform plan for a later switch back);
 * pipe_get_plan reports 3 while it is selected.  pipe_set_plan returns
 * PIPE_EINVAL for values outside those sets and PIPE_EUNSUPPORTED for t_kind
 * 1 or 2 on other meshes, for t_kind 3 on a handle the mode-space form cannot
 * take, and for t_kind 0..2 on a handle only the mode-space form takes; a
 * variant that does not fit the device (shared memory) makes the next solve
 * fail with PIPE_ECUDA.  pipe_autotune, on a handle that both forms take,
 * also times a few solves of each and keeps the faster form.
 * The free-space (Hockney) handle ignores t_kind. */
int pipe_get_plan(pipe_handle* h, int* z_warps, int* z_pipe, int* t_h, int* t_threads, int* t_kind);
int pipe_set_plan(pipe_handle* h, int z_warps, int z_pipe, int t_h, int t_threads, int t_kind);

/* The handle's device-side error word, read and cleared (synchronous: waits
 * for the device).  PIPE_OK, or PIPE_ETIMEOUT when a bounded wait of the
 * staged transverse kernel (t_kind 2) for its own asynchronous copies gave up
 * since the last read; the results of the solves in between are then
 * undefined.  Errors: PIPE_EINVAL (null handle), PIPE_ECUDA. */
int pipe_status(pipe_handle* h);

/* Failure detection without a GPU fault, for tests: the next solve or
 * adjoint of this handle (pipe_poisson_solve / _adjoint) whose transverse
 * stage is the staged kernel (t_kind 2) has its first CTA leave out its bulk
 * copy number drop_copy (0 = the first) and gives every wait at most
 * poll_limit polls.  The wait for the left-out copy gives up, PIPE_ETIMEOUT
 * is recorded (pipe_status), no further copy is issued by that CTA and the
 * kernel still ends; the results of that call are undefined, later calls are
 * unaffected.  The request is consumed by the next solve or adjoint whatever
 * its plan.  Errors: PIPE_EINVAL (null handle, drop_copy < 0,
 * poll_limit < 1). */
int pipe_inject_stage_fault(pipe_handle* h, int drop_copy, long long poll_limit);

/* Electric field E = -grad phi on the handle's mesh (device arrays of the
 * handle's dtype; FP32 for PIPE_F32_C16): phi [nx][ny][nz], E [3][nx][ny][nz]
 * (x, y, z components, each laid out like phi).  The paper defines no
 * discrete gradient: second-order central differences inside the mesh,
 * second-order one-sided differences on its faces (exact for potentials
 * quadratic in each coordinate).  Asynchronous on `stream`.
 * Errors: PIPE_EINVAL (null or misaligned pointers), PIPE_ECUDA. */
int pipe_electric_field(pipe_handle* h, const void* phi, void* E, void* stream);

/* Cloud-in-cell deposit of n macroparticles (positions xyz[n][3], FP64 or FP32
 * per the handle's dtype, charge q each) onto the handle's mesh nodes:
 * rho[i][j][k] += q * w / (hx*hy*hz), w the trilinear weight of node (i,j,k).
 * Particles outside the mesh's node range contribute only to the nodes that
 * exist.  rho must be zeroed by the caller.  Device arrays. */
int pipe_cic_deposit(pipe_handle* h, const void* xyz, int64_t n, double q, void* rho,
                     void* stream);

/* Adjoint of the deposit with respect to the positions: for a cotangent
 * grad_rho on the mesh, grad_xyz[p][d] = q/(hx*hy*hz) * sum_nodes grad_rho *
 * d w / d x_d  (derivative of the trilinear weights).  Device arrays. */
int pipe_cic_gather_grad(pipe_handle* h, const void* xyz, int64_t n, double q,
                         const void* grad_rho, void* grad_xyz, void* stream);

/* Release everything the handle owns (synchronises the device first).
 * NULL is ignored. */
void pipe_green_destroy(pipe_handle* h);

/* Static description of a status code. */
const char* pipe_strerror(int status);

/* Host-only self test of the library's compile-time twiddle generator against
 * the C library's cos/sin; returns the maximum absolute error.  Needs no GPU. */
double pipe_selftest_twiddles(void);

/* Library version string. */
const char* pipe_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PIPE_POISSON_H */
