/*
 * igg.h - C ABI of the GB300 (sm_103a) implementation of the heat-diffusion
 * hot path of "Distributed Parallelization of xPU Stencil Computations in
 * Julia" (Omlin, Raess, Utkin; arXiv 2211.15716):
 *   - the implicit global grid of subdomains (Sec. Approach; Fig. 1
 *     init_global_grid, nx_g/ny_g/nz_g, finalize_global_grid),
 *   - the halo update that keeps it consistent (update_halo!),
 *   - the explicit 7-point diffusion step (Fig. 1 step!),
 *   - the boundary/inner split that hides the halo update behind the
 *     inner-block computation (Fig. 1 @hide_communication (16, 2, 2);
 *     Sec. Approach: transfers on high-priority streams),
 *   - and three reshaped forms of the step: reduced-precision storage,
 *     batches of independent uneven problems, and the adjoint step.
 *
 * On one GPU the process topology is virtual: all nsub subdomains live in
 * one device's memory and a field is ONE contiguous device buffer laid out
 * [nsub][nz][ny][nx] (x fastest; subdomain number x fastest over dims).
 * The linear index of local point (ix, iy, iz) of subdomain s is
 *   ix + nx*(iy + ny*(iz + nz*s)),  0-based.
 *
 * Conventions for every function:
 *   - Return value: IGG_OK (0) or a negative error code; igg_last_error()
 *     gives a message for the calling thread. No function aborts or traps.
 *   - Field pointers are DEVICE pointers on the grid's device, owned by the
 *     caller, 16-byte aligned, holding nsub*nx*ny*nz elements of the dtype.
 *     Misaligned or NULL pointers give IGG_EINVAL.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). All device work of a call is ordered after the work already
 *     queued on `stream`, and work queued on `stream` afterwards is ordered
 *     after it; calls return without synchronising unless stated.
 *   - The library owns its handles, descriptor tables, streams, events and
 *     CUDA graphs, and frees them in the matching finalize/destroy call.
 */
#ifndef IGG_H
#define IGG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IGG_ABI_VERSION 1

/* status codes */
#define IGG_OK 0
#define IGG_EINVAL (-1) /* invalid argument (sizes, overlap, widths, dims, pointers) */
#define IGG_ECUDA (-2)  /* a CUDA runtime call failed; message has the CUDA error text */
#define IGG_ENOMEM (-3) /* device or host allocation failed */
#define IGG_ESTATE (-4) /* handle used in a wrong state */

/* element types of the fields (Fig. 1's @init_parallel_stencil(CUDA,
 * Float64, 3) picks FP64; FP32 and BF16 storage are the reduced-precision
 * forms). F64 computes in FP64, F32 in FP32, BF16 loads BF16, computes in
 * FP32 and rounds the result to BF16 (nearest-even). */
typedef enum { IGG_F64 = 0, IGG_F32 = 1, IGG_BF16 = 2 } igg_dtype;

typedef struct igg_grid igg_grid;
typedef struct igg_batch igg_batch;

/* Message of the last failing call on this thread ("" if none). The pointer
 * stays valid until the next call on this thread. */
const char *igg_last_error(void);

/* IGG_ABI_VERSION of the library. */
int igg_abi_version(void);

/* ---------------------------------------------------------------------------
 * Implicit global grid (Sec. Approach; Fig. 1 init_global_grid).
 *
 * Creates a virtual Cartesian topology of subdomains, each a local array of
 * nx*ny*nz points, on the CURRENT CUDA device.
 *   dims[3]    : subdomains per dimension; entries equal to 0 are chosen so
 *                that dims[0]*dims[1]*dims[2] == nsub, as balanced as
 *                possible and non-increasing over the free entries
 *                (MPI_Dims_create's rule). NULL = all free.
 *   nsub       : number of subdomains (used when dims has zeros; must equal
 *                the product otherwise).
 *   overlap[3] : planes shared by neighbouring subdomains, >= 2 (halo width
 *                1). NULL = (2, 2, 2).
 *   periods[3] : nonzero = periodic dimension. NULL = none.
 * Global size per dimension: n_g = dims*(n - o) + o, or dims*(n - o) when
 * periodic. Requires n >= 3 and 2 <= o <= n - 1 per dimension, so that both
 * send planes (indices o-1 and n-o) are inner points.
 * 2-D and 1-D grids: ny = 1 and/or nz = 1 makes that dimension absent (its
 * dims entry 1 or free, not periodic, n_g = 1): its only index counts as
 * inner, it has no neighbours, no halo and no second difference (pass an
 * infinite spacing, whose weight dt*lam/dd^2 is then exactly 0). Steps on
 * such grids run the vector or scalar kernels; the hidden step runs as the
 * plain step followed by the halo update (same result). The adjoint and the
 * acoustic step need a 3-D grid.
 * Creates the library's high- and low-priority streams and events.
 * On success *out owns the grid; release it with igg_finalize_global_grid.
 * ------------------------------------------------------------------------- */
int igg_init_global_grid(int nx, int ny, int nz, const int dims[3], int nsub,
                         const int overlap[3], const int periods[3],
                         igg_grid **out);

/* Fig. 1 finalize_global_grid: frees every resource of the grid. NULL is
 * accepted. The caller must not use the handle afterwards. Waits for the
 * grid's outstanding work before freeing. */
int igg_finalize_global_grid(igg_grid *grid);

/* Fig. 1 nx_g(), ny_g(), nz_g(): the global grid size. */
int igg_global_size(const igg_grid *grid, int n_g[3]);

/* Local size, dims, overlap, periods and subdomain count of the grid (any
 * output pointer may be NULL). */
int igg_grid_shape(const igg_grid *grid, int n[3], int dims[3], int overlap[3],
                   int periods[3], int *nsub);

/* Subdomain `sub`: its Cartesian coordinates (x fastest numbering), its
 * left/right neighbours per dimension (-1 at a physical boundary) and the
 * global index of its local point 0 per dimension (coords*(n - o); the
 * global index of local point i is offset + i, modulo n_g when periodic).
 * Any output pointer may be NULL. */
int igg_subdomain_info(const igg_grid *grid, int sub, int coords[3],
                       int left[3], int right[3], int offset[3]);

/* ---------------------------------------------------------------------------
 * Halo update (update_halo!, Sec. Approach; Fig. 1 update_halo!(T2)).
 *
 * For each of the nfields fields (device pointers of `dtype`, layout above),
 * the result of this exchange for the dimensions in the order x, y, z:
 * every subdomain's first plane (index 0) receives plane n-o of its left
 * neighbour, and its last plane (index n-1) receives plane o-1 of its right
 * neighbour. Whole planes, including points in other dimensions' halos, so
 * edges and corners end up exactly as after the sequential x, y, z exchange.
 * The copy is bit exact. On 3-D grids each field takes one launch that
 * gathers every halo cell's value directly from the point the sequential
 * copies would bring to it (following them back: z, then y, then x); 2-D and
 * 1-D grids take one plane-copy launch per dimension for all the fields.
 * Work is ordered on `stream`.
 * ------------------------------------------------------------------------- */
int igg_update_halo(igg_grid *grid, void *const fields[], int nfields,
                    igg_dtype dtype, void *stream);

/* update_halo! on fields of a staggered grid (Sec. Approach: regular
 * staggered grids): each of the nfields fields has local size nf (x, y, z;
 * layout [nsub][nf[2]][nf[1]][nf[0]]) with |nf[d] - n[d]| <= 1, e.g. fluxes
 * or face velocities one point shorter or longer than the grid's arrays.
 * The field's overlap is o + (nf - n) per dimension (the staggered points on
 * a shared face are shared as well): its first plane receives plane nf - o_f
 * of the left neighbour, its last plane plane o_f - 1 of the right one, in
 * the order x, y, z as igg_update_halo; a dimension where o_f < 2 exchanges
 * nothing (neighbours then share one plane and have no halo plane). Plane
 * tables are built once per size and kept on the grid. IGG_EINVAL for sizes
 * off by more than one or below 3, NULL or misaligned fields. */
int igg_update_halo_staggered(igg_grid *grid, void *const fields[], int nfields,
                              igg_dtype dtype, const int nf[3], void *stream);

/* update_halo!(A...) on fields of possibly different staggered sizes:
 * sizes[3*i .. 3*i+2] is field i's local size (each within one point of the
 * grid's, rules of igg_update_halo_staggered). One launch per dimension
 * serves all fields (x, then y, then z), with the same result as updating
 * the fields one by one. */
int igg_update_halo_fields(igg_grid *grid, void *const fields[], const int *sizes,
                           int nfields, igg_dtype dtype, void *stream);

/* Device error word of the grid's pipelined kernels: bit 1 = a bounded
 * wait inside a kernel gave up (the kernel stopped early and its output is
 * incomplete), bit 2 = waiting for its own copies in flight gave up.
 * Synchronises the device; clear != 0 resets the word to 0. */
#define IGG_DEV_ERR_TIMEOUT 1u
#define IGG_DEV_ERR_DRAIN 2u
#define IGG_DEV_ERR_BOUNDS 4u
int igg_device_status(igg_grid *grid, unsigned *status, int clear);

/* Self-test of that failure detection, without a GPU fault: on the current
 * device, one kernel whose warps wait on two mbarriers with the pipelined
 * kernels' bounded wait (about 2 s); the phase of one completes, nothing
 * ever arrives on the other. The warps agree on stopping through the barrier
 * reduction of the persistent kernels, so none is left waiting, and the
 * kernel records IGG_DEV_ERR_TIMEOUT. *status (host) receives the recorded
 * bits: IGG_DEV_ERR_TIMEOUT when the detection works. Synchronises the
 * device; takes about 2 s. */
int igg_selftest_bounded_wait(unsigned *status);

/* Grid options (wait for the grid's streams; cached CUDA graphs are
 * rebuilt):
 *   IGG_OPT_TMA (default 1): run the regular boxes of the step with the
 *     TMA-pipelined kernel when the row length is a multiple of 16 bytes; 0
 *     selects the register-pipelined vector kernel. Bit-identical results.
 *   IGG_OPT_F64_EMU (default 1): F64 fields use the emulated FP64 cell: for
 *     points whose 7 stencil values share sign and exponent, the second
 *     differences are formed exactly from the bit patterns as integers,
 *     weighted in float-float pairs and applied with one FP64 FMA and an
 *     integer ulp correction (per-step error within about one ulp of T2 plus
 *     2^-44 of Ci sum_d |w_d D_d|); stencils across powers of two or across
 *     zero put their values on the grid of the largest value's ulp (the
 *     aligned path, two FP64 FMAs, error within a few of those ulps); the
 *     rest (relative second differences above about 2^-5, values near
 *     overflow or underflow, weights above 2^40) use the FP64 cell (8 FP64
 *     instructions per point). On the TMA kernel the points outside the
 *     one-FMA path go to a fix-up launch, so fields where many stencils
 *     change sign or exponent step about three times slower (a field that
 *     changes sign: 3.0 x the time of a smooth one, below the FP64
 *     cell's 3.6 x; see igg_fixup_stats).
 *   IGG_OPT_FUSED_HALO (default 1): igg_step_hidden (and igg_run with
 *     widths) run as the full step launch followed by the one-launch halo
 *     update (all subdomains being in the device's memory, no transfer is
 *     left to overlap, and the split's extra launches cost more than they
 *     hide); 0 selects the boundary/inner split described at
 *     igg_step_hidden. Bit-identical results either way.
 *   IGG_OPT_PHASE_TIMES (default 0): every step queued outside CUDA-graph
 *     capture (igg_step, igg_step_hidden, the odd last step of igg_run)
 *     records three CUDA events on its stream: at its start, after its
 *     stencil launches (with the emulated FP64 cell's fix-up launch), at its
 *     end; igg_phase_times reads them. Steps inside igg_run's graphs are not
 *     timed. Setting the option drops the steps recorded so far.
 *   IGG_OPT_HIDE_HALO (default 0): with IGG_OPT_FUSED_HALO = 1, 3-D grids
 *     on the TMA kernel run a step followed by its halo update as two sets
 *     of the full step's tiles: the face tiles (those that read a halo cell
 *     or compute a point of a sent plane) and then the halo update on the
 *     library's high-priority stream, the inner tiles meanwhile on its
 *     low-priority stream; `stream` waits for both. The inner tiles neither
 *     read nor write what the halo update touches, so the result is the
 *     same bit for bit; 0 runs the tiles as one launch and then the halo
 *     update on `stream`. Measured slower on the GB300: the two concurrent
 *     tile sets take longer than the one launch by more than the halo
 *     update they hide (FP64 bench step 1.179 against 1.146 ms). */
#define IGG_OPT_TMA 1
#define IGG_OPT_F64_EMU 2
#define IGG_OPT_FUSED_HALO 3
#define IGG_OPT_PHASE_TIMES 4
#define IGG_OPT_HIDE_HALO 5
int igg_grid_set_option(igg_grid *grid, int option, int value);

/* Per-phase device time of the steps recorded under IGG_OPT_PHASE_TIMES
 * since the last call (at most 4096 steps; later steps are not recorded):
 * ms[0] = the stencil phase (full-step form: the stencil launch and its
 * fix-up launch; split form: from the step's start to the end of the
 * high-priority stream's boundary slabs and halo update), ms[1] = the rest
 * of the step (full-step form: the halo update; split form: the remainder
 * of the inner block until both streams joined), ms[2] = ms[0] + ms[1],
 * each summed over the steps; *steps = their number. Waits for the last
 * recorded step; the record is then emptied. No counterpart in the paper
 * (which times whole steps): a measurement aid of the library. */
int igg_phase_times(igg_grid *grid, double ms[3], int *steps);

/* Bounds-checked build. The library compiled with -DIGG_BOUNDS_CHECK (built
 * beside the release library as libigg_checked.so, chosen by the Python
 * binding when the environment has IGG_BOUNDS_CHECK=1) tests every global
 * index of the default step's kernels (the TMA stencil's stores, the fix-up
 * launch, the one-launch halo update) against its field's extent before the
 * access; a failing test skips the access (no trap) and sets a device flag.
 * igg_bounds_checked: 1 in that build, 0 in the release build.
 * igg_bounds_status: *status = IGG_DEV_ERR_BOUNDS when any test failed since
 * the last clear (always 0 in the release build); synchronises the device;
 * clear != 0 resets the flags. Not in the paper: a debugging aid standing in
 * for a memory checker. */
int igg_bounds_checked(void);
int igg_bounds_status(unsigned *status, int clear);

/* Points the emulated FP64 cell left to its fix-up launch: counts[0] = the
 * 32-point row segments listed, counts[1] = the points in them, summed over
 * every FP64 step the grid ran with the TMA kernel since the grid was made
 * (or last cleared); clear != 0 resets both to 0. Synchronises the device.
 * No counterpart in the paper: it shows how much of a field takes the slow
 * path of the emulated cell (stencils that change sign or cross powers of
 * two). */
int igg_fixup_stats(igg_grid *grid, unsigned long long counts[2], int clear);

/* ---------------------------------------------------------------------------
 * Diffusion step (Fig. 1 step!) on every subdomain:
 *   T2 = T + dt*(lam*Ci*(d2x/dx^2 + d2y/dy^2 + d2z/dz^2))
 * on every inner point (local index 1..n-2 in each dimension), where d2x is
 * the second difference T[x+1] - 2 T[x] + T[x-1]. Points on a subdomain's
 * array boundary are NOT written (Fig. 1's T2 = copy(T) makes them fixed).
 * T2 must not alias T or Ci. No halo update is done.
 * The arithmetic is the same in every kernel of the library (full step,
 * boundary slabs, inner block, batched form), so all of them produce
 * identical bits for the same point.
 * ------------------------------------------------------------------------- */
int igg_step(igg_grid *grid, void *T2, const void *T, const void *Ci,
             igg_dtype dtype, double lam, double dt, double dx, double dy,
             double dz, void *stream);

/* Fig. 1 @hide_communication widths begin step!(T2,T,...); update_halo!(T2)
 * end. By default (IGG_OPT_FUSED_HALO = 1) this is the full step's tiles
 * followed by the one-launch halo update of T2 on `stream`; with
 * IGG_OPT_HIDE_HALO = 1 on 3-D TMA grids the tiles next to the faces go
 * first and the halo update runs beside the inner tiles (two streams of the
 * library, joined into `stream`). With IGG_OPT_FUSED_HALO 0 it is the
 * paper's split: the step on the boundary set of every subdomain (inner points whose
 * 1-based index i has i <= w or i >= n - w + 1 in some dimension, w =
 * widths[d]) runs first on the library's high-priority stream, followed
 * there by the halo update of T2; the inner block runs concurrently on the
 * low-priority stream; `stream` waits for both. Requires widths[d] >=
 * overlap[d] (so all sent planes are in the boundary set). The boundary
 * launches compute whole tiles of the kernel: inner-block points that share
 * a tile with boundary points are computed there as well (before the halo
 * update), and the low-priority launch covers the remaining inner block.
 * Every point is computed once with the same arithmetic, so the result is
 * bit-identical to igg_step followed by igg_update_halo(T2). */
int igg_step_hidden(igg_grid *grid, const int widths[3], void *T2,
                    const void *T, const void *Ci, igg_dtype dtype, double lam,
                    double dt, double dx, double dy, double dz, void *stream);

/* Fig. 1's time loop: nt times { step (hidden when widths != NULL, else
 * plain step then halo update) of T2 from T; swap T and T2 }. The loop is
 * captured once into a CUDA graph (two steps per graph launch) and cached
 * on the grid for the same pointers, dtype, widths and coefficients.
 * T2 must hold a copy of T's boundary values on entry (Fig. 1 T2 =
 * copy(T)). After the call the newest state is in T when nt is even and in
 * T2 when nt is odd (the buffers swap roles every step, as in Fig. 1). */
int igg_run(igg_grid *grid, int nt, const int widths[3], void *T, void *T2,
            const void *Ci, igg_dtype dtype, double lam, double dt, double dx,
            double dy, double dz, void *stream);

/* Fig. 1's solver end to end for callers whose fields live in host memory:
 * on `stream`, copy T0 from T_host into the device buffer T and Ci from
 * Ci_host into Ci, set T2 = copy(T) on the device (Fig. 1), run igg_run's
 * nt steps (widths as there), and copy the newest state back into T_host.
 * T_host and Ci_host hold nsub*nloc elements each in the fields' layout
 * [nsub][nz][ny][nx]; page-locked host memory keeps the copies asynchronous
 * (pageable memory works, but its copies block the calling thread). T, T2
 * and Ci are the caller's device buffers (16-byte aligned, overwritten).
 * The call only enqueues: synchronise `stream` before reading T_host.
 * Errors: IGG_EINVAL for NULL host pointers and igg_run's conditions;
 * IGG_ECUDA if a copy cannot be enqueued. */
int igg_run_host(igg_grid *grid, int nt, const int widths[3], void *T_host,
                 const void *Ci_host, void *T, void *T2, void *Ci, igg_dtype dtype,
                 double lam, double dt, double dx, double dy, double dz,
                 void *stream);

/* ---------------------------------------------------------------------------
 * Staggered-grid acoustics: a multi-field stencil on the grid's regular
 * staggered layout (Sec. Approach), with fields of different sizes per
 * subdomain: P at cells [nsub][nz][ny][nx], Vx at x faces
 * [nsub][nz][ny][nx+1], Vy [nsub][nz][ny+1][nx], Vz [nsub][nz+1][ny][nx].
 * One leapfrog step, in this order:
 *   Vx[i] -= dt/rho*(P[i] - P[i-1])/dx on faces i = 1..nx-1 (all y, z), and
 *   likewise Vy, Vz (the outermost faces are never written: walls, or halo
 *   faces that the halo update fills);
 *   P -= dt*K*((Vx[i+1]-Vx[i])/dx + (Vy[j+1]-Vy[j])/dy + (Vz[k+1]-Vz[k])/dz)
 *   on every cell, with the new velocities;
 * then, if with_halo, update_halo!(P, Vx, Vy, Vz) as igg_update_halo_fields
 * (overlaps o for P and o+1 for each face field in its own dimension): its x
 * exchange is done by the two launches themselves (each sent x plane stored
 * a second time into the neighbour's halo plane, the neighbour's halo cells
 * not stored by their own threads), then the y and z exchanges, with the
 * same result as the plane copies in the order x, y, z. dtype
 * F64 or F32. Coefficients dt/(rho*dd) and dt*K/dd are formed in FP64; the
 * kernels use one FMA per term (P - bx dVx - by dVy - bz dVz, results within
 * rounding of the left-to-right formula).
 * ------------------------------------------------------------------------- */
int igg_acoustic_step(igg_grid *grid, void *P, void *Vx, void *Vy, void *Vz,
                      igg_dtype dtype, double rho, double K, double dt, double dx,
                      double dy, double dz, int with_halo, void *stream);

/* ---------------------------------------------------------------------------
 * Gross-Pitaevskii solver (the quantum-fluid application named in the
 * paper's conclusion, which prints no equations; these are the library's):
 *   i dpsi/dt = -1/2 lap(psi) + V psi + g |psi|^2 psi,  psi = u + i v,
 * u and v real fields of the grid's layout (u at whole, v at half time
 * steps), V a real potential of the same layout, psi fixed on each array's
 * boundary. One step: u += dt*H(v) on inner points, update_halo!(u) if
 * with_halo, v -= dt*H(u) with the new u, update_halo!(v) if with_halo,
 * where H w = -1/2 lap(w) + (V + g*(u^2 + v^2)) w, the density taken from
 * the values at hand (old u in the first half, new u in the second), lap the
 * 7-point operator with spacings dx, dy, dz (+inf for an absent dimension).
 * Stable for dt below 2 / (2 (1/dx^2 + 1/dy^2 + 1/dz^2) + max(V + g rho)).
 * dtype F64 or F32. F32 fields: FMAs (within rounding of the oracle's
 * left-to-right evaluation). F64 fields: each half-step update (q =
 * dt (V + g rho) and the seven terms) is formed in float pairs (~48-bit
 * significands) and rounded once to FP64, within about 2^-45 of |u or v| plus
 * the magnitudes of the terms; points whose values leave the pair ranges
 * (|u|, |v|, |V| outside [2^-40, 2^41), |q| outside [2^-36, 2^37), zero
 * allowed) use the FP64 formula. 3-D grids whose rows are a multiple of 16
 * bytes (and 16-byte aligned fields) run a TMA-pipelined kernel unless
 * IGG_OPT_TMA is 0; other grids a column kernel with the same bits. With the
 * halo update, the TMA kernel does its x exchange itself (the points of the
 * sent x planes stored a second time into the neighbours' halo columns) and
 * the halo launch copies the face rows only: the same halo values.
 * ------------------------------------------------------------------------- */
int igg_gp_step(igg_grid *grid, void *u, void *v, const void *V, igg_dtype dtype,
                double g, double dt, double dx, double dy, double dz, int with_halo,
                void *stream);

/* ---------------------------------------------------------------------------
 * Batched form: nprob independent diffusion problems of uneven sizes (each
 * Fig. 1's step! on one array with fixed boundary values, its own lam, dt,
 * dx, dy, dz), advanced together by ONE persistent kernel launch per step.
 *
 * Layout: every field of the batch is one device buffer; problem b is an
 * array [nz_b][ny_b][pitch_b] (x fastest; rows padded to pitch_b >= nx_b
 * elements, pitch_b * element size a multiple of 16 bytes, igg_batch_pitches)
 * starting at element offset offsets[b] (igg_batch_layout), each offset a
 * multiple of 256 bytes; point (x, y, z) of problem b is element
 * offsets[b] + x + pitch_b*(y + ny_b*z). The buffer holds `total` elements of
 * the dtype. Row padding and gaps between problems are never written.
 * ------------------------------------------------------------------------- */

/* sizes: nprob triples (nx, ny, nz), each >= 3. Creates the tile table of
 * the default kernel (variant 4, else 3; z depth 32 planes). */
int igg_batch_create(int nprob, const int *sizes, igg_dtype dtype,
                     igg_batch **out);

/* Frees the batch (waits for its capture stream). NULL is accepted. */
int igg_batch_destroy(igg_batch *batch);

/* offsets[nprob] (may be NULL) and the total element count of a field. */
int igg_batch_layout(const igg_batch *batch, long long *offsets,
                     long long *total);

/* pitches[nprob]: the row pitch of each problem in elements. */
int igg_batch_pitches(const igg_batch *batch, int *pitches);

/* Per-problem coefficients from host arrays of nprob doubles each; required
 * before the first step. */
int igg_batch_set_coefs(igg_batch *batch, const double *lam, const double *dt,
                        const double *dx, const double *dy, const double *dz);

/* Kernel and tiling: variant 4 = the TMA-pipelined kernel over every
 * problem's tiles (per-problem tensor maps, encoded on the first step with a
 * pair of field pointers and kept on the batch; ctas_per_sm must be 0;
 * IGG_EINVAL without the driver's tensor-map encoder; the default where it
 * is available); variant 3 = the 16-byte vector kernel,
 * one CTA per tile of 8 warps of row segments (ctas_per_sm must be 0);
 * variants 0, 1, 2 = the persistent scalar kernel with 32x8, 32x4, 64x4
 * columns per tile and ctas_per_sm CTAs per SM (0 = as many as are
 * resident; more than resident gives IGG_EINVAL). zb = z planes per tile (0 =
 * the whole problem depth). The arithmetic does not depend on the kernel or
 * the tiling: every configuration gives the same bits. */
int igg_batch_configure(igg_batch *batch, int variant, int zb, int ctas_per_sm);

/* Current tiling {variant, zb, ctas_per_sm} and the number of tiles. */
int igg_batch_get_config(const igg_batch *batch, int cfg[3], int *ntiles);

/* One step of every problem: T2 = step(T) on inner points (layout above). */
int igg_batch_step(igg_batch *batch, void *T2, const void *T, const void *Ci,
                   void *stream);

/* nt steps with swaps, captured once into a CUDA graph (two steps per
 * launch, cached for the same pointers); newest state in T for even nt and
 * in T2 for odd nt. T2 must hold T's boundary values on entry. */
int igg_batch_run(igg_batch *batch, int nt, void *T, void *T2, const void *Ci,
                  void *stream);

/* Autotuner: times every tiling (3 tile shapes x z depths {8,16,32,64,all}
 * x {resident, half of resident} CTAs per SM) for `reps` steps T -> T2 on the
 * caller's fields, on `stream`, keeps the fastest and returns it in
 * best_cfg[3] with its time per step in *best_ms. Writes T2's inner points
 * and synchronises `stream`. reps = 0 times 3 steps.
 * The choice is cached per (GPU name, dtype, problem sizes): in the process,
 * and in the file named by the environment variable IGG_AUTOTUNE_CACHE when
 * it is set (lines appended, read once per process). A call whose key is
 * cached applies the cached tiling without timing anything (T2 untouched;
 * *best_ms = the cached time); reps < 0 ignores the cache, times 3 steps and
 * stores the new choice. */
int igg_batch_autotune(igg_batch *batch, void *T2, const void *T,
                       const void *Ci, int reps, void *stream, int best_cfg[3],
                       float *best_ms);

/* ---------------------------------------------------------------------------
 * Adjoint form: gradients of a function J(T_nt) of the state after nt steps
 * of Fig. 1's loop with respect to Ci and to the initial state T_0 (the
 * differentiated solver; dt is held fixed). 3-D grids of any topology
 * (periodic and decomposed included); F64 or F32 fields; the Ci gradient is
 * accumulated in FP64. J is a function of every entry of the decomposed
 * field (halo and overlap entries included), and the gradients are per
 * entry of the decomposed T0 and Ci.
 *
 * Forward step on the inner points p of every subdomain: T_{n+1}[p] =
 * T_n[p] + Ci[p]*l(T_n)[p], l(T)[p] = sum_d w_d (T[p-e_d] + T[p+e_d] -
 * 2 T[p]), w_d = dt*lam/dd^2; the other points are unchanged; then the halo
 * update. So a step is H(S(T)) and its adjoint S^T(H^T(lam)):
 * igg_update_halo_adjoint applies H^T, igg_adjoint_step S^T.
 *
 * Arithmetic of a step: F32 fields in F32 with FMAs, the gCi increment in
 * FP64 from the two F32 factors. F64 fields: lam_out is formed in float pairs
 * (~48-bit significands) as a compensated dot product and rounded once to
 * FP64, within about 2^-45 of |lam_in| + sum |w v| (points whose stencil
 * holds |lam| outside [2^-40, 2^41) or Ci outside [2^-20, 2^21), zero
 * allowed, or with weights outside [2^-18, 2^18], use the FP64 sum); l(T_n)
 * for gCi from exact integer second differences where the stencil shares
 * sign and crosses at most one power of two, else in FP64. Rows of a
 * multiple of 16 bytes with 16-byte aligned fields run a TMA-pipelined
 * kernel unless IGG_OPT_TMA is 0; other rows a tiled kernel with the same
 * bits.
 * ------------------------------------------------------------------------- */

/* One backward step. lam_in = dJ/dT_{n+1}; writes lam_out = dJ/dT_n on
 * every point:
 *   v = Ci*lam_in on inner points, 0 elsewhere,
 *   lam_out[q] = lam_in[q] + sum_d w_d (v[q-e_d] + v[q+e_d] - 2 v[q])
 * (neighbours outside the array count as 0), and accumulates
 *   gCi[p] += lam_in[p] * l(T_n)[p] on inner points p (gCi: FP64 array),
 * on every subdomain (one launch each; fields of the grid's shape).
 * lam_out must not alias lam_in. On a grid with halos, apply
 * igg_update_halo_adjoint to lam_in first for the adjoint of a whole step. */
int igg_adjoint_step(igg_grid *grid, void *lam_out, const void *lam_in,
                     const void *T_n, const void *Ci, double *gCi,
                     igg_dtype dtype, double lam, double dt, double dx,
                     double dy, double dz, void *stream);

/* The transpose of update_halo! (the halo update of a field of the grid's
 * own size), in place on an F64 or F32 field lam: the halo update is a
 * product of plane copies field[dst] = field[src], dimensions x, then y,
 * then z; its transpose takes the dimensions z, then y, then x and, for each
 * copy, adds lam[dst] into lam[src] and sets lam[dst] to 0. No counterpart
 * in the paper, which differentiates nothing: the halo part of the adjoint
 * of Fig. 1's loop on the implicit global grid. */
int igg_update_halo_adjoint(igg_grid *grid, void *lam, igg_dtype dtype, void *stream);

/* Number of checkpoints of an nt-step run with one checkpoint every `every`
 * steps: the states T_0, T_every, T_2every, ... before step nt, i.e.
 * ceil(nt/every). Returns the count (> 0) or IGG_EINVAL. */
int igg_checkpoint_slots(int nt, int every);

/* Forward run that keeps checkpoints: nt steps of Fig. 1's loop (step, then
 * the halo update on grids with halos) from T0 (physical boundary values of
 * T0 stay fixed), storing state T_{k*every} in slot k of `ckpt`
 * (igg_checkpoint_slots fields, contiguous) and T_nt in T_out. `work` holds
 * two fields (scratch of the caller). */
int igg_forward_checkpointed(igg_grid *grid, int nt, int every, const void *T0,
                             const void *Ci, igg_dtype dtype, double lam,
                             double dt, double dx, double dy, double dz,
                             void *ckpt, void *work, void *T_out, void *stream);

/* Backward run: from lam_nt = dJ/dT_nt and the checkpoints of
 * igg_forward_checkpointed, recomputes each segment of `every` states from
 * its checkpoint (into `seg`, every-1 fields; unused when every == 1) and
 * runs the adjoint steps backward in time (H^T, then S^T per subdomain).
 * Writes gT0 = dJ/dT_0 (dtype field) and gCi = dJ/dCi (FP64 field,
 * overwritten). `work` holds two fields.
 * Memory: (ceil(nt/every) + every + 3) fields instead of nt + 1; F64 fields
 * on the TMA kernel also take, for the run, a scratch of 8 bytes per point
 * (Ci as float pairs) from the stream-ordered allocator on `stream`. */
int igg_adjoint_checkpointed(igg_grid *grid, int nt, int every,
                             const void *ckpt, const void *Ci,
                             const void *lam_nt, igg_dtype dtype, double lam,
                             double dt, double dx, double dy, double dz,
                             void *seg, void *work, void *gT0, double *gCi,
                             void *stream);

/* out = a - b over n elements (F64 or F32): the gradient T_nt - T_obs of the
 * misfit 0.5*sum((T_nt - T_obs)^2), whose value is 0.5*igg_reduce(
 * IGG_RED_SUM_SQDIFF, T_nt, T_obs). out may alias a. */
int igg_residual(void *out, const void *a, const void *b, size_t n,
                 igg_dtype dtype, void *stream);

/* ---------------------------------------------------------------------------
 * FP64 reductions over n elements of device arrays of `dtype` (used for
 * Fig. 1's maximum(Ci) in the time-step rule and for the checks and the
 * misfit loss):
 *   IGG_RED_MAX      : max_i a[i]                     (b unused)
 *   IGG_RED_SUM      : sum_i a[i]
 *   IGG_RED_SUM_DIV  : sum_i a[i]/b[i]                 (heat content T/Ci)
 *   IGG_RED_SUM_SQDIFF: sum_i (a[i]-b[i])^2
 * Every term is formed and accumulated in FP64 with a fixed order (per-block
 * partial sums in a scratch buffer, then one block combines them), so the
 * result is deterministic. *out_dev is a device pointer to one double that
 * receives the result. The partial sums go to a scratch buffer of at most
 * 1024 doubles taken from the stream-ordered allocator (cudaMallocAsync on
 * `stream`) and released on `stream` after use.
 * ------------------------------------------------------------------------- */
#define IGG_RED_MAX 0
#define IGG_RED_SUM 1
#define IGG_RED_SUM_DIV 2
#define IGG_RED_SUM_SQDIFF 3
int igg_reduce(int op, const void *a, const void *b, size_t n, igg_dtype dtype,
               double *out_dev, void *stream);

/* ---------------------------------------------------------------------------
 * The same reductions without any device allocation. The paper has no
 * counterpart; this entry point exists for callers that cannot allocate
 * device memory at the time they reduce: code running under an allocator
 * that owns all device memory or forbids growth, host callbacks and
 * real-time loops with a fixed memory budget, or stream-capture regions
 * where allocation calls are not allowed.
 *
 * Arguments, ops and dtypes as igg_reduce. Each block of the first kernel
 * reduces one contiguous chunk of 65536 elements, so the summation order
 * (and possibly the last bits of a sum) differ from igg_reduce's; IGG_RED_MAX
 * is exact either way. The partial sums live in a file-scope device array
 * of 32768 doubles (256 KB) that every GPU loading the library holds until
 * the process exits; n above 32768*65536 = 2^31 elements gives IGG_EINVAL.
 * The function calls no cudaMalloc, cudaMallocAsync, cudaFree or other
 * allocating routine. The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress, once per device, with that device current);
 * make that first call before any stream capture. All calls share the one
 * array: calls whose work can overlap on the GPU (different streams, or
 * several host threads) race and must be ordered by the caller. The array
 * keeps the last call's contents; every partial sum a call reads is written
 * by that call first, so nothing has to start at zero.
 * ------------------------------------------------------------------------- */
int igg_reduce_noalloc(int op, const void *a, const void *b, size_t n,
                       igg_dtype dtype, double *out_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* IGG_H */
