// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <vector>

#include "../../include/igg.h"

namespace igg {

// Tile of work for one CTA of the stencil kernels: the columns x0 <= x < xe,
// y0 <= y < ye (at most kTileX x kTileY of them) of one local array, swept
// over z0 <= z < z1. All indices are local to the array; `base` is the
// element offset of the array inside the field buffer. Every point of a tile
// is an inner point of its array.
// In the vector kernels x0 is the (16-byte aligned) first point of lane 0's
// vector and the tile computes the points xb <= x < xe; in the scalar kernels
// xb = x0.
struct Tile {
  long long base;
  int nx, ny;
  int x0, y0, xe, ye;
  int z0, z1;
  int param;  // row of the coefficient table (batched form), else 0
  int xb;
};
static_assert(sizeof(Tile) == 48, "Tile layout");

// Tile extents (threads of a CTA are kTileX x kTileY, one column each).
constexpr int kTileX = 32;
constexpr int kTileY = 8;

// Coefficients of the update T2 = T + Ci*(wx*(Txm+Txp) + wy*(Tym+Typ) +
// wz*(Tzm+Tzp) + wc*T), with w_d = dt*lam/dd^2 and wc = -2*(wx+wy+wz),
// all formed on the host in FP64.
struct Coef {
  double wx, wy, wz, wc;
  int f64_emu;  // FP64 fields: 1 = emulated FP64 cell, 0 = FP64 cell
  // TMA full steps followed by a halo update: the row end cells x = 0 and
  // x = n_x - 1 of every computed row are stored as well, with their values
  // in T (boundary cells keep them; halo cells are overwritten by the halo
  // update), so that every row store covers whole 32-byte sectors
  int ends;
  // points of the field the launch writes (all subdomains), set by the TMA
  // launcher; the bounds-checked build tests global indices against it
  long long npts;
};

Coef make_coef(double lam, double dt, double dx, double dy, double dz);

// Weight groups of the emulated FP64 cell: 1 when wx == wy == wz, 2 when
// wy == wz only (the second differences of equal weights are added exactly
// before the product), else 3.
__host__ __device__ inline int weight_groups(double wx, double wy, double wz) {
  return (wx == wy && wy == wz) ? 1 : (wy == wz ? 2 : 3);
}

// The emulated FP64 cell takes weights of magnitude at most 2^40 (its fast
// path's FP32 products then stay finite); other weights use the FP64 cell.
inline bool emu_weights_ok(const Coef &c) {
  const double lim = 1099511627776.0;  // 2^40
  return fabs(c.wx) <= lim && fabs(c.wy) <= lim && fabs(c.wz) <= lim;
}

// One face-plane copy of the halo update: the plane whose point with both
// in-plane indices 0 is at element offset `src` is copied onto the plane at
// `dst` (same in-plane geometry).
struct PlaneCopy {
  long long dst, src;
};

// error reporting (thread-local message)
int set_error(int code, const char *fmt, ...);
int cuda_error(cudaError_t e, const char *what);
void clear_error();

size_t dtype_size(igg_dtype t);

// kernel launchers (no synchronisation; errors from cudaGetLastError)
cudaError_t launch_stencil(igg_dtype dt, const Tile *tiles, int ntiles, void *T2,
                           const void *T, const void *Ci, const Coef &c,
                           const Coef *table, cudaStream_t s);

// Tile of the vector kernel. Each thread holds V = 16/sizeof(element)
// consecutive points of a row as one 16-byte vector; a row of the tile is a
// segment of lpr = 2^lpr_log2 lanes (lpr*V points), a warp holds 32/lpr rows
// and a CTA kVecWarps warps. Rows are the index r of stride `sr` elements and
// the tile marches over the index m of stride `sm`: rows along y and march
// along z normally, or (swap = 1) rows along z and march along y for boxes
// thin in y. The tile computes the points xb <= x < xe, rows r0 <= r < re,
// marching m0 <= m < m1; lane 0 of a row starts at x0 (a multiple of V).
struct VTile {
  long long base;
  long long sr, sm;
  int nx;
  int x0, xb, xe;
  int r0, re;
  int m0, m1;
  int param;
  unsigned short lpr_log2, swap;
};
static_assert(sizeof(VTile) == 64, "VTile layout");
constexpr int kVecWarps = 8;
// Vector-kernel tiles of the box [x0,x1) x [y0,y1) x [z0,z1) of one array
// [nz][ny][pitch] (rows of pitch >= nx elements, 16-byte aligned) at element
// offset base; zb planes per tile, coefficient-table row param.
void add_box_vec_pitched(std::vector<VTile> &v, long long base, int nx, int pitch, int ny, int x0,
                         int x1, int y0, int y1, int z0, int z1, int zb, int param, int V);
int vec_width(igg_dtype dt);  // V
cudaError_t launch_stencil_vec(igg_dtype dt, const VTile *tiles, int ntiles, void *T2,
                               const void *T, const void *Ci, const Coef &c,
                               const Coef *table, cudaStream_t s);

// Persistent tile-table kernel of the batched form: `variant` selects the
// tile shape (persistent_tile_shape), nctas the number of CTAs that stride
// over the tiles. table[tile.param] holds each tile's coefficients.
constexpr int kPersistentVariants = 3;
void persistent_tile_shape(int variant, int *tx, int *ty);
int persistent_occupancy(igg_dtype dt, int variant);  // resident CTAs per SM (0 on error)
cudaError_t launch_stencil_persistent(igg_dtype dt, int variant, const Tile *tiles, int ntiles,
                                      int nctas, void *T2, const void *T, const void *Ci,
                                      const Coef *table, cudaStream_t s);

// TMA-pipelined kernel. A tile computes xb <= x < xe (lane 0 of a row at x0,
// a multiple of V; the tile spans tma_tile_width points), rows r0 <= r < re
// (at most tma_tile_rows) and march steps m0 <= m < m1 of the array at
// element offset `base`, which starts at plane zoff of the field seen as one
// stack of nsub*nz planes. Variants: TMA_WIDE (rows along y, march along z)
// and TMA_WIDE_SWAP (rows along z, march along y, for y slabs).
struct TmaTile {
  long long base;
  int x0, xb, xe;
  int r0, re;
  int m0, m1;
  int zoff;
  int pad[2];
};
enum { TMA_WIDE = 0, TMA_WIDE_SWAP = 2 };
// TMA tiles of the box [x0,x1) x rows [r0,r1) x march [m0,m1) (chunks of mb
// planes) of one array at element offset base whose planes start at plane
// zoff of the tensor map; tile width Wt, rows Ht, vector width V.
void add_box_tma(std::vector<TmaTile> &v, long long base, long long zoff, int x0, int x1, int r0,
                 int r1, int m0, int m1, int mb, int V, int Wt, int Ht);
// Batched form on the TMA kernel: per problem two tensor maps (T, Ci) in
// device memory, its row pitch and ny, its coefficients; a tile's problem
// is its pad[0]. Maps are 128-byte opaque blocks here (CUtensorMap in tma.cu).
struct alignas(64) TmaMapBytes {
  unsigned char b[128];
};
struct TmaBatch {
  const TmaMapBytes *maps;  // [2 * nprob]: T, Ci
  const int *geom;          // [2 * nprob]: row pitch, ny
  const Coef *coef;         // [nprob]
};
// Encodes the 2*nprob maps of fields T and Ci (problem b at element offset
// off[b], size sizes[3b..3b+2], row pitch pitch[b]) into host memory out.
bool tma_batch_maps(igg_dtype dt, const void *T, const void *Ci, int nprob,
                    const long long *off, const int *sizes, const int *pitch, TmaMapBytes *out);
cudaError_t tma_batch_prepare(igg_dtype dt);
cudaError_t launch_stencil_tma_batch(igg_dtype dt, const TmaTile *tiles, int ntiles, void *T2,
                                     const TmaBatch &b, unsigned *dev_err, cudaStream_t s);
static_assert(sizeof(TmaTile) == 48, "TmaTile layout");
// bits of the device error word: IGG_DEV_ERR_TIMEOUT, IGG_DEV_ERR_DRAIN (igg.h)
int tma_tile_width(igg_dtype dt, int variant);
int tma_tile_rows(igg_dtype dt, int variant);
bool tma_available();
// Sets the kernel's shared-memory attribute and returns its resident CTAs per
// SM; call before launching (and before any stream capture).
cudaError_t tma_prepare(igg_dtype dt, int variant, int *ctas_per_sm);
// Fix-up buffer of an FP64 tile set of the TMA kernel (emulated cell): room
// for cap entries of 16 bytes (one per 32-point row segment with points left
// to the fix-up, so cap = the set's computed points / 32 suffices), then the
// entry count and a block counter, both zero on entry, then two 64-bit
// totals (segments and points fixed up so far). The kernel fills it; the
// fix-up launch that follows on the same stream updates the listed points,
// adds to the totals and resets the count and the counter.
struct FixBuf {
  void *p = nullptr;
  size_t cap = 0;
};
size_t tma_fix_cap(const TmaTile *tiles, int ntiles);
inline size_t tma_fix_bytes(size_t cap) { return cap * 16 + 2 * sizeof(unsigned) + 16; }
cudaError_t launch_stencil_tma(igg_dtype dt, int variant, const TmaTile *tiles, int ntiles,
                               void *T2, const void *T, const void *Ci, int nx, int ny,
                               long long nzt, const Coef &c, unsigned *dev_err,
                               FixBuf fix, cudaStream_t s);

// Staggered-grid acoustics (acoustic.cu): coefficients dt/(rho dd) of the
// velocity update and dt K/dd of the pressure update, formed on the host in
// FP64; one step (velocities, then pressure) on every subdomain.
struct AcCoef {
  double ax, ay, az, bx, by, bz;
  // x exchange by the launches (acoustic.cu): the grid's neighbour table
  // (6 per subdomain: left/right per dimension, -1 none) and x overlap
  const int *nbr = nullptr;
  int ox = 2, xsend = 0;
};
cudaError_t launch_acoustic(igg_dtype dt, int nsub, int nx, int ny, int nz, void *P, void *Vx,
                            void *Vy, void *Vz, const AcCoef &c, cudaStream_t s);

// Gross-Pitaevskii half steps (gp.cu): kd = -dt/(2 dd^2) (0 for an absent
// dimension), kc = -2 (kx + ky + kz), dt and g, formed on the host in FP64.
struct GpCoef {
  double kx, ky, kz, kc, dt, g;
  // x exchange by the TMA half-step launch (gp.cu): the grid's neighbour
  // table (6 per subdomain, -1 none) and x overlap
  const int *nbr = nullptr;
  int ox = 2, xsend = 0;
};
// With `tma`, 3-D grids whose rows allow it take the TMA-pipelined kernel;
// *xsent = true when that kernel ran with c.xsend (it stored the x planes
// that the halo update sends into the neighbours' halo columns).
cudaError_t launch_gp_half(igg_dtype dt, int which, int nsub, int nx, int ny, int nz, void *u,
                           void *v, const void *V, const GpCoef &c, bool tma, unsigned *dev_err,
                           cudaStream_t s, bool *xsent);

// One dimension of the halo update for one field: ncopies plane copies,
// each plane having na x nb points with element strides sa, sb.
// The copies of one dimension of up to kMaxHaloJobs fields in one launch
// (fields of different sizes: each job its own plane table and geometry as
// for launch_halo; vec is set by the launch).
constexpr int kMaxHaloJobs = 16;

// Bounds-checked build (compiled with -DIGG_BOUNDS_CHECK into a library of its
// own): the kernels of the default step (the TMA stencil's stores, the fix-up
// launch, the one-launch halo update) test each global index against the
// extent of its field before the access. A failing test skips the access
// and sets the translation unit's flag, which igg_bounds_status reads: the
// kernel does not trap and the context stays usable. In the release build
// the tests compile to nothing.
#ifdef IGG_BOUNDS_CHECK
static __device__ unsigned g_bounds_flag;
__device__ __forceinline__ bool in_bounds(long long i, long long n) {
  if (i >= 0 && i < n) return true;
  atomicOr(&g_bounds_flag, 1u);
  return false;
}
static inline cudaError_t read_bounds_flag(unsigned *out, bool clear) {
  cudaError_t e = cudaMemcpyFromSymbol(out, g_bounds_flag, sizeof(unsigned));
  const unsigned zero = 0u;
  if (e == cudaSuccess && clear) e = cudaMemcpyToSymbol(g_bounds_flag, &zero, sizeof zero);
  return e;
}
#else
__device__ __forceinline__ bool in_bounds(long long, long long) { return true; }
static inline cudaError_t read_bounds_flag(unsigned *out, bool) {
  *out = 0u;
  return cudaSuccess;
}
#endif
// the flags of the translation units with checked kernels
cudaError_t tma_bounds_flag(unsigned *out, bool clear);
cudaError_t halo_bounds_flag(unsigned *out, bool clear);
struct HaloJob {
  const PlaneCopy *copies;
  void *field;
  long long sa, sb;
  int ncopies, na, nb, vec;
};
struct HaloJobs {
  HaloJob j[kMaxHaloJobs];
};
cudaError_t launch_halo_jobs(size_t elem_size, HaloJobs jobs, int njobs, cudaStream_t s);
cudaError_t launch_halo(size_t elem_size, const PlaneCopy *copies, int ncopies,
                        void *field, int na, int nb, long long sa, long long sb,
                        cudaStream_t s);
// The halo update of a field of the grid's own size (3-D grids) in one
// launch (the gather form, halo.cu): nbr[6 sub + 2 d + side] is the left
// (side 0) or right (side 1) neighbour in dimension d, -1 none.
struct HaloGather {
  const int *nbr = nullptr;
  int n[3] = {0, 0, 0}, o[3] = {0, 0, 0};
  long long nloc = 0;
  int nsub = 0;
  // 1: the x-face columns with y, z inner are already filled (the launch
  // before stored its sent x planes into them); only the face rows are copied
  int skipx = 0;
};
cudaError_t launch_halo_gather(size_t elem_size, void *field, const HaloGather &h,
                               cudaStream_t s);
// The transpose of one dimension's plane copies on an F64 (elem_size 8) or
// F32 (4) field: field[src] += field[dst], field[dst] = 0 (halo.cu).
cudaError_t launch_halo_adjoint(size_t elem_size, const PlaneCopy *copies, int ncopies,
                                void *field, int na, int nb, long long sa, long long sb,
                                cudaStream_t s);

// Adjoint step over every point of one array, and out = a - b elementwise.
// With `tma`, fields that allow it take the TMA-pipelined kernel; FP64 fields
// with `ci_pairs` (Ci as pairs from launch_pair_ci, n elements of 8 bytes)
// load those instead of splitting Ci (same results).
cudaError_t launch_adjoint(igg_dtype dt, int nx, int ny, int nz, void *lam_out,
                           const void *lam_in, const void *Tn, const void *Ci, double *gCi,
                           const Coef &c, bool tma, unsigned *dev_err, cudaStream_t s,
                           const void *ci_pairs = nullptr);
// TMA adjoint kernel: applies to F64/F32 rows of a multiple of 16 bytes and
// 16-byte aligned fields (and a driver with tensor maps).
bool adjoint_tma_applies(igg_dtype dt, int nx, const void *lam_out, const void *lam_in,
                         const void *Tn, const void *Ci, const double *gCi);
cudaError_t launch_adjoint_tma(igg_dtype dt, int nx, int ny, int nz, void *lam_out,
                               const void *lam_in, const void *Tn, const void *Ci, double *gCi,
                               const Coef &c, unsigned *dev_err, cudaStream_t s,
                               const void *ci_pairs = nullptr);
// FP64 Ci (n values) as pairs for the adjoint kernel (8 bytes each)
cudaError_t launch_pair_ci(const void *Ci, void *pairs, long long n, cudaStream_t s);
cudaError_t launch_sub(igg_dtype dt, long long n, void *out, const void *a, const void *b,
                       cudaStream_t s);

cudaError_t launch_reduce(int op, const void *a, const void *b, size_t n,
                          igg_dtype dt, double *scratch, int nblocks,
                          double *out, cudaStream_t s);

}  // namespace igg
