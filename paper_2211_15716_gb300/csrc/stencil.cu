// Stencil kernels: Fig. 1's step! on lists of tiles.
//
// One kernel serves the full step, the boundary slabs and the inner block of
// the hidden step, and the batched form: the host turns each of them into a
// table of tiles, and every CTA sweeps one tile along z with the three z
// planes of its column kept in registers (z-marching). The x and y
// neighbours are read through the read-only data cache, where the
// neighbouring columns of the same CTA have just brought them.
//
// Arithmetic (identical in every launch, so every kernel gives the same bits
// for the same point):
//   FP64: s_d = T[-d] + T[+d];  l = wc*T;  l += wx*s_x;  l += wy*s_y;
//         l += wz*s_z;  T2 = T + Ci*l  (FMA where written, round-to-nearest
//         intrinsics so that no other contraction can happen).
//   FP32 / BF16 storage: the differences are formed first, which is exact
//   for neighbouring values within a factor 2:
//         e_d = (T[+d] - T) + (T[-d] - T);  l = wx*e_x;  l += wy*e_y;
//         l += wz*e_z;  T2 = T + Ci*l.
// No CUDA math-library function is used: only + - * and FMA.
#include <cuda_bf16.h>

#include "cell.cuh"
#include "igg_internal.h"

namespace igg {
namespace {

// Sweep one tile along z: every thread owns one (x, y) column of the tile,
// keeps T at z-1, z, z+1 in registers and reads x/y neighbours through the
// read-only cache.
template <class S>
__device__ __forceinline__ void sweep_tile(const Tile &t, int tx, int ty, S *__restrict__ T2,
                                           const S *__restrict__ T, const S *__restrict__ Ci,
                                           const W<typename Num<S>::C> &w) {
  using N = Num<S>;
  using C = typename N::C;
  const int x = t.x0 + tx;
  const int y = t.y0 + ty;
  if (x >= t.xe || y >= t.ye) return;
  // absent dimensions (2-D and 1-D grids: ny = 1, or z range [0, 1)) have a
  // zero neighbour stride
  const long long sy = t.ny > 1 ? t.nx : 0;
  const long long sz = t.z0 > 0 ? (long long)t.nx * t.ny : 0;
  long long p = t.base + x + sy * y + sz * (t.z0 - 1);
  C zm = N::ld(T + p);
  C zc = N::ld(T + p + sz);
  for (int z = t.z0; z < t.z1; ++z) {
    p += sz;
    const C zp = N::ld(T + p + sz);
    const C xm = N::ld(T + p - 1);
    const C xp = N::ld(T + p + 1);
    const C ym = N::ld(T + p - sy);
    const C yp = N::ld(T + p + sy);
    const C ci = N::ld(Ci + p);
    N::st(T2 + p, cell(zc, xm, xp, ym, yp, zm, zp, ci, w));
    zm = zc;
    zc = zp;
  }
}

// One CTA per tile.
template <class S>
__global__ void __launch_bounds__(kTileX *kTileY)
    k_stencil_tiles(const Tile *__restrict__ tiles, S *__restrict__ T2,
                    const S *__restrict__ T, const S *__restrict__ Ci, Coef c0,
                    const Coef *__restrict__ table) {
  using C = typename Num<S>::C;
  const Tile t = tiles[blockIdx.x];
  const W<C> w = make_w(table ? table[t.param] : c0, C(0));
  sweep_tile<S>(t, (int)threadIdx.x, (int)threadIdx.y, T2, T, Ci, w);
}

// Persistent form: a fixed grid of CTAs strides over the tile table (the
// batched form's one launch per step). Tiles of TX x TY columns.
template <class S, int TX, int TY>
__global__ void __launch_bounds__(TX *TY)
    k_stencil_persistent(const Tile *__restrict__ tiles, int ntiles, S *__restrict__ T2,
                         const S *__restrict__ T, const S *__restrict__ Ci,
                         const Coef *__restrict__ table) {
  using C = typename Num<S>::C;
  const int tx = (int)(threadIdx.x % TX), ty = (int)(threadIdx.x / TX);
  for (int i = blockIdx.x; i < ntiles; i += gridDim.x) {
    const Tile t = tiles[i];
    const W<C> w = make_w(table[t.param], C(0));
    sweep_tile<S>(t, tx, ty, T2, T, Ci, w);
  }
}

template <class S>
cudaError_t launch_persistent_t(int variant, const Tile *tiles, int ntiles, int nctas, void *T2,
                                const void *T, const void *Ci, const Coef *table,
                                cudaStream_t s) {
  switch (variant) {
    case 0:
      k_stencil_persistent<S, 32, 8><<<nctas, 256, 0, s>>>(tiles, ntiles, (S *)T2, (const S *)T,
                                                          (const S *)Ci, table);
      break;
    case 1:
      k_stencil_persistent<S, 32, 4><<<nctas, 128, 0, s>>>(tiles, ntiles, (S *)T2, (const S *)T,
                                                          (const S *)Ci, table);
      break;
    case 2:
      k_stencil_persistent<S, 64, 4><<<nctas, 256, 0, s>>>(tiles, ntiles, (S *)T2, (const S *)T,
                                                          (const S *)Ci, table);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Vector form. One warp per tile row; lane l holds the V = 16/sizeof(S)
// points x0 + l*V .. x0 + l*V + V-1 of that row as one 16-byte vector and
// keeps the planes z-1, z, z+1 of its vector in registers. x neighbours come
// from the neighbouring lane by shuffle (lanes 0 and 31 load the one point
// beyond the warp), y neighbours are 16-byte loads of the rows above and
// below (cache hits: the neighbouring warps load those rows as their own).
// Only points with xb <= x < xe are written; a vector with every point
// inside is stored whole, otherwise point by point.
// ---------------------------------------------------------------------------
template <class S>
__global__ void __launch_bounds__(32 * kVecWarps)
    k_stencil_vec(const VTile *__restrict__ tiles, S *__restrict__ T2, const S *__restrict__ T,
                  const S *__restrict__ Ci, Coef c0, const Coef *__restrict__ table) {
  using C = typename Num<S>::C;
  constexpr int V = Vec<S>::V;
  const VTile t = tiles[blockIdx.x];
  const W<C> w = make_w(table ? table[t.param] : c0, C(0));
  const int lane = threadIdx.x & 31;
  const int lpr = 1 << t.lpr_log2;
  const int rows_per_warp = 32 >> t.lpr_log2;
  const int row0 = t.r0 + (int)(threadIdx.x >> 5) * rows_per_warp;
  if (row0 >= t.re) return;  // the whole warp has no row of the tile
  const int sl = lane & (lpr - 1);
  const int r = row0 + (lane >> t.lpr_log2);
  const bool row_ok = r < t.re;
  const int xs = t.x0 + sl * V;
  // this lane's vector is needed if it overlaps [xb - 1, xe + 1) inside the row
  const bool need = row_ok && xs < t.nx && xs + V > t.xb - 1 && xs < t.xe + 1;
  const bool comp = row_ok && xs + V > t.xb && xs < t.xe;  // has points to compute
  const long long sr = t.sr, sm = t.sm;
  long long p = t.base + xs + sr * r + sm * (t.m0 - 1);
  Vec<S> mm, mc, mp, rm, rp, ci;
#pragma unroll
  for (int i = 0; i < V; ++i) mm.v[i] = mc.v[i] = mp.v[i] = C(0);
  if (need) {
    ldvec(T + p, mm);
    ldvec(T + p + sm, mc);
  }
  const bool left_ld = sl == 0 && comp && xs > 0;
  const bool right_ld = sl == lpr - 1 && comp && xs + V < t.nx;
  const bool swap = t.swap != 0;
  for (int m = t.m0; m < t.m1; ++m) {
    p += sm;
    if (need) ldvec(T + p + sm, mp);
    if (comp) {
      ldvec(T + p - sr, rm);
      ldvec(T + p + sr, rp);
      ldvec(Ci + p, ci);
    }
    C left = __shfl_up_sync(0xffffffffu, mc.v[V - 1], 1, lpr);
    C right = __shfl_down_sync(0xffffffffu, mc.v[0], 1, lpr);
    if (left_ld) left = ld1(T + p - 1);
    if (right_ld) right = ld1(T + p + V);
    if (comp) {
      Vec<S> out;
#pragma unroll
      for (int i = 0; i < V; ++i) {
        const C xm = i == 0 ? left : mc.v[i - 1];
        const C xp = i == V - 1 ? right : mc.v[i + 1];
        // rows along y: (row pair, march pair) = (y, z); swapped: (z, y)
        const C ym = swap ? mm.v[i] : rm.v[i], yp = swap ? mp.v[i] : rp.v[i];
        const C zm = swap ? rm.v[i] : mm.v[i], zp = swap ? rp.v[i] : mp.v[i];
        out.v[i] = cell(mc.v[i], xm, xp, ym, yp, zm, zp, ci.v[i], w);
      }
      if (xs >= t.xb && xs + V <= t.xe) {
        *reinterpret_cast<uint4 *>(T2 + p) = pack(out);
      } else {
#pragma unroll
        for (int i = 0; i < V; ++i)
          if (xs + i >= t.xb && xs + i < t.xe) Num<S>::st(T2 + p + i, out.v[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < V; ++i) {
      mm.v[i] = mc.v[i];
      mc.v[i] = mp.v[i];
    }
  }
}

}  // namespace

cudaError_t launch_stencil(igg_dtype dt, const Tile *tiles, int ntiles, void *T2,
                           const void *T, const void *Ci, const Coef &c,
                           const Coef *table, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  const dim3 block(kTileX, kTileY);
  switch (dt) {
    case IGG_F64:
      k_stencil_tiles<double><<<ntiles, block, 0, s>>>(
          tiles, (double *)T2, (const double *)T, (const double *)Ci, c, table);
      break;
    case IGG_F32:
      k_stencil_tiles<float><<<ntiles, block, 0, s>>>(
          tiles, (float *)T2, (const float *)T, (const float *)Ci, c, table);
      break;
    case IGG_BF16:
      k_stencil_tiles<__nv_bfloat16><<<ntiles, block, 0, s>>>(
          tiles, (__nv_bfloat16 *)T2, (const __nv_bfloat16 *)T,
          (const __nv_bfloat16 *)Ci, c, table);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <class S>
int occupancy_t(int variant) {
  int n = 0;
  cudaError_t e = cudaErrorInvalidValue;
  switch (variant) {
    case 0:
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_stencil_persistent<S, 32, 8>, 256, 0);
      break;
    case 1:
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_stencil_persistent<S, 32, 4>, 128, 0);
      break;
    case 2:
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_stencil_persistent<S, 64, 4>, 256, 0);
      break;
  }
  return e == cudaSuccess ? n : 0;
}

int persistent_occupancy(igg_dtype dt, int variant) {
  switch (dt) {
    case IGG_F64: return occupancy_t<double>(variant);
    case IGG_F32: return occupancy_t<float>(variant);
    case IGG_BF16: return occupancy_t<__nv_bfloat16>(variant);
  }
  return 0;
}

int vec_width(igg_dtype dt) {
  const size_t s = dtype_size(dt);
  return s ? (int)(16 / s) : 0;
}

cudaError_t launch_stencil_vec(igg_dtype dt, const VTile *tiles, int ntiles, void *T2,
                               const void *T, const void *Ci, const Coef &c,
                               const Coef *table, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  switch (dt) {
    case IGG_F64:
      k_stencil_vec<double><<<ntiles, 32 * kVecWarps, 0, s>>>(
          tiles, (double *)T2, (const double *)T, (const double *)Ci, c, table);
      break;
    case IGG_F32:
      k_stencil_vec<float><<<ntiles, 32 * kVecWarps, 0, s>>>(
          tiles, (float *)T2, (const float *)T, (const float *)Ci, c, table);
      break;
    case IGG_BF16:
      k_stencil_vec<__nv_bfloat16><<<ntiles, 32 * kVecWarps, 0, s>>>(
          tiles, (__nv_bfloat16 *)T2, (const __nv_bfloat16 *)T, (const __nv_bfloat16 *)Ci, c,
          table);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

void persistent_tile_shape(int variant, int *tx, int *ty) {
  static const int shapes[kPersistentVariants][2] = {{32, 8}, {32, 4}, {64, 4}};
  *tx = shapes[variant][0];
  *ty = shapes[variant][1];
}

cudaError_t launch_stencil_persistent(igg_dtype dt, int variant, const Tile *tiles, int ntiles,
                                      int nctas, void *T2, const void *T, const void *Ci,
                                      const Coef *table, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  if (variant < 0 || variant >= kPersistentVariants || nctas <= 0) return cudaErrorInvalidValue;
  switch (dt) {
    case IGG_F64: return launch_persistent_t<double>(variant, tiles, ntiles, nctas, T2, T, Ci, table, s);
    case IGG_F32: return launch_persistent_t<float>(variant, tiles, ntiles, nctas, T2, T, Ci, table, s);
    case IGG_BF16:
      return launch_persistent_t<__nv_bfloat16>(variant, tiles, ntiles, nctas, T2, T, Ci, table, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace igg
