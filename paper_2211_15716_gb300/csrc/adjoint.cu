// Adjoint of Fig. 1's step! (the transposed stencil run backward in time) and
// the checkpointed drivers' kernels: gradients of a function of T_nt with
// respect to Ci and the initial T. The per-point arithmetic (adj_cell.cuh) is
// shared with the TMA-pipelined adjoint kernel (adjoint_tma.cu); this file
// holds the plain tiled kernel, used where the TMA kernel does not apply
// (rows whose byte length is not a multiple of 16, unaligned fields, TMA
// switched off), and the residual kernel.
#include <algorithm>
#include <cstring>

#include "adj_cell.cuh"
#include "igg_internal.h"

namespace igg {
namespace {

constexpr int kAdjX = 32, kAdjY = 8, kAdjRing = 2 * (kAdjX + 2) + 2 * kAdjY;

__device__ __forceinline__ bool adj_inner(int x, int y, int z, int nx, int ny, int nz) {
  return x >= 1 && x <= nx - 2 && y >= 1 && y <= ny - 2 && z >= 1 && z <= nz - 2;
}

// v at (x, y, z) in FP64 from global memory (the FP64 sum's inputs)
__device__ __forceinline__ double v64_at(const double *__restrict__ lam_in,
                                         const double *__restrict__ Ci, int x, int y, int z,
                                         int nx, int ny, int nz) {
  if (!adj_inner(x, y, z, nx, ny, nz)) return 0.0;
  const long long p = x + (long long)nx * (y + (long long)ny * z);
  return adj_v64(__ldg(lam_in + p), __ldg(Ci + p), true);
}

// One CTA per 32x8 block of (x, y) columns and a chunk of zb planes, every
// point of the array. Per plane, v and T_n of the block and of the ring of
// one point around it go to shared memory (two buffers, one barrier per
// plane); each v is formed once, by the thread of its point or of its ring
// position. The column's planes z-1, z, z+1 stay in registers. Every thread
// runs every plane (the warp votes inside need all lanes); stores are masked.
template <class S>
__global__ void __launch_bounds__(kAdjX *kAdjY)
    k_adjoint(int nx, int ny, int nz, int zb, S *__restrict__ lam_out,
              const S *__restrict__ lam_in, const S *__restrict__ Tn,
              const S *__restrict__ Ci, double *__restrict__ gCi, Coef c) {
  using Ops = AdjOps<S>;
  using VT = typename Ops::VT;
  __shared__ VT vs[2][kAdjY + 2][kAdjX + 2];
  __shared__ S ts[2][kAdjY + 2][kAdjX + 2];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kAdjX + tx;
  const int x0 = blockIdx.x * kAdjX, y0 = blockIdx.y * kAdjY;
  const int x = x0 + tx, y = y0 + ty;
  const int z0 = blockIdx.z * zb, z1 = min(z0 + zb, nz);
  const typename Ops::WT aw = Ops::weights(c);
  const long long sy = nx, sz = (long long)nx * ny;
  // ring position of this thread (tid < kAdjRing): rows y0-1 and y0+kAdjY
  // over x0-1 .. x0+kAdjX, then columns x0-1 and x0+kAdjX over y0 .. y0+kAdjY-1
  int rx = 0, ry = 0, sxr = 0, syr = 0;
  if (tid < kAdjRing) {
    if (tid < 2 * (kAdjX + 2)) {
      const int i = tid % (kAdjX + 2);
      rx = x0 - 1 + i;
      ry = tid < kAdjX + 2 ? y0 - 1 : y0 + kAdjY;
    } else {
      const int i = tid - 2 * (kAdjX + 2);
      rx = i < kAdjY ? x0 - 1 : x0 + kAdjX;
      ry = y0 + (i % kAdjY);
    }
    sxr = rx - x0 + 1;
    syr = ry - y0 + 1;
  }
  const bool own = x < nx && y < ny;
  const bool ring = tid < kAdjRing && rx >= 0 && rx < nx && ry >= 0 && ry < ny;
  const bool in_xy = x > 0 && x < nx - 1 && y > 0 && y < ny - 1;
  const bool rin_xy = rx > 0 && rx < nx - 1 && ry > 0 && ry < ny - 1;
  const S zero = S(0);
  // v and T at (xx, yy, z): v = 0 off the inner points, T = 0 off the array
  auto vload = [&](bool ok, bool inner, long long p, int z) -> VT {
    const bool in = ok && inner && z > 0 && z < nz - 1;
    return Ops::v(Ops::lam(in ? __ldg(lam_in + p) : zero), in ? __ldg(Ci + p) : zero, in);
  };
  auto tload = [&](bool ok, long long p, int z) -> S {
    return (ok && z >= 0 && z < nz) ? __ldg(Tn + p) : zero;
  };
  const long long pc = x + sy * y, pr = rx + sy * ry;
  VT vm = vload(own, in_xy, pc + sz * (z0 - 1), z0 - 1), vc = vload(own, in_xy, pc + sz * z0, z0);
  S tm = tload(own, pc + sz * (z0 - 1), z0 - 1), tc = tload(own, pc + sz * z0, z0);
  S la = own ? __ldg(lam_in + pc + sz * z0) : zero;
  // ring values of the current plane, loaded one plane ahead
  VT rv = vload(ring, rin_xy, pr + sz * z0, z0);
  S rt = tload(ring, pr + sz * z0, z0);
  for (int z = z0; z < z1; ++z) {
    const int b = z & 1;
    const long long p = pc + sz * z;
    vs[b][ty + 1][tx + 1] = vc;
    ts[b][ty + 1][tx + 1] = tc;
    if (tid < kAdjRing) {
      vs[b][syr][sxr] = rv;
      ts[b][syr][sxr] = rt;
      rv = vload(ring, rin_xy, pr + sz * (z + 1), z + 1);
      rt = tload(ring, pr + sz * (z + 1), z + 1);
    }
    const VT vp = vload(own, in_xy, p + sz, z + 1);
    const S tp = tload(own, p + sz, z + 1);
    const S lap = own && z + 1 < nz ? __ldg(lam_in + p + sz) : zero;
    __syncthreads();
    S out;
    const bool ok = Ops::out(Ops::lam(la), vc, vs[b][ty + 1][tx], vs[b][ty + 1][tx + 2],
                             vs[b][ty][tx + 1], vs[b][ty + 2][tx + 1], vm, vp, aw, out);
    if constexpr (sizeof(S) == 8) {
      // points outside the pair path's ranges: the FP64 sum
      if (__any_sync(0xffffffffu, own && !ok)) {
        if (own && !ok) {
          const double *L = reinterpret_cast<const double *>(lam_in);
          const double *C = reinterpret_cast<const double *>(Ci);
          out = adj_out_f64(la, v64_at(L, C, x, y, z, nx, ny, nz), v64_at(L, C, x - 1, y, z, nx, ny, nz),
                            v64_at(L, C, x + 1, y, z, nx, ny, nz), v64_at(L, C, x, y - 1, z, nx, ny, nz),
                            v64_at(L, C, x, y + 1, z, nx, ny, nz), v64_at(L, C, x, y, z - 1, nx, ny, nz),
                            v64_at(L, C, x, y, z + 1, nx, ny, nz), aw.w);
        }
      }
    }
    if (own) lam_out[p] = out;
    const bool inner = own && in_xy && z > 0 && z < nz - 1;
    const double g = inner ? gCi[p] : 0.0;
    const double gn = gci_add(g, inner, la, tc, ts[b][ty + 1][tx], ts[b][ty + 1][tx + 2],
                              ts[b][ty][tx + 1], ts[b][ty + 2][tx + 1], tm, tp, Ops::lapw(aw));
    if (inner) gCi[p] = gn;
    vm = vc;
    vc = vp;
    tm = tc;
    tc = tp;
    la = lap;
  }
}

template <class S>
__global__ void __launch_bounds__(256)
    k_sub(long long n, S *out, const S *a, const S *b) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = a[i] - b[i];
}

}  // namespace

cudaError_t launch_adjoint(igg_dtype dt, int nx, int ny, int nz, void *lam_out,
                           const void *lam_in, const void *Tn, const void *Ci, double *gCi,
                           const Coef &c, bool tma, unsigned *dev_err, cudaStream_t s,
                           const void *ci_pairs) {
  if (tma && adjoint_tma_applies(dt, nx, lam_out, lam_in, Tn, Ci, gCi))
    return launch_adjoint_tma(dt, nx, ny, nz, lam_out, lam_in, Tn, Ci, gCi, c, dev_err, s,
                              dt == IGG_F64 ? ci_pairs : nullptr);
  const int zb = std::min(nz, 32);
  const dim3 grid((nx + kAdjX - 1) / kAdjX, (ny + kAdjY - 1) / kAdjY, (nz + zb - 1) / zb);
  const dim3 block(kAdjX, kAdjY);
  switch (dt) {
    case IGG_F64:
      k_adjoint<double><<<grid, block, 0, s>>>(nx, ny, nz, zb, (double *)lam_out,
                                               (const double *)lam_in, (const double *)Tn,
                                               (const double *)Ci, gCi, c);
      break;
    case IGG_F32:
      k_adjoint<float><<<grid, block, 0, s>>>(nx, ny, nz, zb, (float *)lam_out,
                                              (const float *)lam_in, (const float *)Tn,
                                              (const float *)Ci, gCi, c);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_sub(igg_dtype dt, long long n, void *out, const void *a, const void *b,
                       cudaStream_t s) {
  long long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  switch (dt) {
    case IGG_F64:
      k_sub<double><<<(int)blocks, 256, 0, s>>>(n, (double *)out, (const double *)a,
                                                (const double *)b);
      break;
    case IGG_F32:
      k_sub<float><<<(int)blocks, 256, 0, s>>>(n, (float *)out, (const float *)a,
                                               (const float *)b);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace igg
