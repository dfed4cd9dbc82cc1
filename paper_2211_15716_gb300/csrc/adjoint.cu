// Adjoint of Fig. 1's step! (the transposed stencil run backward in time) and
// the checkpointed drivers that give gradients of a function of T_nt with
// respect to Ci and the initial T.
//
// Forward step on inner points p:  T_{n+1}[p] = T_n[p] + Ci[p] * l(T_n)[p],
// l(T)[p] = sum_d w_d (T[p-e_d] + T[p+e_d] - 2 T[p]),  w_d = dt*lam/dd^2,
// identity on the array boundary. Given lam_in = dJ/dT_{n+1}:
//   v[q]       = Ci[q]*lam_in[q] on inner q, 0 elsewhere,
//   lam_out[q] = lam_in[q] + sum_d w_d (v[q-e_d] + v[q+e_d] - 2 v[q]),
//                on every point q (neighbours outside the array are 0),
//   gCi[p]    += lam_in[p] * l(T_n)[p] on inner p (accumulated in FP64).
// FP64 fields form l(T_n) with the emulated cell's exact differences where the
// stencil allows it (cell.cuh), else in FP64; the v sums are FP64 (lam_in
// changes sign from point to point, which the emulation cannot take).
#include <algorithm>
#include <cstring>

#include "cell.cuh"
#include "igg_internal.h"

namespace igg {
namespace {

template <class S>
struct AdjNum;
template <>
struct AdjNum<double> {
  using C = double;
  static __device__ __forceinline__ double ld(const double *p) { return __ldg(p); }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  // l from the z-summed and neighbour values, forward-FP64 order
  static __device__ __forceinline__ double lsum(double c, double xm, double xp, double ym,
                                                double yp, double zm, double zp, double wx,
                                                double wy, double wz, double wc) {
    const double sx = __dadd_rn(xm, xp), sy = __dadd_rn(ym, yp), sz = __dadd_rn(zm, zp);
    double l = __dmul_rn(wc, c);
    l = __fma_rn(wx, sx, l);
    l = __fma_rn(wy, sy, l);
    return __fma_rn(wz, sz, l);
  }
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double fma(double a, double b, double c) {
    return __fma_rn(a, b, c);
  }
};
template <>
struct AdjNum<float> {
  using C = float;
  static __device__ __forceinline__ float ld(const float *p) { return __ldg(p); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  // forward-FP32 order: differences first
  static __device__ __forceinline__ float lsum(float c, float xm, float xp, float ym, float yp,
                                               float zm, float zp, float wx, float wy, float wz,
                                               float) {
    const float ex = __fadd_rn(__fsub_rn(xp, c), __fsub_rn(xm, c));
    const float ey = __fadd_rn(__fsub_rn(yp, c), __fsub_rn(ym, c));
    const float ez = __fadd_rn(__fsub_rn(zp, c), __fsub_rn(zm, c));
    float l = __fmul_rn(wx, ex);
    l = __fmaf_rn(wy, ey, l);
    return __fmaf_rn(wz, ez, l);
  }
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float fma(float a, float b, float c) {
    return __fmaf_rn(a, b, c);
  }
};

constexpr int kAdjX = 32, kAdjY = 8, kAdjRing = 2 * (kAdjX + 2) + 2 * kAdjY;

// l(T_n) * lam_in added to gCi on inner points: FP64 fields use the emulated
// cell's exact second differences where the stencil shares sign and exponent
// (T_n is a forward state, smooth), else the FP64 sum; FP32 fields their
// FP32 sum. `inner` is the same for the whole warp's call; the FP64 sum is
// reached only by warps with a point that needs it (a branch on a warp vote,
// so that it is not evaluated, predicated off, on every point).
__device__ __forceinline__ void gci_update(double *gp, bool inner, double la, double t, double xm,
                                           double xp, double ym, double yp, double zm, double zp,
                                           const W<double> &w) {
  const double tn[6] = {xm, xp, ym, yp, zm, zp};
  unsigned hn[6];
  unsigned long long nb[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    hn[i] = dhi(tn[i]);
    nb[i] = dbits(tn[i]);
  }
  const bool ok = emu_fast_ok(dhi(t), hn);
  if (__all_sync(0xffffffffu, ok || !inner)) {
    if (!inner) return;
    const double g = *gp;
    if (w.ng == 1) *gp = emu_apply(g, la, emu_lap<1>(t, nb, w));
    else if (w.ng == 2) *gp = emu_apply(g, la, emu_lap<2>(t, nb, w));
    else *gp = emu_apply(g, la, emu_lap<3>(t, nb, w));
  } else if (inner) {
    const double g = *gp;
    if (ok) {
      if (w.ng == 1) *gp = emu_apply(g, la, emu_lap<1>(t, nb, w));
      else if (w.ng == 2) *gp = emu_apply(g, la, emu_lap<2>(t, nb, w));
      else *gp = emu_apply(g, la, emu_lap<3>(t, nb, w));
    } else {
      *gp = __fma_rn(la, AdjNum<double>::lsum(t, xm, xp, ym, yp, zm, zp, w.wx, w.wy, w.wz, w.wc),
                     g);
    }
  }
}
__device__ __forceinline__ void gci_update(double *gp, bool inner, float la, float t, float xm,
                                           float xp, float ym, float yp, float zm, float zp,
                                           const W<float> &w) {
  if (inner)
    *gp = __fma_rn((double)la,
                   (double)AdjNum<float>::lsum(t, xm, xp, ym, yp, zm, zp, w.wx, w.wy, w.wz, w.wc),
                   *gp);
}

// One CTA per 32x8 block of (x, y) columns and a chunk of zb planes, every
// point of the array. Per plane, v = Ci*lam_in and T_n of the block and of
// the ring of one point around it go to shared memory (two buffers, one
// barrier per plane); each v is formed once, by the thread of its point or
// of its ring position. The column's planes z-1, z, z+1 stay in registers.
template <class S>
__global__ void __launch_bounds__(kAdjX *kAdjY)
    k_adjoint(int nx, int ny, int nz, int zb, S *__restrict__ lam_out,
              const S *__restrict__ lam_in, const S *__restrict__ Tn,
              const S *__restrict__ Ci, double *__restrict__ gCi, Coef c) {
  using N = AdjNum<S>;
  using C = typename N::C;
  __shared__ C vs[2][kAdjY + 2][kAdjX + 2];
  __shared__ C ts[2][kAdjY + 2][kAdjX + 2];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kAdjX + tx;
  const int x0 = blockIdx.x * kAdjX, y0 = blockIdx.y * kAdjY;
  const int x = x0 + tx, y = y0 + ty;
  const int z0 = blockIdx.z * zb, z1 = min(z0 + zb, nz);
  const W<C> w = make_w(c, C(0));
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
  // v and T at (xx, yy, z): v = 0 off the inner points, T = 0 off the array
  auto vload = [&](bool ok, bool inner, long long p, int z) -> C {
    return (ok && inner && z > 0 && z < nz - 1) ? N::mul(N::ld(Ci + p), N::ld(lam_in + p)) : C(0);
  };
  auto tload = [&](bool ok, long long p, int z) -> C {
    return (ok && z >= 0 && z < nz) ? N::ld(Tn + p) : C(0);
  };
  const long long pc = x + sy * y, pr = rx + sy * ry;
  C vm = vload(own, in_xy, pc + sz * (z0 - 1), z0 - 1), vc = vload(own, in_xy, pc + sz * z0, z0);
  C tm = tload(own, pc + sz * (z0 - 1), z0 - 1), tc = tload(own, pc + sz * z0, z0);
  C la = own ? N::ld(lam_in + pc + sz * z0) : C(0);
  // ring values of the current plane, loaded one plane ahead
  C rv = vload(ring, rin_xy, pr + sz * z0, z0), rt = tload(ring, pr + sz * z0, z0);
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
    const C vp = vload(own, in_xy, p + sz, z + 1);
    const C tp = tload(own, p + sz, z + 1);
    const C lap = own && z + 1 < nz ? N::ld(lam_in + p + sz) : C(0);
    __syncthreads();
    if (own) {
      const C vxm = vs[b][ty + 1][tx], vxp = vs[b][ty + 1][tx + 2];
      const C vym = vs[b][ty][tx + 1], vyp = vs[b][ty + 2][tx + 1];
      // lam_out = lam_in + wc v + sum_d w_d (v[-d] + v[+d])
      C acc = N::fma(w.wc, vc, la);
      acc = N::fma(w.wx, N::add(vxm, vxp), acc);
      acc = N::fma(w.wy, N::add(vym, vyp), acc);
      acc = N::fma(w.wz, N::add(vm, vp), acc);
      lam_out[p] = (S)acc;
    }
    // every thread of the warp takes part (warp vote inside)
    gci_update(gCi + (own ? p : 0), own && in_xy && z > 0 && z < nz - 1, la, tc,
               ts[b][ty + 1][tx], ts[b][ty + 1][tx + 2], ts[b][ty][tx + 1], ts[b][ty + 2][tx + 1],
               tm, tp, w);
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
                           const Coef &c, cudaStream_t s) {
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
