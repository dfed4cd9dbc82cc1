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
// The v and l sums use the same arithmetic as the forward kernels.
#include <algorithm>
#include <cstring>

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
};

constexpr int kAdjX = 32, kAdjY = 8;

// One thread per (x, y) column of a z-chunk; every point of the array.
template <class S>
__global__ void __launch_bounds__(kAdjX *kAdjY)
    k_adjoint(int nx, int ny, int nz, int zb, S *__restrict__ lam_out,
              const S *__restrict__ lam_in, const S *__restrict__ Tn,
              const S *__restrict__ Ci, double *__restrict__ gCi, Coef c) {
  using N = AdjNum<S>;
  using C = typename N::C;
  const int x = blockIdx.x * kAdjX + threadIdx.x;
  const int y = blockIdx.y * kAdjY + threadIdx.y;
  if (x >= nx || y >= ny) return;
  const int z0 = blockIdx.z * zb;
  const int z1 = min(z0 + zb, nz);
  const C wx = (C)c.wx, wy = (C)c.wy, wz = (C)c.wz, wc = (C)c.wc;
  const long long sy = nx, sz = (long long)nx * ny;
  const bool in_xy = x > 0 && x < nx - 1 && y > 0 && y < ny - 1;
  // v at (x, y, z) of this column, 0 off the inner points
  auto vcol = [&](int z) -> C {
    if (!in_xy || z <= 0 || z >= nz - 1) return C(0);
    const long long p = x + sy * y + sz * z;
    return N::mul(N::ld(Ci + p), N::ld(lam_in + p));
  };
  auto vat = [&](int xx, int yy, int z) -> C {
    if (xx <= 0 || xx >= nx - 1 || yy <= 0 || yy >= ny - 1 || z <= 0 || z >= nz - 1) return C(0);
    const long long p = xx + sy * yy + sz * z;
    return N::mul(N::ld(Ci + p), N::ld(lam_in + p));
  };
  C vm = vcol(z0 - 1), vc = vcol(z0);
  for (int z = z0; z < z1; ++z) {
    const C vp = vcol(z + 1);
    const long long p = x + sy * y + sz * z;
    const C la = N::ld(lam_in + p);
    const C adj = N::lsum(vc, vat(x - 1, y, z), vat(x + 1, y, z), vat(x, y - 1, z),
                          vat(x, y + 1, z), vm, vp, wx, wy, wz, wc);
    lam_out[p] = (S)N::add(la, adj);
    if (in_xy && z > 0 && z < nz - 1) {
      const C t = N::ld(Tn + p);
      const C l = N::lsum(t, N::ld(Tn + p - 1), N::ld(Tn + p + 1), N::ld(Tn + p - sy),
                          N::ld(Tn + p + sy), N::ld(Tn + p - sz), N::ld(Tn + p + sz), wx, wy, wz,
                          wc);
      gCi[p] = __fma_rn((double)la, (double)l, gCi[p]);
    }
    vm = vc;
    vc = vp;
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
