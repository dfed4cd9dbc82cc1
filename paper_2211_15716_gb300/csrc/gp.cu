// Gross-Pitaevskii half steps on the implicit global grid: a complex field
// psi = u + i v kept as two real fields of the grid's layout, u at whole and
// v at half time steps:
//   which 0:  u += dt * H(v),   which 1:  v -= dt * H(u),
//   H w = -1/2 lap(w) + (V + g (u^2 + v^2)) w,
// on inner points (psi fixed on each array's boundary), lap the 7-point
// operator with the grid's spacings. One thread per (x, y) column of a
// subdomain marches along z keeping w's z neighbours in registers; absent
// dimensions (size 1) have zero neighbour strides and zero weights.
#include "igg_internal.h"

namespace igg {
namespace {

constexpr int kGpX = 32, kGpY = 8, kGpZ = 32;

template <class S>
struct GpNum;
template <>
struct GpNum<double> {
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double fma(double a, double b, double c) {
    return __fma_rn(a, b, c);
  }
};
template <>
struct GpNum<float> {
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float fma(float a, float b, float c) {
    return __fmaf_rn(a, b, c);
  }
};

// blockIdx.z = subdomain * zchunks + z chunk; inner ranges [lo, hi) per
// dimension (absent dimensions: [0, 1) with zero stride)
template <class S, int WHICH>
__global__ void __launch_bounds__(kGpX *kGpY)
    k_gp_half(int nx, int ny, int nz, int zchunks, S *__restrict__ u, S *__restrict__ v,
              const S *__restrict__ V, GpCoef c) {
  using N = GpNum<S>;
  const int ylo = ny > 1 ? 1 : 0, yhi = ny > 1 ? ny - 1 : 1;
  const int zlo = nz > 1 ? 1 : 0, zhi = nz > 1 ? nz - 1 : 1;
  const int i = 1 + blockIdx.x * kGpX + threadIdx.x, j = ylo + blockIdx.y * kGpY + threadIdx.y;
  if (i >= nx - 1 || j >= yhi) return;
  const long long sub = blockIdx.z / zchunks;
  const int k0 = zlo + (int)(blockIdx.z % zchunks) * kGpZ, k1 = min(k0 + kGpZ, zhi);
  if (k0 >= k1) return;
  const long long nloc = (long long)nx * ny * nz;
  const long long sy = ny > 1 ? nx : 0, sz = nz > 1 ? (long long)nx * ny : 0;
  S *out = (WHICH == 0 ? u : v) + sub * nloc;
  const S *w = (WHICH == 0 ? v : u) + sub * nloc;
  const S *us = u + sub * nloc, *vs = v + sub * nloc, *Vs = V + sub * nloc;
  // h scaled by dt: kx s_x + ky s_y + kz s_z + kc w + dt (V + g rho) w,
  // kd = -dt/(2 dd^2), kc = -2 (kx + ky + kz)
  const S kx = (S)c.kx, ky = (S)c.ky, kz = (S)c.kz, kc = (S)c.kc, dt = (S)c.dt, g = (S)c.g;
  long long p = i + (long long)nx * j + (long long)nx * ny * k0;
  S wm = w[p - sz], wc = w[p];
  for (int k = k0; k < k1; ++k, p += (long long)nx * ny) {
    const S wp = w[p + sz];
    const S uc = us[p], vc = vs[p];
    S h = N::mul(kc, wc);
    h = N::fma(kx, N::add(w[p - 1], w[p + 1]), h);
    h = N::fma(ky, N::add(w[p - sy], w[p + sy]), h);
    h = N::fma(kz, N::add(wm, wp), h);
    const S q = N::mul(dt, N::fma(g, N::fma(uc, uc, N::mul(vc, vc)), Vs[p]));
    h = N::fma(q, wc, h);
    out[p] = WHICH == 0 ? N::add(out[p], h) : N::add(out[p], -h);
    wm = wc;
    wc = wp;
  }
}

template <class S, int WHICH>
cudaError_t launch_w(int nsub, int nx, int ny, int nz, void *u, void *v, const void *V,
                     const GpCoef &c, cudaStream_t s) {
  const int ny_in = ny > 1 ? ny - 2 : 1, nz_in = nz > 1 ? nz - 2 : 1;
  const int zchunks = (nz_in + kGpZ - 1) / kGpZ;
  const long long gz = (long long)nsub * zchunks;
  if (gz > 65535 || nx < 3) return cudaErrorInvalidValue;
  const dim3 grid((nx - 2 + kGpX - 1) / kGpX, (ny_in + kGpY - 1) / kGpY, (unsigned)gz);
  k_gp_half<S, WHICH><<<grid, dim3(kGpX, kGpY), 0, s>>>(nx, ny, nz, zchunks, (S *)u, (S *)v,
                                                       (const S *)V, c);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gp_half(igg_dtype dt, int which, int nsub, int nx, int ny, int nz, void *u,
                           void *v, const void *V, const GpCoef &c, cudaStream_t s) {
  switch (dt) {
    case IGG_F64:
      return which == 0 ? launch_w<double, 0>(nsub, nx, ny, nz, u, v, V, c, s)
                        : launch_w<double, 1>(nsub, nx, ny, nz, u, v, V, c, s);
    case IGG_F32:
      return which == 0 ? launch_w<float, 0>(nsub, nx, ny, nz, u, v, V, c, s)
                        : launch_w<float, 1>(nsub, nx, ny, nz, u, v, V, c, s);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace igg
