// Staggered-grid acoustics (a multi-field stencil on the implicit global grid
// whose fields have different sizes): P at cells [nz][ny][nx], Vx at x faces
// [nz][ny][nx+1], Vy at y faces [nz][ny+1][nx], Vz at z faces [nz+1][ny][nx],
// every field of every subdomain in one buffer [nsub][...]. One leapfrog step:
//   Vx[i] -= dt/(rho dx) (P[i] - P[i-1]) on faces 1..nx-1 (all y, z), likewise
//   Vy, Vz;  then  P -= dt K / dx (Vx[i+1] - Vx[i]) + ... on every cell.
// The outermost faces are never written (walls, or halo faces of a
// subdomain that the halo update fills). One thread per (x, y) column marches
// along z, keeping the z neighbour in a register.
#include "igg_internal.h"

namespace igg {
namespace {

constexpr int kAcX = 32, kAcY = 8, kAcZ = 32;

template <class S>
struct AcNum;
template <>
struct AcNum<double> {
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double fma(double a, double b, double c) {
    return __fma_rn(a, b, c);
  }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
};
template <>
struct AcNum<float> {
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float fma(float a, float b, float c) {
    return __fmaf_rn(a, b, c);
  }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
};

// blockIdx.z = subdomain * zchunks + z chunk
template <class S>
__global__ void __launch_bounds__(kAcX *kAcY)
    k_acoustic_v(int nx, int ny, int nz, int zchunks, const S *__restrict__ P, S *__restrict__ Vx,
                 S *__restrict__ Vy, S *__restrict__ Vz, AcCoef c) {
  using N = AcNum<S>;
  const int i = blockIdx.x * kAcX + threadIdx.x, j = blockIdx.y * kAcY + threadIdx.y;
  if (i >= nx || j >= ny) return;
  const long long sub = blockIdx.z / zchunks;
  const int k0 = (int)(blockIdx.z % zchunks) * kAcZ, k1 = min(k0 + kAcZ, nz);
  const S ax = (S)c.ax, ay = (S)c.ay, az = (S)c.az;
  const long long np = (long long)nx * ny * nz;
  const S *Ps = P + sub * np;
  S *Vxs = Vx + sub * (long long)(nx + 1) * ny * nz;
  S *Vys = Vy + sub * (long long)nx * (ny + 1) * nz;
  S *Vzs = Vz + sub * (long long)nx * ny * (nz + 1);
  S pzm = k0 > 0 ? Ps[i + (long long)nx * (j + (long long)ny * (k0 - 1))] : S(0);
  for (int k = k0; k < k1; ++k) {
    const long long p = i + (long long)nx * (j + (long long)ny * k);
    const S pc = Ps[p];
    if (i > 0) {
      S *v = Vxs + i + (long long)(nx + 1) * (j + (long long)ny * k);
      *v = N::fma(-ax, N::sub(pc, Ps[p - 1]), *v);
    }
    if (j > 0) {
      S *v = Vys + i + (long long)nx * (j + (long long)(ny + 1) * k);
      *v = N::fma(-ay, N::sub(pc, Ps[p - nx]), *v);
    }
    if (k > 0) {
      S *v = Vzs + p;
      *v = N::fma(-az, N::sub(pc, pzm), *v);
    }
    pzm = pc;
  }
}

template <class S>
__global__ void __launch_bounds__(kAcX *kAcY)
    k_acoustic_p(int nx, int ny, int nz, int zchunks, S *__restrict__ P,
                 const S *__restrict__ Vx, const S *__restrict__ Vy, const S *__restrict__ Vz,
                 AcCoef c) {
  using N = AcNum<S>;
  const int i = blockIdx.x * kAcX + threadIdx.x, j = blockIdx.y * kAcY + threadIdx.y;
  if (i >= nx || j >= ny) return;
  const long long sub = blockIdx.z / zchunks;
  const int k0 = (int)(blockIdx.z % zchunks) * kAcZ, k1 = min(k0 + kAcZ, nz);
  const S bx = (S)c.bx, by = (S)c.by, bz = (S)c.bz;
  const long long np = (long long)nx * ny * nz;
  S *Ps = P + sub * np;
  const S *Vxs = Vx + sub * (long long)(nx + 1) * ny * nz;
  const S *Vys = Vy + sub * (long long)nx * (ny + 1) * nz;
  const S *Vzs = Vz + sub * (long long)nx * ny * (nz + 1);
  S vzc = Vzs[i + (long long)nx * (j + (long long)ny * k0)];
  for (int k = k0; k < k1; ++k) {
    const long long p = i + (long long)nx * (j + (long long)ny * k);
    const long long px = i + (long long)(nx + 1) * (j + (long long)ny * k);
    const long long py = i + (long long)nx * (j + (long long)(ny + 1) * k);
    const S vzp = Vzs[p + (long long)nx * ny];
    S div = N::mul(bx, N::sub(Vxs[px + 1], Vxs[px]));
    div = N::fma(by, N::sub(Vys[py + nx], Vys[py]), div);
    div = N::fma(bz, N::sub(vzp, vzc), div);
    Ps[p] = N::sub(Ps[p], div);
    vzc = vzp;
  }
}

template <class S>
cudaError_t launch_t(int nsub, int nx, int ny, int nz, void *P, void *Vx, void *Vy, void *Vz,
                     const AcCoef &c, cudaStream_t s) {
  const int zchunks = (nz + kAcZ - 1) / kAcZ;
  const long long gz = (long long)nsub * zchunks;
  if (gz > 65535) return cudaErrorInvalidValue;
  const dim3 grid((nx + kAcX - 1) / kAcX, (ny + kAcY - 1) / kAcY, (unsigned)gz);
  const dim3 block(kAcX, kAcY);
  k_acoustic_v<S><<<grid, block, 0, s>>>(nx, ny, nz, zchunks, (const S *)P, (S *)Vx, (S *)Vy,
                                          (S *)Vz, c);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_acoustic_p<S><<<grid, block, 0, s>>>(nx, ny, nz, zchunks, (S *)P, (const S *)Vx,
                                          (const S *)Vy, (const S *)Vz, c);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_acoustic(igg_dtype dt, int nsub, int nx, int ny, int nz, void *P, void *Vx,
                            void *Vy, void *Vz, const AcCoef &c, cudaStream_t s) {
  switch (dt) {
    case IGG_F64: return launch_t<double>(nsub, nx, ny, nz, P, Vx, Vy, Vz, c, s);
    case IGG_F32: return launch_t<float>(nsub, nx, ny, nz, P, Vx, Vy, Vz, c, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace igg
