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

// blockIdx.z = subdomain * zchunks + z chunk. The z march is software
// pipelined: the loads of plane k + 1 are issued before the stores of plane
// k, so that each thread keeps two planes of loads in flight (the launches
// are bound by memory latency otherwise).
//
// x sends (AcCoef::xsend): update_halo!'s x exchange done by the launches
// themselves. A field of x size nf and x overlap of sends its plane nf - of
// to the right neighbour's plane 0 and its plane of - 1 to the left
// neighbour's plane nf - 1 (P, Vy, Vz: of = o; Vx: nf = nx + 1, of = o + 1);
// the thread of a sent column stores every value of it as the launch leaves
// it (computed, or a wall face it does not compute) a second time into the
// neighbour, and the threads of receiving columns do not store there. The y
// and z exchanges run after both launches.
// The x sends of one thread: sm bit 0 / 1 its column is sent right / left;
// dr, dl the neighbours' subdomain offsets (xr - sub, xl - sub). The copy of
// the value at own index q of a field of np points per subdomain and x send
// distance h = nf - of goes to q + dr np - h (right) and q + dl np + h (left).
struct AcSend {
  unsigned sm;
  int dr, dl;
};

__device__ __forceinline__ AcSend ac_send(int i, int nf, int of, long long sub, int xl, int xr) {
  AcSend a;
  a.sm = (xr >= 0 && i == nf - of ? 1u : 0u) | (xl >= 0 && i == of - 1 ? 2u : 0u);
  a.dr = xr - (int)sub;
  a.dl = xl - (int)sub;
  return a;
}

template <class S>
__device__ __forceinline__ void ac_put(S *p, S v, const AcSend &a, long long np, int h) {
  if (a.sm & 1u) p[(long long)a.dr * np - h] = v;
  if (a.sm & 2u) p[(long long)a.dl * np + h] = v;
}

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
  const long long sp = (long long)nx * ny, sx = (long long)(nx + 1) * ny,
                  sy = (long long)nx * (ny + 1);
  const long long npx = sx * nz, npy = sy * nz, npz = sp * (nz + 1);
  const S *Ps = P + sub * np + i + (long long)nx * j;
  S *Vxs = Vx + sub * npx + i + (long long)(nx + 1) * j;
  S *Vys = Vy + sub * npy + i + (long long)nx * j;
  S *Vzs = Vz + sub * npz + i + (long long)nx * j;
  // x sends (Vx: nf = nx + 1, of = o + 1; Vy, Vz: nf = nx, of = o; the
  // send distance nf - of is nx - o for all three) and the receiving columns
  // (halo cells: Vy and Vz not stored)
  AcSend ex{0u, 0, 0}, ev = ex;
  bool keep = true;
  const int h = nx - c.ox;
  if (c.xsend) {
    const int xl = c.nbr[6 * sub], xr = c.nbr[6 * sub + 1];
    ex = ac_send(i, nx + 1, c.ox + 1, sub, xl, xr);
    ev = ac_send(i, nx, c.ox, sub, xl, xr);
    keep = !((i == 0 && xl >= 0) || (i == nx - 1 && xr >= 0));
  }
  const bool sv = ev.sm != 0u;  // sends Vy and Vz (wall faces too)
  S pzm = k0 > 0 ? Ps[sp * (k0 - 1)] : S(0);
  // plane k0
  S pc = Ps[sp * k0];
  S pxm = i > 0 ? Ps[sp * k0 - 1] : S(0);
  S pym = j > 0 ? Ps[sp * k0 - nx] : S(0);
  S vx = i > 0 ? Vxs[sx * k0] : S(0);
  S vy = (j > 0 || sv) ? Vys[sy * k0] : S(0);
  S vz = (k0 > 0 || sv) ? Vzs[sp * k0] : S(0);
  for (int k = k0; k < k1; ++k) {
    // plane k + 1
    const bool nxt = k + 1 < k1;
    S pc1 = S(0), pxm1 = S(0), pym1 = S(0), vx1 = S(0), vy1 = S(0), vz1 = S(0);
    if (nxt) {
      pc1 = Ps[sp * (k + 1)];
      if (i > 0) {
        pxm1 = Ps[sp * (k + 1) - 1];
        vx1 = Vxs[sx * (k + 1)];
      }
      if (j > 0) pym1 = Ps[sp * (k + 1) - nx];
      if (j > 0 || sv) vy1 = Vys[sy * (k + 1)];
      vz1 = Vzs[sp * (k + 1)];
    }
    if (i > 0) {
      vx = N::fma(-ax, N::sub(pc, pxm), vx);
      Vxs[sx * k] = vx;
    }
    if (j > 0) {
      vy = N::fma(-ay, N::sub(pc, pym), vy);
      if (keep) Vys[sy * k] = vy;
    }
    if (k > 0) {
      vz = N::fma(-az, N::sub(pc, pzm), vz);
      if (keep) Vzs[sp * k] = vz;
    }
    if (ex.sm) ac_put(Vxs + sx * k, vx, ex, npx, h);
    if (sv) {
      ac_put(Vys + sy * k, vy, ev, npy, h);
      ac_put(Vzs + sp * k, vz, ev, npz, h);
      // the last face row of Vy (y = ny, a wall or halo face no thread
      // computes)
      if (j == ny - 1) ac_put(Vys + sy * k + nx, Vys[sy * k + nx], ev, npy, h);
    }
    pzm = pc;
    pc = pc1;
    pxm = pxm1;
    pym = pym1;
    vx = vx1;
    vy = vy1;
    vz = vz1;
  }
  // the last plane of Vz (z = nz, a wall or halo face no thread computes)
  if (sv && k1 == nz) ac_put(Vzs + sp * nz, Vzs[sp * nz], ev, npz, h);
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
  const long long sp = (long long)nx * ny, sx = (long long)(nx + 1) * ny,
                  sy = (long long)nx * (ny + 1);
  S *Ps = P + sub * np + i + (long long)nx * j;
  const S *Vxs = Vx + sub * (long long)(nx + 1) * ny * nz + i + (long long)(nx + 1) * j;
  const S *Vys = Vy + sub * (long long)nx * (ny + 1) * nz + i + (long long)nx * j;
  const S *Vzs = Vz + sub * (long long)nx * ny * (nz + 1) + i + (long long)nx * j;
  AcSend ep{0u, 0, 0};
  bool keep = true;
  const int h = nx - c.ox;
  if (c.xsend) {
    const int xl = c.nbr[6 * sub], xr = c.nbr[6 * sub + 1];
    ep = ac_send(i, nx, c.ox, sub, xl, xr);
    keep = !((i == 0 && xl >= 0) || (i == nx - 1 && xr >= 0));
  }
  S vzc = Vzs[sp * k0];
  // plane k0
  S pc = Ps[sp * k0], x0 = Vxs[sx * k0], x1 = Vxs[sx * k0 + 1], y0 = Vys[sy * k0],
    y1 = Vys[sy * k0 + nx], vzp = Vzs[sp * (k0 + 1)];
  for (int k = k0; k < k1; ++k) {
    // plane k + 1
    const bool nxt = k + 1 < k1;
    S pc1 = S(0), x01 = S(0), x11 = S(0), y01 = S(0), y11 = S(0), vzp1 = S(0);
    if (nxt) {
      pc1 = Ps[sp * (k + 1)];
      x01 = Vxs[sx * (k + 1)];
      x11 = Vxs[sx * (k + 1) + 1];
      y01 = Vys[sy * (k + 1)];
      y11 = Vys[sy * (k + 1) + nx];
      vzp1 = Vzs[sp * (k + 2)];
    }
    // P - bx dVx - by dVy - bz dVz, one FMA per term (6 FP64 instructions
    // per cell for FP64 fields, whose launches the FP64 pipe bounds)
    S pn = N::fma(-bx, N::sub(x1, x0), pc);
    pn = N::fma(-by, N::sub(y1, y0), pn);
    pn = N::fma(-bz, N::sub(vzp, vzc), pn);
    if (keep) Ps[sp * k] = pn;
    if (ep.sm) ac_put(Ps + sp * k, pn, ep, np, h);
    vzc = vzp;
    pc = pc1;
    x0 = x01;
    x1 = x11;
    y0 = y01;
    y1 = y11;
    vzp = vzp1;
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
