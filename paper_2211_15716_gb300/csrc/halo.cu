// Halo update kernels (update_halo!, Sec. Approach): on one GPU every
// neighbour lives in the same device memory, so packing, sending and
// unpacking a face collapse into device-to-device copies. Fields of the
// grid's own size take one gather launch (k_halo_gather, below); staggered
// sizes take the plane copies: one launch copies all face planes of one
// dimension of one field, the host issuing the dimensions in the order x, y,
// z on one stream, which gives edges and corners the values of the
// sequential exchange.
#include <algorithm>

#include "igg_internal.h"

namespace igg {
namespace {

// One block per (copy, plane row b): the row's na points at stride sa. VEC:
// rows contiguous (sa = 1) and 16-byte aligned, copied as 16-byte vectors.
template <class E, bool VEC>
__global__ void __launch_bounds__(256)
    k_halo_planes(const PlaneCopy *__restrict__ copies, E *__restrict__ f, int na, int nb,
                  long long sa, long long sb) {
  const int ci = blockIdx.x / nb, b = blockIdx.x % nb;
  const PlaneCopy c = copies[ci];
  const long long rb = (long long)b * sb;
  if (VEC) {
    const uint4 *src = reinterpret_cast<const uint4 *>(f + c.src + rb);
    uint4 *dst = reinterpret_cast<uint4 *>(f + c.dst + rb);
    const int nv = na * (int)sizeof(E) / 16;
    for (int i = threadIdx.x; i < nv; i += blockDim.x) dst[i] = src[i];
  } else {
    for (int a = threadIdx.x; a < na; a += blockDim.x) f[c.dst + rb + a * sa] = f[c.src + rb + a * sa];
  }
}

template <class E>
cudaError_t launch_e(const PlaneCopy *copies, int ncopies, void *field, int na, int nb,
                     long long sa, long long sb, bool vec, cudaStream_t s) {
  const unsigned blocks = (unsigned)((long long)ncopies * nb);
  if (vec)
    k_halo_planes<E, true><<<blocks, 256, 0, s>>>(copies, (E *)field, na, nb, sa, sb);
  else
    k_halo_planes<E, false><<<blocks, 256, 0, s>>>(copies, (E *)field, na, nb, sa, sb);
  return cudaGetLastError();
}

// Several fields' copies of one dimension in one launch: blockIdx.y picks the
// job (a field with its plane table and geometry), blockIdx.x a (copy, plane
// row) of it; blocks beyond a job's copies x rows exit.
template <class E>
__global__ void __launch_bounds__(256) k_halo_jobs(const HaloJobs jobs) {
  const HaloJob &j = jobs.j[blockIdx.y];
  const long long blk = blockIdx.x;
  if (blk >= (long long)j.ncopies * j.nb) return;
  const int ci = (int)(blk / j.nb), b = (int)(blk % j.nb);
  const PlaneCopy c = j.copies[ci];
  E *f = reinterpret_cast<E *>(j.field);
  const long long rb = (long long)b * j.sb;
  if (j.vec) {
    const uint4 *src = reinterpret_cast<const uint4 *>(f + c.src + rb);
    uint4 *dst = reinterpret_cast<uint4 *>(f + c.dst + rb);
    const int nv = j.na * (int)sizeof(E) / 16;
    for (int i = threadIdx.x; i < nv; i += blockDim.x) dst[i] = src[i];
  } else {
    for (int a = threadIdx.x; a < j.na; a += blockDim.x) f[c.dst + rb + a * j.sa] = f[c.src + rb + a * j.sa];
  }
}

// The halo update of a field of the grid's own size in one launch (the
// gather form of update_halo!): every halo cell receives the value that the
// plane copies in the order x, y, z would leave in it. Following the copies
// backwards from the cell (z, then y, then x), wherever its coordinate in
// dimension d is 0 (n_d - 1) and its current subdomain has a left (right)
// neighbour in d, the value comes from that neighbour's cell with coordinate
// n_d - o_d (o_d - 1). The chain ends at a cell that no copy writes (an inner
// point, or a boundary cell without neighbour), so the launch never reads a
// cell it writes, and one launch gives the sequential result.
//
// One block per row of the subdomain's boundary shell: rows of the z faces
// (2 ny per subdomain, x from 0 to nx - 1), of the y faces with z inner
// (2 (nz - 2)), and the x face columns with y, z inner (2 (nz - 2), y along
// the row). A face row's z and y steps are the same for every x: it is copied
// as a whole from its source row, then its two end cells take their x step.
// With HaloGather::skipx the x-face columns are left out (the launch before
// filled them); the rows do not read them (their end cells' x step reads
// the source point itself).
__device__ __forceinline__ void gather_step(const HaloGather &h, int d, int &s, int &c,
                                            bool &moved) {
  const int side = c == 0 ? 0 : (c == h.n[d] - 1 ? 1 : -1);
  if (side < 0) return;
  const int nb = h.nbr[6 * s + 2 * d + side];
  if (nb < 0) return;
  s = nb;
  c = side ? h.o[d] - 1 : h.n[d] - h.o[d];
  moved = true;
}

template <class E, bool VEC>
__global__ void __launch_bounds__(256) k_halo_gather(E *__restrict__ f, const HaloGather h) {
  const int nx = h.n[0], ny = h.n[1], nz = h.n[2];
  const int rows = 2 * ny + (h.skipx ? 2 : 4) * (nz - 2);
  const int s0 = (int)(blockIdx.x / rows);
  int row = (int)(blockIdx.x % rows);
  const long long sy = nx, sz = (long long)nx * ny;
  if (row < 2 * ny + 2 * (nz - 2)) {
    int y, z;
    if (row < 2 * ny) {
      y = row % ny;
      z = row < ny ? 0 : nz - 1;
    } else {
      row -= 2 * ny;
      z = 1 + row % (nz - 2);
      y = row < nz - 2 ? 0 : ny - 1;
    }
    int s = s0, cy = y, cz = z;
    bool moved = false;
    gather_step(h, 2, s, cz, moved);
    gather_step(h, 1, s, cy, moved);
    const long long di = (long long)s0 * h.nloc + sy * y + sz * z;
    const long long si = (long long)s * h.nloc + sy * cy + sz * cz;
    E *dst = f + di;
    const E *src = f + si;
    const long long total = h.nloc * h.nsub;
    if (moved && in_bounds(di, total) && in_bounds(di + nx - 1, total) && in_bounds(si, total) &&
        in_bounds(si + nx - 1, total)) {
      if (VEC) {
        const int nv = nx * (int)sizeof(E) / 16;
        for (int i = threadIdx.x; i < nv; i += blockDim.x)
          reinterpret_cast<uint4 *>(dst)[i] = reinterpret_cast<const uint4 *>(src)[i];
      } else {
        for (int x = threadIdx.x; x < nx; x += blockDim.x) dst[x] = src[x];
      }
    }
    __syncthreads();  // the row's end cells after its whole-row copy
    if (threadIdx.x < 2) {
      const int x = threadIdx.x ? nx - 1 : 0;
      int ss = s, cx = x;
      bool mx = false;
      gather_step(h, 0, ss, cx, mx);
      const long long xi = (long long)ss * h.nloc + cx + sy * cy + sz * cz;
      if (mx && in_bounds(di + x, total) && in_bounds(xi, total)) dst[x] = f[xi];
    }
  } else {
    // an x face column: x = 0 or nx - 1, z inner, y = 1 .. ny - 2
    row -= 2 * ny + 2 * (nz - 2);
    const int z = 1 + row % (nz - 2), x = row < nz - 2 ? 0 : nx - 1;
    int s = s0, cx = x;
    bool moved = false;
    gather_step(h, 0, s, cx, moved);
    if (!moved) return;
    const long long di = (long long)s0 * h.nloc + x + sz * z;
    const long long si = (long long)s * h.nloc + cx + sz * z;
    const long long total = h.nloc * h.nsub;
    E *dst = f + di;
    const E *src = f + si;
    for (int y = 1 + threadIdx.x; y <= ny - 2; y += blockDim.x)
      if (in_bounds(di + sy * y, total) && in_bounds(si + sy * y, total)) dst[sy * y] = src[sy * y];
  }
}

// The transpose of one dimension's plane copies (the adjoint of
// update_halo!, dimension by dimension in the order z, y, x): per (copy,
// plane row b), every point adds its dst entry into its src entry and sets
// the dst entry to 0. The copies' dst planes (0, n - 1) are never src planes
// (o - 1, n - o); a src plane feeds one dst plane, except on a dimension of
// 2o - 1 points, where o - 1 = n - o feeds both: the adds are atomic.
template <class E>
__global__ void __launch_bounds__(256)
    k_halo_planes_adj(const PlaneCopy *__restrict__ copies, E *__restrict__ f, int na, int nb,
                      long long sa, long long sb) {
  const int ci = blockIdx.x / nb, b = blockIdx.x % nb;
  const PlaneCopy c = copies[ci];
  const long long rb = (long long)b * sb;
  for (int a = threadIdx.x; a < na; a += blockDim.x) {
    const long long i = c.dst + rb + a * sa, j = c.src + rb + a * sa;
    atomicAdd(f + j, f[i]);
    f[i] = E(0);
  }
}

bool vec_rows(size_t elem_size, int na, long long sa, long long sb, const void *field) {
  return sa == 1 && ((long long)na * (long long)elem_size) % 16 == 0 && sb % na == 0 &&
         reinterpret_cast<uintptr_t>(field) % 16 == 0;
}

}  // namespace

cudaError_t launch_halo_jobs(size_t elem_size, HaloJobs jobs, int njobs, cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  if (njobs > kMaxHaloJobs) return cudaErrorInvalidValue;
  long long blocks = 0;
  for (int i = 0; i < njobs; ++i) {
    HaloJob &j = jobs.j[i];
    j.vec = vec_rows(elem_size, j.na, j.sa, j.sb, j.field) ? 1 : 0;
    blocks = std::max(blocks, (long long)j.ncopies * j.nb);
  }
  if (blocks == 0) return cudaSuccess;
  if (blocks >= (1ll << 31)) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)blocks, (unsigned)njobs);
  switch (elem_size) {
    case 8: k_halo_jobs<unsigned long long><<<grid, 256, 0, s>>>(jobs); break;
    case 4: k_halo_jobs<unsigned int><<<grid, 256, 0, s>>>(jobs); break;
    case 2: k_halo_jobs<unsigned short><<<grid, 256, 0, s>>>(jobs); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_halo(size_t elem_size, const PlaneCopy *copies, int ncopies,
                        void *field, int na, int nb, long long sa, long long sb,
                        cudaStream_t s) {
  if (ncopies <= 0) return cudaSuccess;
  if ((long long)ncopies * nb >= (1ll << 31)) return cudaErrorInvalidValue;
  // 16-byte vectors: contiguous rows (sa = 1) of a 16-byte multiple whose
  // starts are multiples of the row length (the halo tables' plane offsets
  // are multiples of n_x = na for the y and z planes, and so is sb)
  const bool vec = vec_rows(elem_size, na, sa, sb, field);
  switch (elem_size) {
    case 8: return launch_e<unsigned long long>(copies, ncopies, field, na, nb, sa, sb, vec, s);
    case 4: return launch_e<unsigned int>(copies, ncopies, field, na, nb, sa, sb, vec, s);
    case 2: return launch_e<unsigned short>(copies, ncopies, field, na, nb, sa, sb, vec, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_halo_adjoint(size_t elem_size, const PlaneCopy *copies, int ncopies,
                                void *field, int na, int nb, long long sa, long long sb,
                                cudaStream_t s) {
  if (ncopies <= 0) return cudaSuccess;
  if ((long long)ncopies * nb >= (1ll << 31)) return cudaErrorInvalidValue;
  const unsigned blocks = (unsigned)((long long)ncopies * nb);
  if (elem_size == 8)
    k_halo_planes_adj<double><<<blocks, 256, 0, s>>>(copies, (double *)field, na, nb, sa, sb);
  else if (elem_size == 4)
    k_halo_planes_adj<float><<<blocks, 256, 0, s>>>(copies, (float *)field, na, nb, sa, sb);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_halo_gather(size_t elem_size, void *field, const HaloGather &h,
                               cudaStream_t s) {
  if (h.n[0] < 3 || h.n[1] < 3 || h.n[2] < 3) return cudaErrorInvalidValue;
  const long long blocks = (long long)h.nsub * (2 * h.n[1] + (h.skipx ? 2 : 4) * (h.n[2] - 2));
  if (blocks <= 0) return cudaSuccess;
  if (blocks >= (1ll << 31)) return cudaErrorInvalidValue;
  const bool vec = ((long long)h.n[0] * (long long)elem_size) % 16 == 0 &&
                   reinterpret_cast<uintptr_t>(field) % 16 == 0;
  const unsigned b = (unsigned)blocks;
  switch (elem_size) {
    case 8:
      if (vec) k_halo_gather<unsigned long long, true><<<b, 256, 0, s>>>((unsigned long long *)field, h);
      else k_halo_gather<unsigned long long, false><<<b, 256, 0, s>>>((unsigned long long *)field, h);
      break;
    case 4:
      if (vec) k_halo_gather<unsigned, true><<<b, 256, 0, s>>>((unsigned *)field, h);
      else k_halo_gather<unsigned, false><<<b, 256, 0, s>>>((unsigned *)field, h);
      break;
    case 2:
      if (vec) k_halo_gather<unsigned short, true><<<b, 256, 0, s>>>((unsigned short *)field, h);
      else k_halo_gather<unsigned short, false><<<b, 256, 0, s>>>((unsigned short *)field, h);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t halo_bounds_flag(unsigned *out, bool clear) { return read_bounds_flag(out, clear); }

}  // namespace igg
