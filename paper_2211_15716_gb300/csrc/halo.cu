// Halo update kernel (update_halo!, Sec. Approach): on one GPU every
// neighbour lives in the same device memory, so packing, sending and
// unpacking a face collapse into one device-to-device copy of the face plane
// from the sending subdomain's array into the receiving subdomain's halo
// plane. One launch copies all face planes of one dimension of one field;
// the host issues the dimensions in the order x, y, z on one stream, which
// gives edges and corners the values of the sequential exchange.
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

}  // namespace igg
