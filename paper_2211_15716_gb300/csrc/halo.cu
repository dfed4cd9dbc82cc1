// Halo update kernel (update_halo!, Sec. Approach): on one GPU every
// neighbour lives in the same device memory, so packing, sending and
// unpacking a face collapse into one device-to-device copy of the face plane
// from the sending subdomain's array into the receiving subdomain's halo
// plane. One launch copies all face planes of one dimension of one field;
// the host issues the dimensions in the order x, y, z on one stream, which
// gives edges and corners the values of the sequential exchange.
#include "igg_internal.h"

namespace igg {
namespace {

template <class E>
__global__ void __launch_bounds__(256)
    k_halo_planes(const PlaneCopy *__restrict__ copies, E *__restrict__ f, int na,
                  int nb, long long sa, long long sb) {
  const PlaneCopy c = copies[blockIdx.y];
  const long long npts = (long long)na * nb;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < npts;
       i += (long long)gridDim.x * blockDim.x) {
    const long long a = i % na;
    const long long b = i / na;
    const long long off = a * sa + b * sb;
    f[c.dst + off] = f[c.src + off];
  }
}

}  // namespace

cudaError_t launch_halo(size_t elem_size, const PlaneCopy *copies, int ncopies,
                        void *field, int na, int nb, long long sa, long long sb,
                        cudaStream_t s) {
  if (ncopies <= 0) return cudaSuccess;
  const long long npts = (long long)na * nb;
  long long bx = (npts + 255) / 256;
  if (bx > 1024) bx = 1024;
  const dim3 grid((unsigned)bx, (unsigned)ncopies);
  switch (elem_size) {
    case 8:
      k_halo_planes<unsigned long long><<<grid, 256, 0, s>>>(
          copies, (unsigned long long *)field, na, nb, sa, sb);
      break;
    case 4:
      k_halo_planes<unsigned int><<<grid, 256, 0, s>>>(copies, (unsigned int *)field,
                                                       na, nb, sa, sb);
      break;
    case 2:
      k_halo_planes<unsigned short><<<grid, 256, 0, s>>>(
          copies, (unsigned short *)field, na, nb, sa, sb);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace igg
