// FP64 reductions with a fixed summation order: each block of the first
// kernel walks a fixed grid-stride sequence and combines its threads in a
// fixed tree, writing one partial per block to a scratch array; one block of
// the second kernel combines the partials the same way. The result does not
// depend on timing, so repeated calls give identical bits.
#include <cuda_bf16.h>

#include "igg_internal.h"

namespace igg {
namespace {

constexpr int kRedThreads = 256;

__device__ __forceinline__ double to64(const double *p, size_t i) { return p[i]; }
__device__ __forceinline__ double to64(const float *p, size_t i) { return (double)p[i]; }
__device__ __forceinline__ double to64(const __nv_bfloat16 *p, size_t i) {
  return (double)__bfloat162float(p[i]);
}

__device__ __forceinline__ double neg_inf() {
  return __longlong_as_double((long long)0xfff0000000000000ULL);
}

template <int OP>
__device__ __forceinline__ double combine(double acc, double v) {
  if (OP == IGG_RED_MAX) return v > acc ? v : acc;
  return acc + v;
}

template <int OP>
__device__ double block_reduce(double v) {
  __shared__ double sh[kRedThreads];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] = combine<OP>(sh[threadIdx.x], sh[threadIdx.x + w]);
    __syncthreads();
  }
  return sh[0];
}

template <int OP, class S>
__global__ void __launch_bounds__(kRedThreads)
    k_reduce_partial(const S *__restrict__ a, const S *__restrict__ b, size_t n,
                     double *__restrict__ partial) {
  double acc = OP == IGG_RED_MAX ? neg_inf() : 0.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double va = to64(a, i);
    double term;
    if (OP == IGG_RED_SUM_DIV) {
      term = va / to64(b, i);
    } else if (OP == IGG_RED_SUM_SQDIFF) {
      const double d = va - to64(b, i);
      term = d * d;
    } else {
      term = va;
    }
    acc = combine<OP>(acc, term);
  }
  const double r = block_reduce<OP>(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = r;
}

template <int OP>
__global__ void __launch_bounds__(kRedThreads)
    k_reduce_final(const double *__restrict__ partial, int np, double *__restrict__ out) {
  double acc = OP == IGG_RED_MAX ? neg_inf() : 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc = combine<OP>(acc, partial[i]);
  const double r = block_reduce<OP>(acc);
  if (threadIdx.x == 0) *out = r;
}

template <int OP, class S>
cudaError_t run(const void *a, const void *b, size_t n, double *scratch, int nblocks,
                double *out, cudaStream_t s) {
  k_reduce_partial<OP, S><<<nblocks, kRedThreads, 0, s>>>((const S *)a, (const S *)b, n, scratch);
  k_reduce_final<OP><<<1, kRedThreads, 0, s>>>(scratch, nblocks, out);
  return cudaGetLastError();
}

template <int OP>
cudaError_t run_t(igg_dtype dt, const void *a, const void *b, size_t n, double *scratch,
                  int nblocks, double *out, cudaStream_t s) {
  switch (dt) {
    case IGG_F64: return run<OP, double>(a, b, n, scratch, nblocks, out, s);
    case IGG_F32: return run<OP, float>(a, b, n, scratch, nblocks, out, s);
    case IGG_BF16: return run<OP, __nv_bfloat16>(a, b, n, scratch, nblocks, out, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_reduce(int op, const void *a, const void *b, size_t n, igg_dtype dt,
                          double *scratch, int nblocks, double *out, cudaStream_t s) {
  switch (op) {
    case IGG_RED_MAX: return run_t<IGG_RED_MAX>(dt, a, b, n, scratch, nblocks, out, s);
    case IGG_RED_SUM: return run_t<IGG_RED_SUM>(dt, a, b, n, scratch, nblocks, out, s);
    case IGG_RED_SUM_DIV: return run_t<IGG_RED_SUM_DIV>(dt, a, b, n, scratch, nblocks, out, s);
    case IGG_RED_SUM_SQDIFF:
      return run_t<IGG_RED_SUM_SQDIFF>(dt, a, b, n, scratch, nblocks, out, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace igg
