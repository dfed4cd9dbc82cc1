// FP64 reductions with a fixed summation order: each block of the first
// kernel walks a fixed grid-stride sequence and combines its threads in a
// fixed tree, writing one partial per block to a scratch array; one block of
// the second kernel combines the partials the same way. The result does not
// depend on timing, so repeated calls give identical bits.
#include <cuda_bf16.h>

#include <mutex>

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

// ===========================================================================
// Reduction that allocates nothing (igg_reduce_noalloc).
//
// Same terms and the same final kernel as igg_reduce, but the first kernel
// gives each block one contiguous chunk of kNoAllocChunk elements, and the
// partial sums go to a file-scope device array instead of allocated memory.
// The array lives in every GPU that loads the library, until the process
// exits. Every partial the final kernel reads is written earlier in the same
// call, so stale contents from a previous call never reach a result.
// ===========================================================================
namespace igg {
namespace {

constexpr size_t kNoAllocChunk = 65536;       // elements per block
constexpr int kNoAllocMaxPartials = 32768;    // 256 KB of partial sums
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxPartials];

template <int OP, class S>
__global__ void __launch_bounds__(kRedThreads)
    k_reduce_chunks(const S *__restrict__ a, const S *__restrict__ b, size_t n,
                    double *__restrict__ partial) {
  double acc = OP == IGG_RED_MAX ? neg_inf() : 0.0;
  const size_t begin = (size_t)blockIdx.x * kNoAllocChunk;
  size_t end = begin + kNoAllocChunk;
  if (end > n) end = n;
  for (size_t i = begin + threadIdx.x; i < end; i += kRedThreads) {
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

template <int OP, class S>
cudaError_t run_chunks(const void *a, const void *b, size_t n, double *partials, int nb,
                       double *out, cudaStream_t s) {
  k_reduce_chunks<OP, S><<<nb, kRedThreads, 0, s>>>((const S *)a, (const S *)b, n, partials);
  k_reduce_final<OP><<<1, kRedThreads, 0, s>>>(partials, nb, out);
  return cudaGetLastError();
}

template <int OP>
cudaError_t run_chunks_t(igg_dtype dt, const void *a, const void *b, size_t n, double *partials,
                         int nb, double *out, cudaStream_t s) {
  switch (dt) {
    case IGG_F64: return run_chunks<OP, double>(a, b, n, partials, nb, out, s);
    case IGG_F32: return run_chunks<OP, float>(a, b, n, partials, nb, out, s);
    case IGG_BF16: return run_chunks<OP, __nv_bfloat16>(a, b, n, partials, nb, out, s);
  }
  return cudaErrorInvalidValue;
}

std::mutex g_noalloc_mu;
double *g_noalloc_addr[kNoAllocMaxDevices] = {nullptr};

// Device address of g_noalloc_partials on the current device, looked up once
// per device. In host code the array's name is only a host-side stand-in, so
// the kernels get this address instead.
int noalloc_partials(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= kNoAllocMaxDevices)
    return set_error(IGG_EINVAL, "device index %d >= %d", dev, kNoAllocMaxDevices);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(partial sums)");
    g_noalloc_addr[dev] = (double *)p;
  }
  *out = g_noalloc_addr[dev];
  return IGG_OK;
}

}  // namespace
}  // namespace igg

extern "C" int igg_reduce_noalloc(int op, const void *a, const void *b, size_t n, igg_dtype dt,
                                  double *out_dev, void *stream) {
  using namespace igg;
  clear_error();
  if (op < IGG_RED_MAX || op > IGG_RED_SUM_SQDIFF) return set_error(IGG_EINVAL, "bad op %d", op);
  if (dtype_size(dt) == 0) return set_error(IGG_EINVAL, "unknown dtype %d", (int)dt);
  if (n > 0 && !a) return set_error(IGG_EINVAL, "a is NULL");
  if (n > 0 && (op == IGG_RED_SUM_DIV || op == IGG_RED_SUM_SQDIFF) && !b)
    return set_error(IGG_EINVAL, "b is NULL");
  if (!out_dev) return set_error(IGG_EINVAL, "out_dev is NULL");
  const size_t max_n = kNoAllocChunk * (size_t)kNoAllocMaxPartials;
  if (n > max_n)
    return set_error(IGG_EINVAL,
                     "igg_reduce_noalloc: n = %zu exceeds the maximum of %zu elements "
                     "(%d partial sums of %zu elements each)",
                     n, max_n, kNoAllocMaxPartials, kNoAllocChunk);
  double *partials = nullptr;
  if (int rc = noalloc_partials(&partials)) return rc;
  int nb = (int)((n + kNoAllocChunk - 1) / kNoAllocChunk);
  if (nb < 1) nb = 1;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  switch (op) {
    case IGG_RED_MAX: e = run_chunks_t<IGG_RED_MAX>(dt, a, b, n, partials, nb, out_dev, s); break;
    case IGG_RED_SUM: e = run_chunks_t<IGG_RED_SUM>(dt, a, b, n, partials, nb, out_dev, s); break;
    case IGG_RED_SUM_DIV:
      e = run_chunks_t<IGG_RED_SUM_DIV>(dt, a, b, n, partials, nb, out_dev, s);
      break;
    default:
      e = run_chunks_t<IGG_RED_SUM_SQDIFF>(dt, a, b, n, partials, nb, out_dev, s);
      break;
  }
  if (e != cudaSuccess) return cuda_error(e, "igg_reduce_noalloc launch");
  return IGG_OK;
}
