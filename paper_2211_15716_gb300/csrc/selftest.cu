// Self-test of the failure detection of the pipelined kernels, without a GPU
// fault: one CTA whose warps wait on two mbarriers with the kernels' bounded
// wait (about 2 s of globaltimer). Thread 0 completes the phase of the
// second; nothing ever arrives on the first, which warp 0 waits on. The
// warps then agree on stopping through the barrier reduction the persistent
// column kernels use (bar.red.or over named barrier 1), so that no warp is
// left waiting, and the CTA records IGG_DEV_ERR_TIMEOUT in a device word.
#include "igg_internal.h"
#include "tma_util.cuh"

namespace igg {
namespace {

__global__ void __launch_bounds__(256) k_selftest_wait(unsigned *__restrict__ dev_err) {
  __shared__ __align__(8) unsigned long long bars[2];
  const unsigned b_never = smem_u32(&bars[0]), b_done = smem_u32(&bars[1]);
  if (threadIdx.x == 0) {
    mbar_init(b_never, 1);
    mbar_init(b_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_arrive(b_done);  // completes phase 0 of b_done
  const int warp = threadIdx.x >> 5;
  const bool good = __all_sync(0xffffffffu, mbar_wait(warp == 0 ? b_never : b_done, 0));
  if (all_any(!good, blockDim.x) && threadIdx.x == 0) atomicOr(dev_err, IGG_DEV_ERR_TIMEOUT);
}

}  // namespace
}  // namespace igg

extern "C" {

int igg_selftest_bounded_wait(unsigned *status) {
  using namespace igg;
  clear_error();
  if (!status) return set_error(IGG_EINVAL, "status is NULL");
  unsigned *word = nullptr;
  cudaError_t e = cudaMalloc((void **)&word, sizeof(unsigned));
  if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(self-test word)");
  e = cudaMemset(word, 0, sizeof(unsigned));
  if (e == cudaSuccess) {
    k_selftest_wait<<<1, 256>>>(word);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(status, word, sizeof(unsigned), cudaMemcpyDeviceToHost);
  const cudaError_t ef = cudaFree(word);
  if (e != cudaSuccess) return cuda_error(e, "self-test kernel");
  if (ef != cudaSuccess) return cuda_error(ef, "cudaFree(self-test word)");
  return IGG_OK;
}

}  // extern "C"
