// TMA and mbarrier helpers shared by the TMA-pipelined kernels: shared
// memory addresses, bounded mbarrier waits (about 2 s of globaltimer, false on
// timeout), 3-D tiled bulk tensor loads, the host-side tensor map encoder
// reached through the runtime's driver entry point, and the work order and
// barrier reduction of the persistent column kernels.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <mutex>

namespace igg {
namespace {

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_test(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s

// Bounded wait for the phase of the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (true) {
    for (int i = 0; i < 64; ++i)
      if (mbar_test(bar, parity)) return true;
    if (globaltimer() - t0 > kWaitNs) return false;
  }
}

__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap *map, int x, int y,
                                            int z, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

template <class S>
bool encode(CUtensorMap *m, const void *base, int nx, int ny, long long nzt, int bx, int by,
            int bz) {
  auto fn = encode_fn();
  if (!fn) return false;
  CUtensorMapDataType t = sizeof(S) == 8   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                          : sizeof(S) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                           : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nzt};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * sizeof(S), (cuuint64_t)nx * ny * sizeof(S)};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, t, 3, const_cast<void *>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

constexpr int kShareZc = 32;  // z chunk of the work order of Share

// Barrier of all warps (named barrier 1) that returns, to every thread,
// whether any thread passed true.
__device__ __forceinline__ bool all_any(bool pred, unsigned nthreads) {
  unsigned r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n"
      " selp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"((unsigned)pred), "r"(nthreads)
      : "memory");
  return r != 0;
}

// One segment of a CTA's share: planes [m0, m1) of column col.
struct Seg {
  int col, m0, m1;
};

// The share [u, u1) of a persistent CTA in the work order (z chunk, column,
// plane in chunk) of ncol columns of nz planes each, walked one segment at a
// time; CTA b of G takes [U b / G, U (b + 1) / G), U = ncol nz, so every CTA
// gets the same number of planes (within one).
struct Share {
  long long u, u1;
  int nz, ncol;
  __device__ bool next(Seg &s) {
    if (u >= u1) return false;
    const long long per = (long long)ncol * kShareZc;   // positions of a full chunk
    const int c = (int)(u / per);
    const int zc = min(kShareZc, nz - c * kShareZc);      // planes per column in chunk c
    const long long w = u - (long long)c * per;
    s.col = (int)(w / zc);
    const int zi = (int)(w - (long long)s.col * zc);
    const int len = (int)min((long long)(zc - zi), u1 - u);
    s.m0 = c * kShareZc + zi;
    s.m1 = s.m0 + len;
    u += len;
    return true;
  }
};

}  // namespace
}  // namespace igg
