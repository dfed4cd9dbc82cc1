// Per-point arithmetic of the diffusion step and 16-byte vector helpers,
// shared by every stencil kernel of the library so that all of them produce
// the same bits for the same point.
//
// Update of one inner point (Fig. 1 step!, reassociated):
//   FP64: s_d = T[-d] + T[+d];  l = wc*T;  l += wx*s_x;  l += wy*s_y;
//         l += wz*s_z;  T2 = T + Ci*l  (FMA where written; round-to-nearest
//         intrinsics so that no other contraction can happen).
//   FP32 / BF16 storage: the differences are formed first, exact for
//   neighbouring values within a factor 2:
//         e_d = (T[+d] - T) + (T[-d] - T);  l = wx*e_x;  l += wy*e_y;
//         l += wz*e_z;  T2 = T + Ci*l.
// w_d = dt*lam/dd^2 and wc = -2*(wx+wy+wz) come from the host in FP64. Only
// + - * and FMA are used.
#pragma once

#include <cuda_bf16.h>

#include "igg_internal.h"

namespace igg {
namespace {

template <class S>
struct Num;

template <>
struct Num<double> {
  using C = double;
  static __device__ __forceinline__ double ld(const double *p) { return __ldg(p); }
  static __device__ __forceinline__ double cv(double v) { return v; }
  static __device__ __forceinline__ void st(double *p, double v) { *p = v; }
};
template <>
struct Num<float> {
  using C = float;
  static __device__ __forceinline__ float ld(const float *p) { return __ldg(p); }
  static __device__ __forceinline__ float cv(float v) { return v; }
  static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
};
template <>
struct Num<__nv_bfloat16> {
  using C = float;
  static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) {
    return __bfloat162float(__ldg(p));
  }
  static __device__ __forceinline__ float cv(__nv_bfloat16 v) { return __bfloat162float(v); }
  static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v) {
    *p = __float2bfloat16_rn(v);
  }
};

template <class C>
struct W {
  C wx, wy, wz, wc;
};

__device__ __forceinline__ W<double> make_w(const Coef &c, double) {
  return {c.wx, c.wy, c.wz, c.wc};
}
__device__ __forceinline__ W<float> make_w(const Coef &c, float) {
  return {(float)c.wx, (float)c.wy, (float)c.wz, (float)c.wc};
}

// The update of one inner point (see the file comment for the order).
__device__ __forceinline__ double cell(double t, double xm, double xp, double ym,
                                       double yp, double zm, double zp, double ci,
                                       const W<double> &w) {
  const double sx = __dadd_rn(xm, xp);
  const double sy = __dadd_rn(ym, yp);
  const double sz = __dadd_rn(zm, zp);
  double l = __dmul_rn(w.wc, t);
  l = __fma_rn(w.wx, sx, l);
  l = __fma_rn(w.wy, sy, l);
  l = __fma_rn(w.wz, sz, l);
  return __fma_rn(ci, l, t);
}

__device__ __forceinline__ float cell(float t, float xm, float xp, float ym,
                                      float yp, float zm, float zp, float ci,
                                      const W<float> &w) {
  const float ex = __fadd_rn(__fsub_rn(xp, t), __fsub_rn(xm, t));
  const float ey = __fadd_rn(__fsub_rn(yp, t), __fsub_rn(ym, t));
  const float ez = __fadd_rn(__fsub_rn(zp, t), __fsub_rn(zm, t));
  float l = __fmul_rn(w.wx, ex);
  l = __fmaf_rn(w.wy, ey, l);
  l = __fmaf_rn(w.wz, ez, l);
  return __fmaf_rn(ci, l, t);
}

template <class S>
struct Vec {
  static constexpr int V = 16 / (int)sizeof(S);
  using C = typename Num<S>::C;
  C v[V];
};

__device__ __forceinline__ void unpack(const uint4 &r, Vec<double> &o) {
  o.v[0] = __hiloint2double((int)r.y, (int)r.x);
  o.v[1] = __hiloint2double((int)r.w, (int)r.z);
}
__device__ __forceinline__ uint4 pack(const Vec<double> &o) {
  uint4 r;
  r.x = (unsigned)__double2loint(o.v[0]);
  r.y = (unsigned)__double2hiint(o.v[0]);
  r.z = (unsigned)__double2loint(o.v[1]);
  r.w = (unsigned)__double2hiint(o.v[1]);
  return r;
}
__device__ __forceinline__ void unpack(const uint4 &r, Vec<float> &o) {
  o.v[0] = __uint_as_float(r.x);
  o.v[1] = __uint_as_float(r.y);
  o.v[2] = __uint_as_float(r.z);
  o.v[3] = __uint_as_float(r.w);
}
__device__ __forceinline__ uint4 pack(const Vec<float> &o) {
  return make_uint4(__float_as_uint(o.v[0]), __float_as_uint(o.v[1]), __float_as_uint(o.v[2]),
                    __float_as_uint(o.v[3]));
}
// BF16 -> FP32 is exact: the 16 bits become the upper half of the float.
__device__ __forceinline__ void unpack(const uint4 &r, Vec<__nv_bfloat16> &o) {
  const unsigned w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    o.v[2 * i] = __uint_as_float(w[i] << 16);
    o.v[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
  }
}
// two FP32 values -> one BF16x2 word (round to nearest even, one packed
// conversion instruction)
__device__ __forceinline__ unsigned bf16x2_bits(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const unsigned *>(&h);
}
__device__ __forceinline__ uint4 pack(const Vec<__nv_bfloat16> &o) {
  return make_uint4(bf16x2_bits(o.v[0], o.v[1]), bf16x2_bits(o.v[2], o.v[3]),
                    bf16x2_bits(o.v[4], o.v[5]), bf16x2_bits(o.v[6], o.v[7]));
}

template <class S>
__device__ __forceinline__ void ldvec(const S *p, Vec<S> &o) {
  unpack(__ldg(reinterpret_cast<const uint4 *>(p)), o);
}

template <class S>
__device__ __forceinline__ typename Num<S>::C ld1(const S *p) {
  return Num<S>::ld(p);
}

}  // namespace
}  // namespace igg
