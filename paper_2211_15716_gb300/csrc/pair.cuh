// Float-pair ("double-float") arithmetic on the FP32 pipe for FP64 data:
// bit-move conversions between FP64 values and pairs h + l of FP32 values
// (~48-bit significands), and the steps of a compensated dot product (Dot2
// of Ogita, Rump and Oishi) on pairs. GB300 issues about two FP64
// instructions per SM and clock against 128 FP32 lanes, so sums of many
// FP64 terms whose signs vary (where exact integer differences do not
// apply) run faster this way, ending in one FP64 add.
#pragma once

#include <cuda_runtime.h>

namespace igg {
namespace {

// float pair h + l
struct FF {
  float h, l;
};

// True when x is zero or its exponent field lies in [1023 - r, 1023 + r].
// Radii of at most 127 keep that inside pair_split's range [949, 1150].
constexpr unsigned kPairMaxRadius = 127;
__device__ __forceinline__ bool pair_ok(double x, unsigned r) {
  const unsigned hw = (unsigned)__double2hiint(x), lw = (unsigned)__double2loint(x);
  const unsigned E = (hw >> 20) & 0x7FFu;
  return E - (1023u - r) <= 2u * r || ((hw << 1) | lw) == 0u;
}

// x = h + l by bit moves; meaningful for zero and exponent fields in
// [949, 1150] (at 1151 the head's FP32 exponent field would be 255; callers
// check pair_ok with radii of at most 127), any input runs without faults.
__device__ __forceinline__ FF pair_split(double x) {
  const unsigned hw = (unsigned)__double2hiint(x), lw = (unsigned)__double2loint(x);
  const unsigned s = hw & 0x80000000u;
  // (E - 896) << 20 | top fraction bits, then shifted in with the next 3 bits
  const unsigned t = (hw & 0x7FFFFFFFu) - (896u << 20);
  const unsigned hb = __funnelshift_l(lw, t, 3) | s;
  // +-2^(E-1075): the weight of the last fraction bit
  const unsigned sc = (((hw & 0x7FF00000u) - (948u << 20)) << 3) | s;
  FF r;
  r.h = __uint_as_float(hb);
  r.l = __fmul_rn(__uint2float_rn(lw & 0x1FFFFFFFu), __uint_as_float(sc));
  const bool zero = ((hw << 1) | lw) == 0u;
  r.h = zero ? 0.f : r.h;
  r.l = zero ? 0.f : r.l;
  return r;
}

// float -> double by bit moves: exact for normal numbers, infinities and
// NaNs; zero and subnormal inputs give a zero of the same sign.
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned s = b & 0x80000000u, e8 = b & 0x7F800000u;
  unsigned hi = s | (((b & 0x7FFFFFFFu) >> 3) + (896u << 20));
  hi = e8 == 0x7F800000u ? (s | 0x7FF00000u | ((b & 0x007FFFFFu) >> 3)) : hi;
  hi = e8 == 0u ? s : hi;
  const unsigned lo = e8 == 0u ? 0u : b << 29;
  return __hiloint2double((int)hi, (int)lo);
}

// float -> double by bit moves for finite inputs: exact for normal numbers,
// zero and subnormal inputs give a zero of the same sign.
__device__ __forceinline__ double f2d_finite(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned s = b & 0x80000000u;
  const bool z = (b & 0x7F800000u) == 0u;
  const unsigned hi = z ? s : s | (((b & 0x7FFFFFFFu) >> 3) + (896u << 20));
  return __hiloint2double((int)hi, z ? 0 : (int)(b << 29));
}

// error-free sum of two floats: a + b = s + e exactly
__device__ __forceinline__ float pair_two_sum(float a, float b, float &e) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}

// acc + err += w * v (w, v pairs): error-free leading product and sum, the
// small parts into err
__device__ __forceinline__ void dot2_term(float &acc, float &err, float wh, float wl, float vh,
                                          float vl) {
  const float p = __fmul_rn(wh, vh);
  float q = __fmaf_rn(wh, vh, -p);
  q = __fmaf_rn(wh, vl, q);
  q = __fmaf_rn(wl, vh, q);
  float e;
  acc = pair_two_sum(acc, p, e);
  err = __fadd_rn(err, __fadd_rn(e, q));
}

// acc + err += w * (a + b) for the neighbour pair (a, b)
__device__ __forceinline__ void dot2_pair(float &acc, float &err, float wh, float wl, const FF &a,
                                          const FF &b) {
  float t;
  const float s = pair_two_sum(a.h, b.h, t);
  t = __fadd_rn(t, __fadd_rn(a.l, b.l));
  const float p = __fmul_rn(wh, s);
  float q = __fmaf_rn(wh, s, -p);
  q = __fmaf_rn(wh, t, q);
  q = __fmaf_rn(wl, s, q);
  float e;
  acc = pair_two_sum(acc, p, e);
  err = __fadd_rn(err, __fadd_rn(e, q));
}

}  // namespace
}  // namespace igg
