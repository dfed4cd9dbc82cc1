// Per-point arithmetic of the adjoint step, shared by the adjoint kernels so
// that every kernel produces the same bits for the same point.
//
// Given lam_in = dJ/dT_{n+1} (the adjoint of Fig. 1's step!, transposed):
//   v[q]       = Ci[q] * lam_in[q] on inner q, 0 elsewhere,
//   lam_out[q] = lam_in[q] + wc v[q] + sum_d w_d (v[q-e_d] + v[q+e_d]),
//   gCi[p]    += lam_in[p] * l(T_n)[p] on inner p (FP64 accumulator).
//
// FP32 fields: v and lam_out in FP32 (FMA order below), the gCi increment
// lam_in * l in FP64 from the two FP32 factors widened exactly by bit moves.
//
// FP64 fields: lam_in changes sign from point to point, so the emulated
// cell's exact integer differences do not apply to the v sums; GB300 issues
// about two FP64 instructions per SM and clock, so the seven-term FP64 sum
// (eight FP64 instructions with v) caps the step near a third of HBM speed.
// The sum is formed in float pairs (h + l, ~48-bit significand) on the FP32
// pipe instead:
//   * each FP64 input x splits into x = h + l by moving bit fields (h: sign,
//     exponent and the leading 23 fraction bits; l: the other 29 bits,
//     rounded to 24), |x - (h + l)| <= 2^-48 |x|;
//   * v = Ci * lam with an error-free FMA product of the pairs, normalised;
//   * lam_out = lam_in + wc v + sum_d w_d (v- + v+) as a compensated dot
//     product (Ogita, Rump and Oishi's Dot2 on the pairs): error-free
//     products and two-sums of the leading parts, every small part gathered
//     in one FP32 accumulator; the pair (acc, err) is widened exactly and
//     rounded to FP64 with one FP64 add.
// The result lies within about 2^-45 of |lam_in| + sum |w v| of the exact
// sum (the FP64 sum: about 2^-51). The pair path needs |lam| in
// [2^-40, 2^41), Ci in [2^-20, 2^21) (or zero) and weights w_d in
// [2^-18, 2^18], so that no partial product or error term leaves the normal
// FP32 range; a point whose stencil holds any other value takes the FP64 sum
// (below), chosen from the point's own inputs only.
#pragma once

#include "cell.cuh"
#include "pair.cuh"

namespace igg {
namespace {

// exponent half-widths of the pair path's input ranges
constexpr unsigned kPairLamE = 40, kPairCiE = 20;
static_assert(kPairLamE <= kPairMaxRadius && kPairCiE <= kPairMaxRadius,
              "pair_ok radii must stay inside pair_split's range");

// lam as a pair, NaN in h when lam lies outside the pair range (the
// point's lam_out then takes the FP64 sum)
__device__ __forceinline__ FF pair_lam(double lam) {
  FF q = pair_split(lam);
  q.h = pair_ok(lam, kPairLamE) ? q.h : __int_as_float(0x7FC00000);
  return q;
}

// Ci as a pair, NaN in h outside the pair range
__device__ __forceinline__ FF pair_ci(double ci) {
  FF b = pair_split(ci);
  b.h = pair_ok(ci, kPairCiE) ? b.h : __int_as_float(0x7FC00000);
  return b;
}

// v of one point for FP64 fields as a normalised pair from the pairs of lam
// (pair_lam) and Ci (pair_ci); (0, 0) off the inner points; NaN in h when
// either pair holds one (a value outside the pair range).
__device__ __forceinline__ FF adj_v_pairs(const FF &a, const FF &b, bool inner) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  e = __fmaf_rn(a.l, b.l, e);
  FF v;
  float q;
  v.h = fast_two_sum(p, e, q);
  v.l = q;
  v.h = inner ? v.h : 0.f;
  v.l = inner ? v.l : 0.f;
  return v;
}

__device__ __forceinline__ FF adj_v_pair(const FF &a, double ci, bool inner) {
  return adj_v_pairs(a, pair_ci(ci), inner);
}

// v of one point for FP64 fields in FP64 (the FP64 sum's input)
__device__ __forceinline__ double adj_v64(double lam, double ci, bool inner) {
  return inner ? __dmul_rn(ci, lam) : 0.0;
}

// v of one point for FP32 fields
__device__ __forceinline__ float adj_v32(float lam, float ci, bool inner) {
  return inner ? __fmul_rn(ci, lam) : 0.f;
}

// Weights of the adjoint: the FP64 weights, the same as float pairs (x, y,
// z, centre), and whether the pair path may run (weights in range).
struct AdjW {
  W<double> w;
  float wh[4], wl[4];
  bool pair;
};

__device__ __forceinline__ AdjW make_adj_w(const Coef &c) {
  AdjW a;
  a.w = make_w(c, 0.0);
  const double d[4] = {c.wx, c.wy, c.wz, c.wc};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    a.wh[i] = __double2float_rn(d[i]);
    a.wl[i] = __double2float_rn(__dsub_rn(d[i], (double)a.wh[i]));
  }
  bool ok = true;
#pragma unroll
  for (int i = 0; i < 3; ++i) ok = ok && d[i] >= 0x1p-18 && d[i] <= 0x1p18;
  a.pair = ok;
  return a;
}

// lam_out of one point on the pair path from lam as a pair (pair_lam);
// false when the point must take the FP64 sum (a value outside the pair
// ranges: a NaN reaches acc; or weights outside theirs).
__device__ __forceinline__ bool adj_out_pair(const FF &lq, const FF &vc, const FF &vxm,
                                             const FF &vxp, const FF &vym, const FF &vyp,
                                             const FF &vzm, const FF &vzp, const AdjW &a,
                                             double &out) {
  float acc = lq.h, err = lq.l;
  dot2_term(acc, err, a.wh[3], a.wl[3], vc.h, vc.l);
  dot2_pair(acc, err, a.wh[0], a.wl[0], vxm, vxp);
  dot2_pair(acc, err, a.wh[1], a.wl[1], vym, vyp);
  dot2_pair(acc, err, a.wh[2], a.wl[2], vzm, vzp);
  // a finite acc bounds err: both widen exactly (f2d_finite)
  out = __dadd_rn(f2d_finite(acc), f2d_finite(err));
  return a.pair && acc == acc;
}

// lam_out of one point in FP64
__device__ __forceinline__ double adj_out_f64(double lam, double vc, double vxm, double vxp,
                                              double vym, double vyp, double vzm, double vzp,
                                              const W<double> &w) {
  double acc = __fma_rn(w.wc, vc, lam);
  acc = __fma_rn(w.wx, __dadd_rn(vxm, vxp), acc);
  acc = __fma_rn(w.wy, __dadd_rn(vym, vyp), acc);
  return __fma_rn(w.wz, __dadd_rn(vzm, vzp), acc);
}

// lam_out of one point for FP32 fields
__device__ __forceinline__ float adj_out_f32(float lam, float vc, float vxm, float vxp, float vym,
                                             float vyp, float vzm, float vzp, const W<float> &w) {
  float acc = __fmaf_rn(w.wc, vc, lam);
  acc = __fmaf_rn(w.wx, __fadd_rn(vxm, vxp), acc);
  acc = __fmaf_rn(w.wy, __fadd_rn(vym, vyp), acc);
  return __fmaf_rn(w.wz, __fadd_rn(vzm, vzp), acc);
}

// The FP64 weighted Laplacian of T_n (the forward cell's FP64 order)
__device__ __forceinline__ double adj_lap64(double c, double xm, double xp, double ym, double yp,
                                            double zm, double zp, const W<double> &w) {
  double l = __dmul_rn(w.wc, c);
  l = __fma_rn(w.wx, __dadd_rn(xm, xp), l);
  l = __fma_rn(w.wy, __dadd_rn(ym, yp), l);
  return __fma_rn(w.wz, __dadd_rn(zm, zp), l);
}

// The FP32 weighted Laplacian of T_n (the forward FP32 cell's order:
// differences first)
__device__ __forceinline__ float adj_lap32(float c, float xm, float xp, float ym, float yp,
                                           float zm, float zp, const W<float> &w) {
  const float ex = __fadd_rn(__fsub_rn(xp, c), __fsub_rn(xm, c));
  const float ey = __fadd_rn(__fsub_rn(yp, c), __fsub_rn(ym, c));
  const float ez = __fadd_rn(__fsub_rn(zp, c), __fsub_rn(zm, c));
  float l = __fmul_rn(w.wx, ex);
  l = __fmaf_rn(w.wy, ey, l);
  return __fmaf_rn(w.wz, ez, l);
}

// g + lam_in * l(T_n) for an inner point, g elsewhere. FP64 fields form l
// with the emulated cell's exact differences: where the stencil shares sign
// and exponent (T_n is a forward state, smooth) from the bit patterns, where
// it crosses one power of two from the shifted significands
// (emu_spread_d); other stencils take the FP64 sum. The second and third
// forms are reached only by warps with a point that needs them (branches on
// warp votes). Every lane of the warp calls it.
__device__ __forceinline__ double gci_add(double g, bool inner, double la, double t, double xm,
                                          double xp, double ym, double yp, double zm, double zp,
                                          const W<double> &w) {
  const double tn[6] = {xm, xp, ym, yp, zm, zp};
  unsigned hn[6];
  unsigned long long nb[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    hn[i] = dhi(tn[i]);
    nb[i] = dbits(tn[i]);
  }
  const bool ok = emu_fast_ok(dhi(t), hn);
  double r = g;
  if (w.ng == 1) r = emu_apply(g, la, emu_lap<1>(t, nb, w));
  else if (w.ng == 2) r = emu_apply(g, la, emu_lap<2>(t, nb, w));
  else r = emu_apply(g, la, emu_lap<3>(t, nb, w));
  if (!__all_sync(0xffffffffu, ok || !inner)) {
    long long D[3];
    unsigned sh;
    const bool ok2 = emu_spread_d(t, nb, D, sh);
    if (inner && !ok && ok2) {
      if (w.ng == 1) r = emu_apply(g, la, emu_lap_d<1>(D, sh, w));
      else if (w.ng == 2) r = emu_apply(g, la, emu_lap_d<2>(D, sh, w));
      else r = emu_apply(g, la, emu_lap_d<3>(D, sh, w));
    }
    const bool f64 = inner && !ok && !ok2;
    if (__any_sync(0xffffffffu, f64)) {
      if (f64) r = __fma_rn(la, adj_lap64(t, xm, xp, ym, yp, zm, zp, w), g);
    }
  }
  return inner ? r : g;
}
__device__ __forceinline__ double gci_add(double g, bool inner, float la, float t, float xm,
                                          float xp, float ym, float yp, float zm, float zp,
                                          const W<float> &w) {
  const float l = adj_lap32(t, xm, xp, ym, yp, zm, zp, w);
  return inner ? __fma_rn(f2d_bits(la), f2d_bits(l), g) : g;
}

// The storage type's adjoint arithmetic behind one interface: the v type,
// the lam type the sum starts from (FP64: the pair of pair_lam), the
// weights, v of a point, lam_out of a point (false: take the FP64 sum) and
// the weights of the Laplacian of T_n.
template <class S>
struct AdjOps;
template <>
struct AdjOps<double> {
  using VT = FF;
  using LT = FF;
  using WT = AdjW;
  static __device__ __forceinline__ AdjW weights(const Coef &c) { return make_adj_w(c); }
  static __device__ __forceinline__ FF lam(double l) { return pair_lam(l); }
  static __device__ __forceinline__ FF v(const FF &lq, double ci, bool inner) {
    return adj_v_pair(lq, ci, inner);
  }
  static __device__ __forceinline__ bool out(const FF &lq, const FF &vc, const FF &vxm,
                                             const FF &vxp, const FF &vym, const FF &vyp,
                                             const FF &vzm, const FF &vzp, const AdjW &a,
                                             double &o) {
    return adj_out_pair(lq, vc, vxm, vxp, vym, vyp, vzm, vzp, a, o);
  }
  static __device__ __forceinline__ const W<double> &lapw(const AdjW &a) { return a.w; }
};
template <>
struct AdjOps<float> {
  using VT = float;
  using LT = float;
  using WT = W<float>;
  static __device__ __forceinline__ W<float> weights(const Coef &c) { return make_w(c, 0.f); }
  static __device__ __forceinline__ float lam(float l) { return l; }
  static __device__ __forceinline__ float v(float lq, float ci, bool inner) {
    return adj_v32(lq, ci, inner);
  }
  static __device__ __forceinline__ bool out(float lq, float vc, float vxm, float vxp, float vym,
                                             float vyp, float vzm, float vzp, const W<float> &w,
                                             float &o) {
    o = adj_out_f32(lq, vc, vxm, vxp, vym, vyp, vzm, vzp, w);
    return true;
  }
  static __device__ __forceinline__ const W<float> &lapw(const W<float> &w) { return w; }
};

}  // namespace
}  // namespace igg
