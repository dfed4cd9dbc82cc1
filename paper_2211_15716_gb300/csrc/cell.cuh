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

// FP64 weights: the doubles, the same weights as float pairs wh + wl for the
// emulated FP64 cell (and scaled copies of them for its fast path: ah, al =
// 2^23 wh, 2^23 wl), and which cell to use.
template <>
struct W<double> {
  double wx, wy, wz, wc;
  float wh[3], wl[3];
  float ah[3], al[3];
  bool emu;
  int ng;  // weight groups (weight_groups)
};

__device__ __forceinline__ W<double> make_w(const Coef &c, double) {
  W<double> w;
  w.wx = c.wx;
  w.wy = c.wy;
  w.wz = c.wz;
  w.wc = c.wc;
  const double d[3] = {c.wx, c.wy, c.wz};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    w.wh[i] = __double2float_rn(d[i]);
    w.wl[i] = __double2float_rn(__dsub_rn(d[i], (double)w.wh[i]));
    w.ah[i] = __fmul_rn(w.wh[i], 8388608.0f);
    w.al[i] = __fmul_rn(w.wl[i], 8388608.0f);
  }
  w.emu = c.f64_emu != 0;
  w.ng = weight_groups(c.wx, c.wy, c.wz);
  return w;
}
__device__ __forceinline__ W<float> make_w(const Coef &c, float) {
  return {(float)c.wx, (float)c.wy, (float)c.wz, (float)c.wc};
}

// The FP64 update of one inner point (see the file comment for the order).
__device__ __forceinline__ double cell_f64(double t, double xm, double xp, double ym,
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


// ---------------------------------------------------------------------------
// FP64 update with FP32/integer arithmetic for the differences ("emulated
// FP64"). GB300 issues about two FP64 instructions per SM and clock, so the
// 8-instruction FP64 cell caps the step near a quarter of HBM speed; the
// emulated cell spends one FP64 FMA per point on its fast path (two on the
// aligned path and in the helpers below) and does the rest on the FP32,
// integer and conversion pipes.
//
// When the seven values of a stencil share sign and exponent field E, their
// IEEE bit patterns, read as 64-bit integers, are K + M with a common K (sign
// and exponent) and 52-bit fractions M, so the second difference in units
// u = 2^(E-1075) is the exact integer
//   D_d = bits(T[-d]) + bits(T[+d]) - 2 bits(T)   (mod 2^64),  |D_d| < 2^53,
// negated for negative values. Dimensions of equal weight are grouped: their
// D_d add exactly into one integer G_g (|G_g| < 2^55), so that the weighted
// sum l = sum_g w_g G_g has one, two or three products. With
// G_g = hi*2^31 + lo (hi = G_g >> 31, |hi| <= 2^24; 0 <= lo < 2^31),
// A = hi*2^31, B1 = lo rounded down to a multiple of 128 and B2 = lo mod 128
// are exact FP32 numbers with G_g = A + B1 + B2. An error-free sum of A and
// B1 gives G_g = s_g + t_g to about 2^-48 relative (A is zero or at least
// 2^31 > B1 in magnitude, so Dekker's fast two-sum is exact); l is formed
// with exact FMA product splits (wh_g + wl_g)(s_g + t_g) and two-sums of the
// leading products (S) plus the small terms (C), to about 2^-44 of
// sum_g |w_g G_g|.
// Finally
//   T2 = fma(+-Ci, S*u, fma(+-Ci, C*u, T))
// in FP64, S*u and C*u widened to FP64 exactly by bit manipulation (the
// scaling by u is an exponent offset folded into the widening).
//
// Stencils whose exponents take two neighbouring values (the shells where a
// smooth field crosses a power of two) get the same weighted sum from exact
// differences of the significands shifted to the smaller exponent's scale
// (emu_spread_d). These helpers form the adjoint's gradient sum (adj_cell.cuh);
// the step's cell (cell_emu, below) uses the one-FMA fast path and, for
// stencils across powers of two or across zero, the aligned path, else
// cell_f64. The choice depends only on the point's inputs, so every kernel
// makes the same choice and produces the same bits.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long dbits(double v) {
  return (unsigned long long)__double_as_longlong(v);
}
__device__ __forceinline__ unsigned dhi(double v) { return (unsigned)__double2hiint(v); }

// float f -> double f * 2^(E-1075), exact for normal f, by moving the float's
// exponent and fraction into the double's fields with the exponent offset
// eoff = (E - 179) << 20 (1023 - 127 + E - 1075 = E - 179). A zero or
// subnormal f gives a value below 2^(E-1201), under 2^-178 of T's magnitude,
// which leaves T2 unchanged.
__device__ __forceinline__ double f2d_scaled(float f, unsigned eoff) {
  const unsigned b = __float_as_uint(f);
  const unsigned hi = (b & 0x80000000u) | (((b & 0x7FFFFFFFu) >> 3) + eoff);
  return __hiloint2double((int)hi, (int)(b << 29));
}

// error-free sum of two floats: a + b = s + e exactly
__device__ __forceinline__ float two_sum(float a, float b, float &e) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}

// error-free sum when |a| >= |b| or a == 0 (Dekker): a + b = s + e exactly
__device__ __forceinline__ float fast_two_sum(float a, float b, float &e) {
  const float s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
  return s;
}

// Fast-path test from the high words: hc of the centre, hn[6] of the
// neighbours. True when all seven share sign and exponent and E lies in
// [949, 1139].
__device__ __forceinline__ bool emu_fast_ok(unsigned hc, const unsigned *hn) {
  const unsigned diff = ((hn[0] ^ hc) | (hn[1] ^ hc) | (hn[2] ^ hc) | (hn[3] ^ hc) |
                         (hn[4] ^ hc) | (hn[5] ^ hc)) &
                        0xFFF00000u;
  const unsigned E = (hc >> 20) & 0x7FFu;
  return diff == 0u && E - 949u <= 190u;
}

// The emulated weighted Laplacian of a fast-path stencil with NG weight
// groups: l = sum_g w_g G_g = (S + C) * u, u = +-2^(E-1075) (sign: bit 31 of
// `sign`; exponent offset for f2d_scaled: eoff). tc is the centre, nb[6] the
// bit patterns of the neighbours in the order x-, x+, y-, y+, z-, z+. Any input
// runs without faults; the value means something only where emu_fast_ok.
struct EmuLap {
  float S, C;
  unsigned eoff, sign;
};

// The weighted sum of exact second differences D[3] (x, y, z; units
// u = +-2^(E-1075), |D_d| < 2^53) with NG weight groups; `scale_hi` is the
// high word of a double with u's sign and exponent field E.
template <int NG>
__device__ __forceinline__ EmuLap emu_lap_d(const long long *D, unsigned scale_hi,
                                            const W<double> &w) {
  long long G[NG];
  if constexpr (NG == 1) {
    G[0] = D[0] + D[1] + D[2];
  } else if constexpr (NG == 2) {
    G[0] = D[0];
    G[1] = D[1] + D[2];
  } else {
    G[0] = D[0];
    G[1] = D[1];
    G[2] = D[2];
  }
  float P[NG], X[NG], R[NG];
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    const unsigned lo = (unsigned)G[g];
    const float A = __fmul_rn(__int2float_rn((int)(G[g] >> 31)), 2147483648.0f);  // hi * 2^31
    const float B1 = __uint2float_rn(lo & 0x7FFFFF80u);
    const float B2 = __uint2float_rn(lo & 0x7Fu);
    float err;
    const float sg = fast_two_sum(A, B1, err);  // A a multiple of 2^31, 0 <= B1 < 2^31
    const float tg = __fadd_rn(err, B2);
    P[g] = __fmul_rn(w.wh[g], sg);
    X[g] = __fmaf_rn(w.wh[g], sg, -P[g]);
    R[g] = __fmaf_rn(w.wl[g], sg, __fmul_rn(w.wh[g], tg));
  }
  EmuLap L;
  if constexpr (NG == 1) {
    L.S = P[0];
    L.C = __fadd_rn(X[0], R[0]);
  } else if constexpr (NG == 2) {
    float e1;
    L.S = two_sum(P[0], P[1], e1);
    L.C = __fadd_rn(__fadd_rn(__fadd_rn(X[0], X[1]), e1), __fadd_rn(R[0], R[1]));
  } else {
    float e1, e2;
    L.S = two_sum(two_sum(P[0], P[1], e1), P[2], e2);
    L.C = __fadd_rn(__fadd_rn(__fadd_rn(X[0], X[1]), __fadd_rn(X[2], e1)),
                    __fadd_rn(__fadd_rn(R[0], R[1]), __fadd_rn(R[2], e2)));
  }
  L.eoff = (scale_hi & 0x7FF00000u) - (179u << 20);
  // the bit differences of negative values carry the opposite sign of the
  // value differences
  L.sign = scale_hi & 0x80000000u;
  return L;
}

template <int NG>
__device__ __forceinline__ EmuLap emu_lap(double tc, const unsigned long long *nb,
                                          const W<double> &w) {
  const unsigned long long c2 = dbits(tc) << 1;
  long long D[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) D[d] = (long long)(nb[2 * d] + nb[2 * d + 1] - c2);
  return emu_lap_d<NG>(D, dhi(tc), w);
}

// base + m * l for an emulated Laplacian l, with two FP64 FMAs (the sign of
// l goes into m).
__device__ __forceinline__ double emu_apply(double base, double m, const EmuLap &L) {
  const double sm =
      __hiloint2double((int)((unsigned)__double2hiint(m) ^ L.sign), __double2loint(m));
  return __fma_rn(sm, f2d_scaled(L.S, L.eoff), __fma_rn(sm, f2d_scaled(L.C, L.eoff), base));
}

// Exact second differences of a stencil whose seven values share the sign
// and whose exponent fields take at most two neighbouring values
// {Emin, Emin + 1} (a smooth field crossing a power of two): each magnitude's
// significand, leading bit included, shifted left by E - Emin is an integer
// of at most 54 bits in units of 2^(Emin - 1075), so the differences are
// exact 64-bit sums. True, with D[3] and the scale's high word (sign,
// exponent field Emin), when the stencil qualifies, Emin lies in
// [949, 1138] and every |D_d| < 2^53 (the range emu_lap_d takes).
__device__ __forceinline__ bool emu_spread_d(double tc, const unsigned long long *nb, long long *D,
                                             unsigned &scale_hi) {
  const unsigned long long cb = dbits(tc);
  const unsigned hc = (unsigned)(cb >> 32);
  unsigned emin = (hc >> 20) & 0x7FFu, emax = emin, sdiff = 0u;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const unsigned h = (unsigned)(nb[i] >> 32);
    const unsigned e = (h >> 20) & 0x7FFu;
    emin = min(emin, e);
    emax = max(emax, e);
    sdiff |= (h ^ hc) & 0x80000000u;
  }
  auto mag = [&](unsigned long long b) -> long long {
    const unsigned e = (unsigned)(b >> 52) & 0x7FFu;
    return (long long)(((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << ((e - emin) & 1u));
  };
  const long long c2 = 2 * mag(cb);
  bool ok = sdiff == 0u && emax - emin <= 1u && emin - 949u <= 189u;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    D[d] = mag(nb[2 * d]) + mag(nb[2 * d + 1]) - c2;
    ok = ok && (unsigned long long)(D[d] + (1ll << 53)) < (1ull << 54);
  }
  scale_hi = (hc & 0x80000000u) | (emin << 20);
  return ok;
}

// ---------------------------------------------------------------------------
// Fast path of the emulated FP64 cell: one FP64 FMA per point.
//
// In units of u = ulp(T) = 2^(E-1075) the update of a stencil whose seven
// values share sign and exponent field E is an update of the bit pattern:
// with the exact integer group sums G_g of the bit-pattern second
// differences (as above, negated differences for negative values included),
//   bits(T2) = bits(T) + Ci * sum_g w_g G_g
// for as long as T2 stays in T's binade. Each G_g is split exactly into
// G_g = Gh 2^23 + Gl with -2^22 <= Gl < 2^22 (Gh = (G_g + 2^22) >> 23).
// Both halves are read off bits as FP32 numbers with exponent 23 minus
// 1.5 2^23: Gl from 2^23 + 2^22 + Gl (the low 23 bits of G_g + 2^22), Gh
// from the integer sum Gh + 0x4B400000, the bits of 1.5 2^23 + Gh, which is
// exact while -2^22 <= Gh < 2^22, i.e. -2^45 - 2^22 <= G_g < 2^45 - 2^22
// (the fast path requires it; the subtraction of 1.5 2^23 is an FP32 add on
// the FMA pipe instead of an integer-to-float conversion). With the weights
// as float pairs,
// S + C = sum_g w_g G_g is formed from error-free FMA products (2^23 wh) Gh,
// the small terms (2^23 wl) Gh and wh Gl, and a two-sum of the leading
// products, to about 2^-46 of sum_g |w_g G_g|. Then
//   T2 = fma(+-Ci, |S| u, T)   (the only FP64 instruction; |S| u widened
//                              to FP64 by moving the FP32 fields),
//   bits(T2) += rint(Ci_f C)   (Ci_f: Ci truncated to 24 bits; rint by
//                              an FP32 FMA adding 1.5 2^23),
// within about one ulp of T2 plus 2^-44 of Ci sum_g |w_g G_g| of the exact
// update. The FP32 arithmetic of the sums runs on pairs of points (float2
// instructions) in the TMA kernel and on single points elsewhere, with the
// same per-point roundings, so both give the same bits.
//
// The fast path applies when the seven values share sign and exponent field
// E in [180, 2008], every Gh in [-2^22, 2^22), Ci is positive with its exponent in
// the FP32 range, |Ci_f C| < 2^22 and T2 (after the correction) keeps T's
// sign and exponent. With |w| <= 2^40 (the host's condition for the emulated
// cell) |S| < 2^90, so |S| u is a normal double for every such E. E, and the
// sign, enter only through the centre; when a point's stencil passes, its
// row neighbour shares them, so the TMA kernel's pairs of points take both
// from the first point of the pair.
// ---------------------------------------------------------------------------
// Pairs of FP32 numbers use the packed instructions. The sums below are
// written so that no product feeds an addition (products are FMAs with a
// zero addend, or folded into the FMA that uses them): the compiler may fuse
// a packed multiply into a following packed addition, which would change the
// rounding against the scalar form.
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float vset(float w, float) { return w; }
__device__ __forceinline__ float2 vset(float w, float2) { return make_float2(w, w); }

constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23

// error-free sum a + b = s + e (Knuth's two-sum), per lane
template <class V>
__device__ __forceinline__ V vtwo_sum(V a, V b, V &e) {
  const V s = vadd(a, b);
  const V bb = vadd(s, vneg(a));
  e = vadd(vadd(a, vneg(vadd(s, vneg(bb)))), vadd(b, vneg(bb)));
  return s;
}

// The centre's part of the fast-path test: sign and exponent field E in
// [180, 2008] (hc: the centre's high word).
__device__ __forceinline__ bool emu2_centre_ok(unsigned hc) {
  return (hc & 0x7FF00000u) - (180u << 20) < (1829u << 20);
}

// Integer part of the fast path for one point: the group sums of the bit-
// pattern second differences, split into the bits gh of the FP32 number
// 1.5 2^23 + Gh and the bits gm of the FP32 number 1.5 2^23 + Gl. True when
// the seven values share sign and exponent and every Gh lies in
// [-2^22, 2^22), i.e. gh in [0x4B000000, 0x4B800000) (the centre's own test
// is emu2_centre_ok). nb: x-, x+, y-, y+, z-, z+.
template <int NG>
__device__ __forceinline__ bool emu2_int(unsigned long long bc, const unsigned long long *nb,
                                         unsigned *gh, unsigned *gm) {
  const unsigned hc = (unsigned)(bc >> 32);
  unsigned o = 0u;
#pragma unroll
  for (int i = 0; i < 6; ++i) o |= (unsigned)(nb[i] >> 32) ^ hc;
  const unsigned long long c2 = bc << 1, B = 1ull << 22;
  unsigned long long G[NG];  // G_g + 2^22 (mod 2^64)
  if constexpr (NG == 1) {
    G[0] = (nb[0] + nb[1] - c2) + (nb[2] + nb[3] - c2) + (nb[4] + nb[5] - c2) + B;
  } else if constexpr (NG == 2) {
    G[0] = nb[0] + nb[1] - c2 + B;
    G[1] = (nb[2] + nb[3] - c2) + (nb[4] + nb[5] - c2) + B;
  } else {
#pragma unroll
    for (int d = 0; d < 3; ++d) G[d] = nb[2 * d] + nb[2 * d + 1] - c2 + B;
  }
  unsigned r = 0u;
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    const unsigned lo = (unsigned)G[g];
    gh[g] = __funnelshift_r(lo, (unsigned)(G[g] >> 32), 23) + 0x4B400000u;
    gm[g] = (lo & 0x7FFFFFu) | 0x4B000000u;
    r |= gh[g] ^ 0x4B000000u;
  }
  return o < (1u << 20) && r < (1u << 23);
}

// S + C = sum_g w_g G_g from the FP32 halves (per lane: one point or two);
// gl holds the FP32 numbers 1.5 2^23 + Gl.
template <int NG, class V>
__device__ __forceinline__ void emu2_sum(const V *gh, const V *gl, const W<double> &w, V &S,
                                         V &C) {
  V P[NG], E[NG], L[NG];
  const V zero = vset(0.0f, V());
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    const V a = vset(w.ah[g], V());
    P[g] = vfma(a, gh[g], zero);  // the rounded product
    E[g] = vfma(a, gh[g], vneg(P[g]));
    L[g] = vadd(gl[g], vset(-kMagic, V()));  // Gl, exact
  }
  V R = vfma(vset(w.wh[0], V()), L[0], zero);
#pragma unroll
  for (int g = 1; g < NG; ++g) R = vfma(vset(w.wh[g], V()), L[g], R);
#pragma unroll
  for (int g = 0; g < NG; ++g) R = vfma(vset(w.al[g], V()), gh[g], R);
  if constexpr (NG == 1) {
    S = P[0];
    C = vadd(E[0], R);
  } else if constexpr (NG == 2) {
    V e;
    S = vtwo_sum(P[0], P[1], e);
    C = vadd(vadd(E[0], E[1]), vadd(e, R));
  } else {
    V e1, e2;
    S = vtwo_sum(vtwo_sum(P[0], P[1], e1), P[2], e2);
    C = vadd(vadd(vadd(E[0], E[1]), vadd(E[2], e1)), vadd(e2, R));
  }
}

// Ci truncated to an FP32 number (meaningful when emu2_apply's Ci condition
// holds: Ci positive with its exponent field in [897, 1150]).
__device__ __forceinline__ float emu2_cif(double ci) {
  return __uint_as_float(__funnelshift_l((unsigned)__double2loint(ci),
                                         (unsigned)__double2hiint(ci) - (896u << 20), 3));
}

// T2 of a fast-path point from S and Kr = fma(Ci_f, C, 1.5 2^23) (one
// rounding: the nearest integer to Ci_f C is bits(Kr) - 0x4B400000 when
// |Ci_f C| < 2^22);
// hc: the high word that gives the point's sign and exponent (see above);
// ok is cleared where the remaining conditions fail.
__device__ __forceinline__ double emu2_apply(unsigned long long bc, unsigned hc, double ci,
                                             float S, float Kr, bool &ok) {
  const unsigned sb = __float_as_uint(S);
  const unsigned eoff = (hc & 0x7FF00000u) - (179u << 20);
  const double sd = __hiloint2double((int)(((sb << 1) >> 4) + eoff), (int)(sb << 29));
  const unsigned cih = (unsigned)__double2hiint(ci);
  const double sci = __hiloint2double((int)(cih ^ ((hc ^ sb) & 0x80000000u)), __double2loint(ci));
  const double t2 = __fma_rn(sci, sd, __longlong_as_double((long long)bc));
  const unsigned long long r =
      dbits(t2) + (unsigned long long)__float_as_uint(Kr) - 0x4B400000ull;
  ok = ok && cih - (897u << 20) < (254u << 20) && fabsf(Kr - kMagic) < 4194304.0f &&
       (((unsigned)(r >> 32) ^ (unsigned)(bc >> 32)) & 0xFFF00000u) == 0u;
  return __longlong_as_double((long long)r);
}

// The fast path for one point; ok tells whether it applies.
template <int NG>
__device__ __forceinline__ double cell_emu_fast(double tc, const unsigned long long *nb,
                                                double ci, const W<double> &w, bool &ok) {
  const unsigned long long bc = dbits(tc);
  unsigned gh[NG], gm[NG];
  ok = emu2_int<NG>(bc, nb, gh, gm) && emu2_centre_ok((unsigned)(bc >> 32));
  float fh[NG], fl[NG];
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    fh[g] = vadd(__uint_as_float(gh[g]), -kMagic);  // Gh, exact where ok
    fl[g] = __uint_as_float(gm[g]);
  }
  float S, C;
  emu2_sum<NG>(fh, fl, w, S, C);
  const float Kr = __fmaf_rn(emu2_cif(ci), C, kMagic);
  return emu2_apply(bc, (unsigned)(bc >> 32), ci, S, Kr, ok);
}

__device__ __forceinline__ double cell_emu_fast(double tc, const unsigned long long *nb,
                                                double ci, const W<double> &w, bool &ok) {
  if (w.ng == 1) return cell_emu_fast<1>(tc, nb, ci, w, ok);
  if (w.ng == 2) return cell_emu_fast<2>(tc, nb, ci, w, ok);
  return cell_emu_fast<3>(tc, nb, ci, w, ok);
}

// ---------------------------------------------------------------------------
// Aligned path of the emulated FP64 cell: stencils whose values differ in
// exponent (a field crossing powers of two) or in sign (a field crossing 0).
//
// Every value is put on the grid of u = 2^(Er-1075), Er the largest exponent
// field of the seven: its significand (leading bit included; none for 0 and
// subnormals, whose exponent field counts as 1) shifted right by Er - E and
// rounded to the nearest integer (halves up), negated when its sign differs
// from the centre's. Values of exponent Er are exact, the others within u/2;
// the second differences of these integers (|I| <= 2^53) are exact. The
// weighted sum S + C = sum_g w_g G_g is formed as on the fast path (same
// split, same float-pair sums) and applied with two FP64 FMAs,
//   T2 = fma(+-Ci, S u, fma(+-Ci, C u, T)),
// so T2 may leave T's binade or sign. The error: the rounding of the values
// to u (at most 2 Ci sum_d w_d u), the two FMAs (an ulp of T2 each, |T2|
// being at most about 2^(Er-1022): within u each) and 2^-44 of
// Ci sum_g |w_g G_g| u, i.e. a few u, u being the ulp of the stencil's
// largest value, like the roundings of the FP64 cell's differences.
// It applies when Er lies in [180, 2008] and every |G_g| < 2^47.
// ---------------------------------------------------------------------------
// b on the grid of 2^(er-1075), signed relative to the centre (bit pattern cb)
__device__ __forceinline__ long long emu3_aligned(unsigned long long b, unsigned long long cb,
                                                  unsigned er) {
  const unsigned e = (unsigned)(b >> 52) & 0x7FFu;
  const unsigned long long m =
      (b & 0xFFFFFFFFFFFFFull) | ((unsigned long long)(e != 0u) << 52);
  const unsigned d = min(er - max(e, 1u), 63u);  // m < 2^53: shifts past 53 give 0
  const unsigned long long q = d ? (m + (1ull << (d - 1u))) >> d : m;
  return ((b ^ cb) >> 63) ? -(long long)q : (long long)q;
}

// Integer part of the aligned path: the group sums of the aligned values'
// second differences split as on the fast path (gh, gm), and er. True when
// er lies in [180, 2008] and every |Gh| < 2^24.
template <int NG>
__device__ __forceinline__ bool emu3_int(unsigned long long bc, const unsigned long long *nb,
                                         int *gh, unsigned *gm, unsigned &er) {
  unsigned e = (unsigned)(bc >> 52) & 0x7FFu;
#pragma unroll
  for (int i = 0; i < 6; ++i) e = max(e, (unsigned)(nb[i] >> 52) & 0x7FFu);
  er = max(e, 1u);
  long long I[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) I[i] = emu3_aligned(nb[i], bc, er);
  const long long c2 = 2 * emu3_aligned(bc, bc, er), B = 1ll << 22;
  long long G[NG];  // G_g + 2^22
  if constexpr (NG == 1) {
    G[0] = (I[0] + I[1] - c2) + (I[2] + I[3] - c2) + (I[4] + I[5] - c2) + B;
  } else if constexpr (NG == 2) {
    G[0] = I[0] + I[1] - c2 + B;
    G[1] = (I[2] + I[3] - c2) + (I[4] + I[5] - c2) + B;
  } else {
#pragma unroll
    for (int d = 0; d < 3; ++d) G[d] = I[2 * d] + I[2 * d + 1] - c2 + B;
  }
  unsigned r = 0u;
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    const unsigned lo = (unsigned)G[g];
    gh[g] = (int)__funnelshift_r(lo, (unsigned)((unsigned long long)G[g] >> 32), 23);
    gm[g] = (lo & 0x7FFFFFu) | 0x4B000000u;
    r |= (unsigned)gh[g] + (1u << 24);
  }
  return er - 180u <= 1828u && r < (1u << 25);
}

// The aligned path for one point; ok tells whether it applies.
template <int NG>
__device__ __forceinline__ double cell_emu_aligned(double tc, const unsigned long long *nb,
                                                   double ci, const W<double> &w, bool &ok) {
  const unsigned long long bc = dbits(tc);
  int gh[NG];
  unsigned gm[NG], er;
  ok = emu3_int<NG>(bc, nb, gh, gm, er);
  float fh[NG], fl[NG];
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    fh[g] = __int2float_rn(gh[g]);
    fl[g] = __uint_as_float(gm[g]);
  }
  EmuLap L;
  emu2_sum<NG>(fh, fl, w, L.S, L.C);
  L.eoff = (er << 20) - (179u << 20);
  L.sign = (unsigned)(bc >> 32) & 0x80000000u;
  return emu_apply(tc, ci, L);
}

__device__ __forceinline__ double cell_emu_aligned(double tc, const unsigned long long *nb,
                                                   double ci, const W<double> &w, bool &ok) {
  if (w.ng == 1) return cell_emu_aligned<1>(tc, nb, ci, w, ok);
  if (w.ng == 2) return cell_emu_aligned<2>(tc, nb, ci, w, ok);
  return cell_emu_aligned<3>(tc, nb, ci, w, ok);
}

// One point: the emulated cell's fast path where it applies, else its
// aligned path where that applies, else cell_f64.
__device__ __forceinline__ double cell_emu(double tc, const double *tn, double ci,
                                           const W<double> &w) {
  unsigned long long nb[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) nb[i] = dbits(tn[i]);
  bool ok;
  double r = cell_emu_fast(tc, nb, ci, w, ok);
  if (ok) return r;
  r = cell_emu_aligned(tc, nb, ci, w, ok);
  if (ok) return r;
  return cell_f64(tc, tn[0], tn[1], tn[2], tn[3], tn[4], tn[5], ci, w);
}

// cell_emu of a point whose fast path is known not to apply (the points a
// kernel left to its fix-up): the aligned path, else cell_f64.
__device__ __forceinline__ double cell_emu_not_fast(double tc, const double *tn, double ci,
                                                    const W<double> &w) {
  if (!w.emu) return cell_f64(tc, tn[0], tn[1], tn[2], tn[3], tn[4], tn[5], ci, w);
  unsigned long long nb[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) nb[i] = dbits(tn[i]);
  bool ok;
  const double r = cell_emu_aligned(tc, nb, ci, w, ok);
  if (ok) return r;
  return cell_f64(tc, tn[0], tn[1], tn[2], tn[3], tn[4], tn[5], ci, w);
}

// The FP64 update used by every kernel: the emulated cell or the FP64 cell.
__device__ __forceinline__ double cell(double t, double xm, double xp, double ym, double yp,
                                       double zm, double zp, double ci, const W<double> &w) {
  if (!w.emu) return cell_f64(t, xm, xp, ym, yp, zm, zp, ci, w);
  const double tn[6] = {xm, xp, ym, yp, zm, zp};
  return cell_emu(t, tn, ci, w);
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
