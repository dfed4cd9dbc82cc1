// Gross-Pitaevskii half steps on the implicit global grid: a complex field
// psi = u + i v kept as two real fields of the grid's layout, u at whole and
// v at half time steps:
//   which 0:  u += dt * H(v),   which 1:  v -= dt * H(u),
//   H w = -1/2 lap(w) + (V + g (u^2 + v^2)) w,
// on inner points (psi fixed on each array's boundary), lap the 7-point
// operator with the grid's spacings. With w the field read and o the field
// written, scaled by dt and the sign s (+1, -1):
//   o += s (kc w + kx (w[-x] + w[+x]) + ky (..) + kz (..) + q w),
//   kd = -dt/(2 dd^2), kc = -2 (kx + ky + kz), q = dt (V + g (u^2 + v^2)).
//
// Per-point arithmetic (shared by both kernels, so they give the same bits):
// FP32 fields in FP32 with FMAs. FP64 fields: q and the seven-term sum in
// float pairs (pair.cuh: error-free products and two-sums, a compensated
// dot product starting from o) and one FP64 add, within about 2^-45 of
// |o| + sum |terms| (the FP64 sum: 13 FP64 instructions per point, which
// bound the step by the FP64 pipe); points whose values leave the pair
// ranges take the FP64 sum.
//
// Kernels: k_gp_tma (3-D grids, rows of a multiple of 16 bytes): the
// persistent TMA column kernel of the adjoint's design (W x 16 tiles, one
// warp per row, equal shares of (z chunk, column, plane) over all
// subdomains, loads issued by thread 0 after each barrier); per plane the w
// box with a one-vector / one-row halo and the o and V boxes; FP64 fields
// form the pairs of w once per point into triple-buffered shared planes.
// k_gp_half: one thread per (x, y) column marching in z (any grid,
// including 2-D and 1-D ones: absent dimensions have zero neighbour strides
// and zero weights).
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "cell.cuh"
#include "igg_internal.h"
#include "pair.cuh"
#include "tma_util.cuh"

namespace igg {
namespace {

// pair ranges: |w|, |o| in [2^-40, 2^41), |q| in [2^-36, 2^37) (or zero),
// weights zero or in [2^-18, 2^18]: no partial product or error term leaves
// the normal FP32 range
constexpr unsigned kGpWE = 40, kGpQE = 36;
static_assert(kGpWE <= kPairMaxRadius && kGpQE <= kPairMaxRadius,
              "pair_ok radii must stay inside pair_split's range");

// weights as pairs, the sign of the half step applied (x, y, z, centre);
// dt and g as pairs
struct GpPairW {
  double k[4];  // s kx, s ky, s kz, s kc (FP64)
  float kh[4], kl[4];
  double dt, g;
  float dth, dtl, gh, gl;
  float s;
  bool pair;
};

__device__ __forceinline__ GpPairW make_gp_w(const GpCoef &c, int which) {
  GpPairW w;
  const double sg = which == 0 ? 1.0 : -1.0;
  const double d[4] = {c.kx, c.ky, c.kz, c.kc};
  bool ok = true;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    w.k[i] = sg * d[i];
    w.kh[i] = __double2float_rn(w.k[i]);
    w.kl[i] = __double2float_rn(__dsub_rn(w.k[i], (double)w.kh[i]));
    // (a zero weight: an absent dimension)
    if (i < 3) ok = ok && (d[i] == 0.0 || (fabs(d[i]) >= 0x1p-18 && fabs(d[i]) <= 0x1p18));
  }
  w.dt = c.dt;
  w.g = c.g;
  w.dth = __double2float_rn(c.dt);
  w.dtl = __double2float_rn(__dsub_rn(c.dt, (double)w.dth));
  w.gh = __double2float_rn(c.g);
  w.gl = __double2float_rn(__dsub_rn(c.g, (double)w.gh));
  w.s = (float)sg;
  // dt and g enter the pair products: dt in [2^-40, 2^20], g zero or in
  // [2^-40, 2^40]
  ok = ok && c.dt >= 0x1p-40 && c.dt <= 0x1p20 &&
       (c.g == 0.0 || (fabs(c.g) >= 0x1p-40 && fabs(c.g) <= 0x1p40));
  w.pair = ok;
  return w;
}

// w as a pair, NaN in h outside the pair range
__device__ __forceinline__ FF gp_pair(double x) {
  FF q = pair_split(x);
  q.h = pair_ok(x, kGpWE) ? q.h : __int_as_float(0x7FC00000);
  return q;
}

// q = dt (V + g (u^2 + v^2)) in FP64 (uc, vc: u and v at the point)
__device__ __forceinline__ double gp_q(double uc, double vc, double pot, const GpPairW &w) {
  return __dmul_rn(w.dt, __fma_rn(w.g, __fma_rn(uc, uc, __dmul_rn(vc, vc)), pot));
}

// q as a normalised pair from the pairs of u and v (NaN in h when a pair
// is, or when the potential lies outside the pair range): error-free
// squares and sum for rho, then g rho + V and dt (..) with FMA product
// splits, about 2^-45 of dt (|V| + |g| rho)
__device__ __forceinline__ FF gp_q_pair(const FF &u, const FF &v, double pot, const GpPairW &w) {
  const float p1 = __fmul_rn(u.h, u.h);
  float e1 = __fmaf_rn(u.h, u.h, -p1);
  e1 = __fmaf_rn(__fadd_rn(u.h, u.h), u.l, e1);
  const float p2 = __fmul_rn(v.h, v.h);
  float e2 = __fmaf_rn(v.h, v.h, -p2);
  e2 = __fmaf_rn(__fadd_rn(v.h, v.h), v.l, e2);
  float t;
  const float rs = pair_two_sum(p1, p2, t);
  t = __fadd_rn(t, __fadd_rn(e1, e2));
  const float a = __fmul_rn(w.gh, rs);
  float ae = __fmaf_rn(w.gh, rs, -a);
  ae = __fmaf_rn(w.gh, t, ae);
  ae = __fmaf_rn(w.gl, rs, ae);
  FF vp = pair_split(pot);
  vp.h = pair_ok(pot, kGpWE) ? vp.h : __int_as_float(0x7FC00000);
  float be;
  const float b = pair_two_sum(a, vp.h, be);
  be = __fadd_rn(be, __fadd_rn(ae, vp.l));
  const float cq = __fmul_rn(w.dth, b);
  float ce = __fmaf_rn(w.dth, b, -cq);
  ce = __fmaf_rn(w.dth, be, ce);
  ce = __fmaf_rn(w.dtl, b, ce);
  FF q;
  q.h = fast_two_sum(cq, ce, q.l);
  return q;
}

// the pair range of q: zero or |q| in [2^-36, 2^37) (from the leading part)
__device__ __forceinline__ bool gp_q_ok(const FF &q) {
  const unsigned b = __float_as_uint(q.h);
  const unsigned e = (b >> 23) & 0xFFu;
  return e - (127u - kGpQE) <= 2u * kGpQE || (b << 1) == 0u;
}

// o + s h on the pair path from the pairs of o (op; o_ok: o in range) and
// q; false: take gp_out_f64
__device__ __forceinline__ bool gp_out_pair(const FF &op, bool o_ok, FF qp, const FF &wc,
                                            const FF &wxm, const FF &wxp, const FF &wym,
                                            const FF &wyp, const FF &wzm, const FF &wzp,
                                            const GpPairW &w, double &res) {
  const bool q_ok = gp_q_ok(qp);
  qp.h *= w.s;
  qp.l *= w.s;
  float acc = op.h, err = op.l;
  dot2_term(acc, err, w.kh[3], w.kl[3], wc.h, wc.l);
  dot2_term(acc, err, qp.h, qp.l, wc.h, wc.l);
  dot2_pair(acc, err, w.kh[0], w.kl[0], wxm, wxp);
  dot2_pair(acc, err, w.kh[1], w.kl[1], wym, wyp);
  dot2_pair(acc, err, w.kh[2], w.kl[2], wzm, wzp);
  res = __dadd_rn(f2d_finite(acc), f2d_finite(err));
  return w.pair && o_ok && q_ok && acc == acc;
}

// o + s h in FP64
__device__ __forceinline__ double gp_out_f64(double o, double q, double wc, double wxm,
                                             double wxp, double wym, double wyp, double wzm,
                                             double wzp, const GpPairW &w) {
  // s is applied through the signed weights: s h = sum of the signed terms
  double h = __dmul_rn(w.k[3], wc);
  h = __fma_rn(w.k[0], __dadd_rn(wxm, wxp), h);
  h = __fma_rn(w.k[1], __dadd_rn(wym, wyp), h);
  h = __fma_rn(w.k[2], __dadd_rn(wzm, wzp), h);
  h = __fma_rn(__dmul_rn((double)w.s, q), wc, h);
  return __dadd_rn(o, h);
}

// o + s h for FP32 fields
__device__ __forceinline__ float gp_out_f32(float o, float uc, float vc, float pot, float wc,
                                            float wxm, float wxp, float wym, float wyp, float wzm,
                                            float wzp, const GpCoef &c, int which) {
  const float kx = (float)c.kx, ky = (float)c.ky, kz = (float)c.kz, kc = (float)c.kc;
  float h = __fmul_rn(kc, wc);
  h = __fmaf_rn(kx, __fadd_rn(wxm, wxp), h);
  h = __fmaf_rn(ky, __fadd_rn(wym, wyp), h);
  h = __fmaf_rn(kz, __fadd_rn(wzm, wzp), h);
  const float q = __fmul_rn((float)c.dt, __fmaf_rn((float)c.g, __fmaf_rn(uc, uc, __fmul_rn(vc, vc)), pot));
  h = __fmaf_rn(q, wc, h);
  return which == 0 ? __fadd_rn(o, h) : __fadd_rn(o, -h);
}

// ---------------------------------------------------------------------------
// tiled kernel (any grid)

constexpr int kGpX = 32, kGpY = 8, kGpZ = 32;

// blockIdx.z = subdomain * zchunks + z chunk; inner ranges [lo, hi) per
// dimension (absent dimensions: [0, 1) with zero stride)
template <class S, int WHICH>
__global__ void __launch_bounds__(kGpX *kGpY)
    k_gp_half(int nx, int ny, int nz, int zchunks, S *__restrict__ u, S *__restrict__ v,
              const S *__restrict__ V, GpCoef c) {
  const int ylo = ny > 1 ? 1 : 0, yhi = ny > 1 ? ny - 1 : 1;
  const int zlo = nz > 1 ? 1 : 0, zhi = nz > 1 ? nz - 1 : 1;
  const int i = 1 + blockIdx.x * kGpX + threadIdx.x, j = ylo + blockIdx.y * kGpY + threadIdx.y;
  // lanes past the last column run along (the FP64 path votes across the
  // warp) and store nothing
  const bool act = i < nx - 1 && j < yhi;
  const long long sub = blockIdx.z / zchunks;
  const int k0 = zlo + (int)(blockIdx.z % zchunks) * kGpZ, k1 = min(k0 + kGpZ, zhi);
  if (k0 >= k1) return;  // uniform over the block
  const int ii = act ? i : 1, jj = act ? j : ylo;
  const long long nloc = (long long)nx * ny * nz;
  const long long sy = ny > 1 ? nx : 0, sz = nz > 1 ? (long long)nx * ny : 0;
  S *out = (WHICH == 0 ? u : v) + sub * nloc;
  const S *w = (WHICH == 0 ? v : u) + sub * nloc;
  const S *Vs = V + sub * nloc;
  long long p = ii + (long long)nx * jj + (long long)nx * ny * k0;
  if constexpr (sizeof(S) == 8) {
    const GpPairW pw = make_gp_w(c, WHICH);
    double wm = w[p - sz], wc = w[p];
    for (int k = k0; k < k1; ++k, p += (long long)nx * ny) {
      const double wp = w[p + sz];
      const double o = out[p], pot = Vs[p];
      const double xm = w[p - 1], xp = w[p + 1], ym = w[p - sy], yp = w[p + sy];
      const FF op = gp_pair(o), cp = gp_pair(wc);
      const FF qp = WHICH == 0 ? gp_q_pair(op, cp, pot, pw) : gp_q_pair(cp, op, pot, pw);
      double r;
      const bool ok = gp_out_pair(op, pair_ok(o, kGpWE), qp, cp, gp_pair(xm), gp_pair(xp),
                                  gp_pair(ym), gp_pair(yp), gp_pair(wm), gp_pair(wp), pw, r);
      if (__any_sync(0xffffffffu, !ok)) {
        if (!ok) {
          const double q = WHICH == 0 ? gp_q(o, wc, pot, pw) : gp_q(wc, o, pot, pw);
          r = gp_out_f64(o, q, wc, xm, xp, ym, yp, wm, wp, pw);
        }
      }
      if (act) out[p] = r;
      wm = wc;
      wc = wp;
    }
  } else {
    S wm = w[p - sz], wc = w[p];
    for (int k = k0; k < k1; ++k, p += (long long)nx * ny) {
      const S wp = w[p + sz];
      const S o = out[p];
      const S uc = WHICH == 0 ? o : wc, vc = WHICH == 0 ? wc : o;
      const S r = gp_out_f32(o, uc, vc, Vs[p], wc, w[p - 1], w[p + 1], w[p - sy], w[p + sy], wm,
                             wp, c, WHICH);
      if (act) out[p] = r;
      wm = wc;
      wc = wp;
    }
  }
}

// ---------------------------------------------------------------------------
// TMA-pipelined kernel (3-D grids)

template <class S>
struct GpShape {
  static constexpr bool PAIRS = sizeof(S) == 8;          // FP64: w as pairs in shared planes
  static constexpr int V = 16 / (int)sizeof(S);          // points per lane
  static constexpr int W = 32 * V;                       // points per row
  static constexpr int BW = W + 2 * V;                   // w box width
  static constexpr int H = 16;                           // rows per tile
  static constexpr int BH = H + 2;
  static constexpr int WARPS = H;
  static constexpr int NS = 6;                           // loads issued NS - 2 ahead
  static constexpr int FB = BW * BH * (int)sizeof(S);    // w box bytes
  static constexpr int FBA = (FB + 127) / 128 * 128;
  static constexpr int OB = W * H * (int)sizeof(S);      // o and V box bytes
  static constexpr int STAGE = FBA + 2 * OB;
  static constexpr int VPL = BW * BH;                    // pair plane elements
  static constexpr int VBA = PAIRS ? (3 * VPL * 8 + 127) / 128 * 128 : 0;
  static constexpr int SMEM = NS * STAGE + VBA + NS * 8 + 16;
  static constexpr int RING = 2 * (W + 2) + 2 * H;
  static constexpr int RPT = (RING + 32 * WARPS - 1) / (32 * WARPS);
  static_assert(OB % 128 == 0, "stage alignment");
  static_assert(BW <= 256 && W <= 256 && BH <= 256, "TMA box dims");
};

template <class S>
__device__ __forceinline__ void gp_lds16(const void *p, Vec<S> &o) {
  unpack(*reinterpret_cast<const uint4 *>(p), o);
}

// mW, mO, mV: tensor maps of the field read (w), the field written (o) and
// the potential over [nsub * nz][ny][nx]; ncxy columns per subdomain
template <class S, int WHICH>
__global__ void __launch_bounds__(32 * GpShape<S>::WARPS, 1)
    k_gp_tma(const __grid_constant__ CUtensorMap mW, const __grid_constant__ CUtensorMap mO,
             const __grid_constant__ CUtensorMap mV, int nx, int ny, int nz, int ncx, int ncxy,
             int ncol, S *__restrict__ out, GpCoef c, unsigned *__restrict__ dev_err) {
  using Sh = GpShape<S>;
  constexpr int V = Sh::V, W = Sh::W, BW = Sh::BW, H = Sh::H, NS = Sh::NS;
  constexpr unsigned NT = 32 * Sh::WARPS;
  extern __shared__ __align__(128) unsigned char smem[];
  const unsigned sbase = smem_u32(smem);
  FF *planes = reinterpret_cast<FF *>(smem + NS * Sh::STAGE);
  const unsigned full0 = sbase + NS * Sh::STAGE + Sh::VBA;
  volatile int *flags = reinterpret_cast<volatile int *>(smem + NS * Sh::STAGE + Sh::VBA + NS * 8);

  const int nzi = nz - 2;  // inner planes per column (z = m + 1)
  const long long U = (long long)ncol * nzi;
  const long long u0 = U * blockIdx.x / gridDim.x, u1 = U * (blockIdx.x + 1) / gridDim.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto origin = [&](int col, int &x0, int &r0, int &zoff) {
    const int sub = col / ncxy, cc = col - sub * ncxy;
    x0 = (cc % ncx) * W;
    r0 = (cc / ncx) * H;
    zoff = sub * nz;
  };

  // load cursor (thread 0): a segment's loads are its planes z0 - 1 .. z1
  Share cur{u0, u1, nzi, ncol};
  Seg cs{0, 0, 0};
  int cj = 0, cK = 0, issued = 0;
  auto issue_upto = [&](int last) {
    while (issued <= last) {
      if (cj >= cK) {
        if (!cur.next(cs)) return;
        cj = 0;
        cK = cs.m1 - cs.m0 + 2;
      }
      int x0, r0, zoff;
      origin(cs.col, x0, r0, zoff);
      const int s = issued % NS;
      const bool ov = cj >= 1 && cj <= cK - 2;  // o and V of the computed planes
      const unsigned bar = full0 + 8 * s, dst = sbase + s * Sh::STAGE;
      mbar_expect_tx(bar, Sh::FB + (ov ? 2 * Sh::OB : 0));
      const int p = zoff + cs.m0 + cj;  // plane z = m0 + 1 - 1 + cj
      tma_load_3d(dst, &mW, x0 - V, r0 - 1, p, bar);
      if (ov) {
        tma_load_3d(dst + Sh::FBA, &mO, x0, r0, p, bar);
        tma_load_3d(dst + Sh::FBA + Sh::OB, &mV, x0, r0, p, bar);
      }
      ++cj;
      ++issued;
    }
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(full0 + 8 * s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    issue_upto(NS - 2);
  }
  __syncthreads();

  const GpPairW pw = make_gp_w(c, WHICH);
  const int r = warp;
  const int ob = (r + 1) * BW + V + lane * V;  // own points in the w box / pair plane
  const int oo = r * W + lane * V;             // own points in the o and V boxes
  const long long sz = (long long)nx * ny;
  auto stage = [&](int kk) { return smem + (kk % NS) * Sh::STAGE; };
  auto wbox = [&](int kk) { return reinterpret_cast<const S *>(stage(kk)); };
  auto wait_full = [&](int kk) {
    return __all_sync(0xffffffffu, mbar_wait(full0 + 8 * (kk % NS), (kk / NS) & 1));
  };

  Share sh{u0, u1, nzi, ncol};
  Seg sg;
  int k = 0, q = 0;
  bool stop = false;
  // own w of planes z-1, z, z+1 (FP64: also as pairs)
  S tm[V], tc[V], tp[V];
  FF pm[V], pc[V], pp[V];
  while (!stop && sh.next(sg)) {
    int x0, r0, zoff;
    origin(sg.col, x0, r0, zoff);
    const int xs = x0 + lane * V, y = r0 + r;
    const bool yin = y >= 1 && y <= ny - 2;
    bool xyin[V];
#pragma unroll
    for (int i = 0; i < V; ++i) xyin[i] = yin && xs + i >= 1 && xs + i <= nx - 2;
    // the halo update's x exchange (GpCoef::xsend): this lane's points of the
    // sent planes nx - o (bits 0..V-1: to the right neighbour's column 0) and
    // o - 1 (bits 8..8+V-1: to the left neighbour's column nx - 1), and the
    // element offsets of their copies
    unsigned sendm = 0u;
    long long dr = 0, dl = 0;
    if (c.xsend) {
      const int sub = zoff / nz, xl = c.nbr[6 * sub], xr = c.nbr[6 * sub + 1];
      const long long nloc = sz * nz, h = nx - c.ox;
      dr = (long long)(xr - sub) * nloc - h;
      dl = (long long)(xl - sub) * nloc + h;
#pragma unroll
      for (int i = 0; i < V; ++i) {
        if (!xyin[i]) continue;
        if (xr >= 0 && xs + i == nx - c.ox) sendm |= 1u << i;
        if (xl >= 0 && xs + i == c.ox - 1) sendm |= 1u << (8 + i);
      }
    }
    int rb[Sh::RPT];
#pragma unroll
    for (int j = 0; j < Sh::RPT; ++j) {
      const int i = threadIdx.x + j * NT;
      int xo = 0, yo = -1;
      if (i < 2 * (W + 2)) {
        xo = i % (W + 2) - 1;
        yo = i < W + 2 ? -1 : H;
      } else {
        const int t = i - 2 * (W + 2);
        xo = t < H ? -1 : W;
        yo = t % H;
      }
      rb[j] = i < Sh::RING ? (yo + 1) * BW + xo + V : -1;
    }
    // own w of load kk (and, FP64, its pairs)
    auto own = [&](int kk, S *t, FF *pr) {
      Vec<S> a;
      gp_lds16<S>(wbox(kk) + ob, a);
#pragma unroll
      for (int i = 0; i < V; ++i) {
        t[i] = a.v[i];
        if constexpr (Sh::PAIRS) pr[i] = gp_pair(a.v[i]);
      }
    };
    // FP64: the pair plane of load kk (own pairs, then the ring)
    auto form = [&](int kk, FF *pl, const FF *pr) {
      if constexpr (Sh::PAIRS) {
        uint4 w4;
        memcpy(&w4, pr, 16);
        *reinterpret_cast<uint4 *>(pl + ob) = w4;
        const S *Wb = wbox(kk);
#pragma unroll
        for (int j = 0; j < Sh::RPT; ++j)
          if (rb[j] >= 0) pl[rb[j]] = gp_pair(Wb[rb[j]]);
      }
    };
    bool good = wait_full(k);
    if (good) {
      own(k, tm, pm);
      ++k;
      good = wait_full(k);
    }
    FF *pl = planes + (q % 3) * Sh::VPL;
    if (good) {
      own(k, tc, pc);
      form(k, pl, pc);
    }
    if (all_any(!good, NT)) {
      stop = true;
      break;
    }
    if (threadIdx.x == 0) issue_upto(k + NS - 2);
    int kc = k;
    ++k;
    const FF *plm = pl;
    ++q;
    for (int m = sg.m0; m < sg.m1; ++m) {
      const int z = m + 1;
      good = wait_full(k);
      FF *pln = planes + (q % 3) * Sh::VPL;
      if (good) {
        own(k, tp, pp);
        form(k, pln, pp);
      }
      if (all_any(!good, NT)) {
        stop = true;
        break;
      }
      if (threadIdx.x == 0) issue_upto(k + NS - 2);
      // plane z
      const S *Wb = wbox(kc);
      const S *Ob = reinterpret_cast<const S *>(stage(kc) + Sh::FBA) + oo;
      const S *Pb = reinterpret_cast<const S *>(stage(kc) + Sh::FBA + Sh::OB) + oo;
      Vec<S> ov, pv, wym, wyp;
      gp_lds16<S>(Ob, ov);
      gp_lds16<S>(Pb, pv);
      gp_lds16<S>(Wb + ob - BW, wym);
      gp_lds16<S>(Wb + ob + BW, wyp);
      const S wl = Wb[ob - 1], wr = Wb[ob + V];
      S res[V];
      if constexpr (Sh::PAIRS) {
        const FF fl = plm[ob - 1], fr = plm[ob + V];
        bool bad = false;
#pragma unroll
        for (int i = 0; i < V; ++i) {
          const FF op = gp_pair(ov.v[i]);
          const FF qp = WHICH == 0 ? gp_q_pair(op, pc[i], pv.v[i], pw)
                                   : gp_q_pair(pc[i], op, pv.v[i], pw);
          const FF xm = i == 0 ? fl : pc[i - 1];
          const FF xp = i == V - 1 ? fr : pc[i + 1];
          const bool ok = gp_out_pair(op, pair_ok(ov.v[i], kGpWE), qp, pc[i], xm, xp,
                                      plm[ob - BW + i], plm[ob + BW + i], pm[i], pp[i], pw,
                                      res[i]);
          bad = bad || (!ok && xyin[i]);
          if (!ok) res[i] = __longlong_as_double(0x7FF8000000000000ll);  // marks the point
        }
        if (__any_sync(0xffffffffu, bad)) {
#pragma unroll
          for (int i = 0; i < V; ++i) {
            if (res[i] != res[i]) {
              const double xm = i == 0 ? wl : tc[i - 1];
              const double xp = i == V - 1 ? wr : tc[i + 1];
              const double q = WHICH == 0 ? gp_q(ov.v[i], tc[i], pv.v[i], pw)
                                          : gp_q(tc[i], ov.v[i], pv.v[i], pw);
              res[i] = gp_out_f64(ov.v[i], q, tc[i], xm, xp, wym.v[i], wyp.v[i], tm[i], tp[i], pw);
            }
          }
        }
      } else {
#pragma unroll
        for (int i = 0; i < V; ++i) {
          const S xm = i == 0 ? wl : tc[i - 1];
          const S xp = i == V - 1 ? wr : tc[i + 1];
          const S uc = WHICH == 0 ? ov.v[i] : tc[i], vc = WHICH == 0 ? tc[i] : ov.v[i];
          res[i] = gp_out_f32(ov.v[i], uc, vc, pv.v[i], tc[i], xm, xp, wym.v[i], wyp.v[i], tm[i],
                              tp[i], c, WHICH);
        }
      }
      const long long p0 = zoff * sz + xs + (long long)nx * y + sz * z;
      bool all_in = true;
#pragma unroll
      for (int i = 0; i < V; ++i) all_in = all_in && xyin[i];
      if (all_in) {
        Vec<S> o;
#pragma unroll
        for (int i = 0; i < V; ++i) o.v[i] = res[i];
        *reinterpret_cast<uint4 *>(out + p0) = pack(o);
      } else {
#pragma unroll
        for (int i = 0; i < V; ++i)
          if (xyin[i]) out[p0 + i] = res[i];
      }
      if (sendm) {
        // the sent points stored again into the neighbours' halo columns
        // (the halo launch then copies the face rows only)
#pragma unroll
        for (int i = 0; i < V; ++i) {
          if (sendm >> i & 1u) out[p0 + i + dr] = res[i];
          if (sendm >> (8 + i) & 1u) out[p0 + i + dl] = res[i];
        }
      }
      kc = k;
      ++k;
      plm = pln;
      ++q;
#pragma unroll
      for (int i = 0; i < V; ++i) {
        tm[i] = tc[i];
        tc[i] = tp[i];
        pm[i] = pc[i];
        pc[i] = pp[i];
      }
    }
  }
  if (threadIdx.x == 0) flags[0] = issued;
  __syncthreads();
  if (threadIdx.x == 0 && stop) {
    atomicOr(dev_err, IGG_DEV_ERR_TIMEOUT);
    for (int kk = k; kk < flags[0]; ++kk) {
      if (!mbar_wait(full0 + 8 * (kk % NS), (kk / NS) & 1)) {
        atomicOr(dev_err, IGG_DEV_ERR_DRAIN);
        break;
      }
    }
  }
}

template <class S, int WHICH>
cudaError_t launch_tma(int nsub, int nx, int ny, int nz, void *u, void *v, const void *V,
                       const GpCoef &c, unsigned *dev_err, cudaStream_t s) {
  using Sh = GpShape<S>;
  static cudaError_t attr = cudaErrorNotReady;
  static std::mutex mu;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (attr == cudaErrorNotReady)
      attr = cudaFuncSetAttribute(k_gp_tma<S, WHICH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  Sh::SMEM);
  }
  if (attr != cudaSuccess) return attr;
  void *o = WHICH == 0 ? u : v;
  const void *w = WHICH == 0 ? v : u;
  const long long nzt = (long long)nsub * nz;
  CUtensorMap mW, mO, mV;
  if (!encode<S>(&mW, w, nx, ny, nzt, Sh::BW, Sh::BH, 1) ||
      !encode<S>(&mO, o, nx, ny, nzt, Sh::W, Sh::H, 1) ||
      !encode<S>(&mV, V, nx, ny, nzt, Sh::W, Sh::H, 1))
    return cudaErrorInvalidValue;
  int per_sm = 0, dev = 0, sms = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gp_tma<S, WHICH>,
                                                                32 * Sh::WARPS, Sh::SMEM);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int ncx = (nx + Sh::W - 1) / Sh::W, ncy = (ny + Sh::H - 1) / Sh::H;
  const long long ncol = (long long)nsub * ncx * ncy;
  if (ncol > (1ll << 30)) return cudaErrorInvalidValue;
  const long long U = ncol * (nz - 2);
  const long long G = std::min<long long>((long long)per_sm * sms, std::max<long long>(1, U / 4));
  k_gp_tma<S, WHICH><<<(unsigned)G, 32 * Sh::WARPS, Sh::SMEM, s>>>(
      mW, mO, mV, nx, ny, nz, ncx, ncx * ncy, (int)ncol, (S *)o, c, dev_err);
  return cudaGetLastError();
}

template <class S, int WHICH>
cudaError_t launch_w(int nsub, int nx, int ny, int nz, void *u, void *v, const void *V,
                     const GpCoef &c, cudaStream_t s) {
  const int ny_in = ny > 1 ? ny - 2 : 1, nz_in = nz > 1 ? nz - 2 : 1;
  const int zchunks = (nz_in + kGpZ - 1) / kGpZ;
  const long long gz = (long long)nsub * zchunks;
  if (gz > 65535 || nx < 3) return cudaErrorInvalidValue;
  const dim3 grid((nx - 2 + kGpX - 1) / kGpX, (ny_in + kGpY - 1) / kGpY, (unsigned)gz);
  k_gp_half<S, WHICH><<<grid, dim3(kGpX, kGpY), 0, s>>>(nx, ny, nz, zchunks, (S *)u, (S *)v,
                                                       (const S *)V, c);
  return cudaGetLastError();
}

template <class S>
bool tma_fits(int nx, int ny, int nz, const void *u, const void *v, const void *V) {
  if (!tma_available() || ny < 3 || nz < 3 || nx < 3) return false;
  if (((size_t)nx * sizeof(S)) % 16 != 0) return false;
  for (const void *p : {u, v, V})
    if (reinterpret_cast<uintptr_t>(p) % 16 != 0) return false;
  return true;
}

}  // namespace

cudaError_t launch_gp_half(igg_dtype dt, int which, int nsub, int nx, int ny, int nz, void *u,
                           void *v, const void *V, const GpCoef &c, bool tma, unsigned *dev_err,
                           cudaStream_t s, bool *xsent) {
  *xsent = false;
  GpCoef cw = c;  // the tiled kernel does no x sends
  cw.xsend = 0;
  switch (dt) {
    case IGG_F64:
      if (tma && tma_fits<double>(nx, ny, nz, u, v, V)) {
        *xsent = c.xsend != 0;
        return which == 0 ? launch_tma<double, 0>(nsub, nx, ny, nz, u, v, V, c, dev_err, s)
                          : launch_tma<double, 1>(nsub, nx, ny, nz, u, v, V, c, dev_err, s);
      }
      return which == 0 ? launch_w<double, 0>(nsub, nx, ny, nz, u, v, V, cw, s)
                        : launch_w<double, 1>(nsub, nx, ny, nz, u, v, V, cw, s);
    case IGG_F32:
      if (tma && tma_fits<float>(nx, ny, nz, u, v, V)) {
        *xsent = c.xsend != 0;
        return which == 0 ? launch_tma<float, 0>(nsub, nx, ny, nz, u, v, V, c, dev_err, s)
                          : launch_tma<float, 1>(nsub, nx, ny, nz, u, v, V, c, dev_err, s);
      }
      return which == 0 ? launch_w<float, 0>(nsub, nx, ny, nz, u, v, V, cw, s)
                        : launch_w<float, 1>(nsub, nx, ny, nz, u, v, V, cw, s);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace igg
