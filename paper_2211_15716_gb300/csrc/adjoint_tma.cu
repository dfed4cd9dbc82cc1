// TMA-pipelined adjoint step over every point of one array (the transposed
// stencil of Fig. 1's step! and the Ci-gradient increment; arithmetic in
// adj_cell.cuh, the same bits as the tiled kernel of adjoint.cu).
//
// Tiles are W x H (x, y) columns (W = 32 lanes x one 16-byte vector: 64
// FP64 or 128 FP32 points; H = 8 FP64 / 16 FP32 rows, one warp per row)
// marching along z. A persistent grid (all CTAs resident) takes equal shares
// of the work order (z chunk, column, plane), so every CTA handles the same
// number of planes; a share splits into segments (runs of planes of one
// column).
//
// Per plane p, cp.async.bulk.tensor (TMA) loads into a ring of NS shared-
// memory stages the (W + 2V) x (H + 2) boxes of lam_in, Ci and T_n around the
// tile (a vector / one row of halo, zero outside the array) and the W x H box
// of gCi. The warps, for plane m + 1 as soon as it lands: form v = Ci * lam_in
// of the tile and its ring once (triple-buffered v planes in shared memory);
// then, after one barrier of all warps, plane m: lam_out from the v planes
// (neighbours in x, y from shared memory, z from registers) and
// gCi += lam_in * l(T_n) from the T_n box, with 16-byte stores.
//
// No producer warp: thread 0 issues the loads right after each barrier. At
// the barrier that follows the forming of load k, every warp has finished
// with load k - 2 (the plane computed in the previous step), so loads up to
// k + NS - 2 can go into their stages; two loads stay in flight while the
// CTA computes. Every wait on a load is bounded (about 2 s); the warps agree
// on stopping through the reduction of their barrier (bar.red.or), so that
// none is left at a barrier; a stopped CTA records IGG_DEV_ERR_TIMEOUT, waits
// (bounded) for the loads it issued and returns.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "adj_cell.cuh"
#include "igg_internal.h"
#include "tma_util.cuh"

namespace igg {
namespace {

template <class S>
struct AdjShape {
  using VT = typename AdjOps<S>::VT;
  static constexpr int V = 16 / (int)sizeof(S);          // points per lane
  static constexpr int W = 32 * V;                       // points per row
  static constexpr int BW = W + 2 * V;                   // box width
  // rows per tile: FP64 8 (two CTAs per SM: measured 8 % faster than one
  // CTA with 16 rows), FP32 16 (one CTA per SM)
  static constexpr int H = sizeof(S) == 8 ? 8 : 16;
  static constexpr int BH = H + 2;                       // box height
  static constexpr int WARPS = H;                        // one warp per row
  static constexpr int MINB = H == 8 ? 2 : 1;            // resident CTAs per SM
  // stages: a segment's first two loads must both be in flight before its
  // first barrier, so loads are issued up to two ahead of the last formed
  static constexpr int NS = 4;
  static constexpr int FB = BW * BH * (int)sizeof(S);    // field box bytes
  static constexpr int FBA = (FB + 127) / 128 * 128;
  static constexpr int GB = W * H * 8;                   // gCi box bytes
  static constexpr int STAGE = 3 * FBA + GB;
  static constexpr int VPL = BW * BH;                    // v plane elements
  static constexpr int VBA = (3 * VPL * (int)sizeof(VT) + 127) / 128 * 128;
  static constexpr int SMEM = NS * STAGE + VBA + NS * 8 + 16;
  static constexpr int RING = 2 * (W + 2) + 2 * H;       // ring points of a tile
  static constexpr int RPT = (RING + 32 * WARPS - 1) / (32 * WARPS);  // ring points per thread
  static_assert(GB % 128 == 0, "stage alignment");
  static_assert(BW <= 256 && W <= 256 && BH <= 256, "TMA box dims");
  static_assert(H == 8 || H == 16, "tile rows");
  static_assert(NS >= 4, "issue rule needs two loads ahead");
};

template <class S>
__device__ __forceinline__ void lds16(const void *p, Vec<S> &o) {
  unpack(*reinterpret_cast<const uint4 *>(p), o);
}

// CIP (FP64 fields): the Ci box holds Ci as pairs (pair_ci, formed once per
// run by k_pair_ci) instead of the FP64 values; the FP64 sum then reads Ci
// from memory.
template <class S, bool CIP>
__global__ void __launch_bounds__(32 * AdjShape<S>::WARPS, AdjShape<S>::MINB)
    k_adjoint_tma(const __grid_constant__ CUtensorMap mL, const __grid_constant__ CUtensorMap mC,
                  const __grid_constant__ CUtensorMap mT, const __grid_constant__ CUtensorMap mG,
                  int nx, int ny, int nz, int ncx, int ncol, S *__restrict__ lam_out,
                  const S *__restrict__ lam_in, const S *__restrict__ Ci,
                  double *__restrict__ gCi, Coef c, unsigned *__restrict__ dev_err) {
  using Sh = AdjShape<S>;
  using Ops = AdjOps<S>;
  using VT = typename Sh::VT;
  using LT = typename Ops::LT;
  constexpr int V = Sh::V, W = Sh::W, BW = Sh::BW, H = Sh::H, NS = Sh::NS;
  constexpr unsigned NT = 32 * Sh::WARPS;
  extern __shared__ __align__(128) unsigned char smem[];
  const unsigned sbase = smem_u32(smem);
  VT *vbuf = reinterpret_cast<VT *>(smem + NS * Sh::STAGE);
  const unsigned full0 = sbase + NS * Sh::STAGE + Sh::VBA;
  volatile int *flags = reinterpret_cast<volatile int *>(smem + NS * Sh::STAGE + Sh::VBA + NS * 8);
  // flags[0]: loads issued

  const long long U = (long long)ncol * nz;
  const long long u0 = U * blockIdx.x / gridDim.x, u1 = U * (blockIdx.x + 1) / gridDim.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // the load cursor (used by thread 0 only): the loads of a segment are its
  // planes m0 - 1 .. m1
  Share cur{u0, u1, nz, ncol};
  Seg cs{0, 0, 0};
  int cj = 0, cK = 0, issued = 0;
  auto issue_upto = [&](int last) {
    while (issued <= last) {
      if (cj >= cK) {
        if (!cur.next(cs)) return;
        cj = 0;
        cK = cs.m1 - cs.m0 + 2;
      }
      const int s = issued % NS;
      const int x0 = (cs.col % ncx) * W, r0 = (cs.col / ncx) * H;
      const bool g = cj >= 1 && cj <= cK - 2;  // gCi of planes m0 .. m1-1
      const unsigned bar = full0 + 8 * s, dst = sbase + s * Sh::STAGE;
      mbar_expect_tx(bar, 3 * Sh::FB + (g ? Sh::GB : 0));
      const int p = cs.m0 - 1 + cj;
      tma_load_3d(dst, &mL, x0 - V, r0 - 1, p, bar);
      tma_load_3d(dst + Sh::FBA, &mC, x0 - V, r0 - 1, p, bar);
      tma_load_3d(dst + 2 * Sh::FBA, &mT, x0 - V, r0 - 1, p, bar);
      if (g) tma_load_3d(dst + 3 * Sh::FBA, &mG, x0, r0, p, bar);
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

  const typename Ops::WT aw = Ops::weights(c);
  const int r = warp;                          // tile row of this warp
  const int ob = (r + 1) * BW + V + lane * V;  // own points in a box / v plane
  const long long sz = (long long)nx * ny;
  auto stage = [&](int kk) { return smem + (kk % NS) * Sh::STAGE; };
  auto box = [&](int kk, int f) {
    return reinterpret_cast<const S *>(stage(kk) + f * Sh::FBA);
  };
  auto wait_full = [&](int kk) {
    return __all_sync(0xffffffffu, mbar_wait(full0 + 8 * (kk % NS), (kk / NS) & 1));
  };
  auto zin = [&](int p) { return p >= 1 && p <= nz - 2; };

  Share sh{u0, u1, nz, ncol};
  Seg sg;
  int k = 0, q = 0;  // loads waited for, v planes formed
  bool stop = false;
  // own values of planes m-1, m, m+1: lam (m, m+1: value and the sum's
  // start), T, v
  S lc[V], lp[V], tm[V], tc[V], tp[V];
  LT qc[V], qp[V];
  VT vm[V], vc[V], vp[V];
  while (!stop && sh.next(sg)) {
    const int x0 = (sg.col % ncx) * W, r0 = (sg.col / ncx) * H;
    const int xs = x0 + lane * V, y = r0 + r;
    const bool yin = y >= 1 && y <= ny - 2, yown = y < ny;
    bool xyin[V];
#pragma unroll
    for (int i = 0; i < V; ++i) xyin[i] = yin && xs + i >= 1 && xs + i <= nx - 2;
    // this thread's ring points: box index and whether (x, y) is inner
    int rb[Sh::RPT];
    bool rxy[Sh::RPT];
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
      const int xx = x0 + xo, yy = r0 + yo;
      rxy[j] = xx >= 1 && xx <= nx - 2 && yy >= 1 && yy <= ny - 2;
    }
    // own values of plane p from load kk
    auto own = [&](int kk, int p, S *l, LT *lq, S *t, VT *v) {
      Vec<S> a, b, d;
      lds16<S>(box(kk, 0) + ob, a);
      lds16<S>(box(kk, 1) + ob, b);
      lds16<S>(box(kk, 2) + ob, d);
      const bool zi = zin(p);
#pragma unroll
      for (int i = 0; i < V; ++i) {
        const LT qq = Ops::lam(a.v[i]);
        if (l) l[i] = a.v[i];
        if (lq) lq[i] = qq;
        t[i] = d.v[i];
        if constexpr (CIP) {
          FF cp;
          memcpy(&cp, &b.v[i], 8);
          v[i] = adj_v_pairs(qq, cp, xyin[i] && zi);
        } else {
          v[i] = Ops::v(qq, b.v[i], xyin[i] && zi);
        }
      }
    };
    // the v plane of plane p from load kk: own values v, the ring from the boxes
    auto form = [&](int kk, int p, VT *vb, const VT *v) {
      uint4 w4;
      static_assert(sizeof(VT) * V == 16, "one 16-byte vector of v per lane");
      memcpy(&w4, v, 16);
      *reinterpret_cast<uint4 *>(vb + ob) = w4;
      const S *L = box(kk, 0), *C = box(kk, 1);
      const bool zi = zin(p);
#pragma unroll
      for (int j = 0; j < Sh::RPT; ++j) {
        if (rb[j] < 0) continue;
        if constexpr (CIP) {
          vb[rb[j]] = adj_v_pairs(Ops::lam(L[rb[j]]), reinterpret_cast<const FF *>(C)[rb[j]],
                                  rxy[j] && zi);
        } else {
          vb[rb[j]] = Ops::v(Ops::lam(L[rb[j]]), C[rb[j]], rxy[j] && zi);
        }
      }
    };
    // load of plane m0 - 1 (own values), then of plane m0 (own values, v plane)
    bool good = wait_full(k);
    if (good) {
      own(k, sg.m0 - 1, nullptr, nullptr, tm, vm);
      ++k;
      good = wait_full(k);
    }
    VT *vb = vbuf + (q % 3) * Sh::VPL;
    if (good) {
      own(k, sg.m0, lc, qc, tc, vc);
      form(k, sg.m0, vb, vc);
    }
    // the barrier also orders this segment's v planes after the previous
    // segment's last reads
    if (all_any(!good, NT)) {
      stop = true;
      break;
    }
    if (threadIdx.x == 0) issue_upto(k + NS - 2);
    int kc = k;  // load of plane m
    ++k;
    const VT *vbm = vb;
    ++q;
    for (int m = sg.m0; m < sg.m1; ++m) {
      // plane m + 1: own values and v plane
      good = wait_full(k);
      VT *vbn = vbuf + (q % 3) * Sh::VPL;
      if (good) {
        own(k, m + 1, lp, qp, tp, vp);
        form(k, m + 1, vbn, vp);
      }
      if (all_any(!good, NT)) {
        stop = true;
        break;
      }
      if (threadIdx.x == 0) issue_upto(k + NS - 2);
      // plane m
      const S *L = box(kc, 0), *C = box(kc, 1), *T = box(kc, 2);
      const double *G =
          reinterpret_cast<const double *>(stage(kc) + 3 * Sh::FBA) + r * W + lane * V;
      const VT vl = vbm[ob - 1], vr = vbm[ob + V];
      S out[V];
      bool okp[V];
      bool any_bad = false;
#pragma unroll
      for (int i = 0; i < V; ++i) {
        const VT xm = i == 0 ? vl : vc[i - 1];
        const VT xp = i == V - 1 ? vr : vc[i + 1];
        okp[i] = Ops::out(qc[i], vc[i], xm, xp, vbm[ob - BW + i], vbm[ob + BW + i], vm[i], vp[i],
                          aw, out[i]);
        any_bad = any_bad || !okp[i];
      }
      if constexpr (sizeof(S) == 8) {
        // points outside the pair path's ranges: the FP64 sum, its v from
        // the boxes of planes m and m + 1 and, for plane m - 1, from memory
        if (__any_sync(0xffffffffu, any_bad && yown)) {
          const S *Ln = box(k, 0), *Cn = box(k, 1);  // plane m + 1 (load k)
#pragma unroll
          for (int i = 0; i < V; ++i) {
            const int x = xs + i;
            if (!okp[i] && x < nx && yown) {
              const int b = ob + i;
              auto in3 = [&](int xx, int yy, int zz) {
                return xx >= 1 && xx <= nx - 2 && yy >= 1 && yy <= ny - 2 && zz >= 1 &&
                       zz <= nz - 2;
              };
              // Ci of an inner point: from the box, or (pairs in the box)
              // from memory
              auto ci_at = [&](const S *Cb, int bb, int xx, int yy, int zz) -> double {
                if constexpr (CIP) return Ci[xx + (long long)nx * yy + sz * zz];
                else return Cb[bb];
              };
              auto v64 = [&](int bb, int xx, int yy) {
                const bool in = in3(xx, yy, m);
                return in ? adj_v64(L[bb], ci_at(C, bb, xx, yy, m), true) : 0.0;
              };
              const bool inm = in3(x, y, m - 1), inp = in3(x, y, m + 1);
              const long long pm = x + (long long)nx * y + sz * (m - 1);
              out[i] = adj_out_f64(lc[i], v64(b, x, y), v64(b - 1, x - 1, y), v64(b + 1, x + 1, y),
                                   v64(b - BW, x, y - 1), v64(b + BW, x, y + 1),
                                   adj_v64(inm ? lam_in[pm] : 0.0, inm ? Ci[pm] : 0.0, inm),
                                   inp ? adj_v64(Ln[b], ci_at(Cn, b, x, y, m + 1), true) : 0.0,
                                   aw.w);
            }
          }
        }
      }
      const long long p0 = xs + (long long)nx * y + sz * m;
      if (yown) {
        if (xs + V <= nx) {
          Vec<S> o;
#pragma unroll
          for (int i = 0; i < V; ++i) o.v[i] = out[i];
          *reinterpret_cast<uint4 *>(lam_out + p0) = pack(o);
        } else {
#pragma unroll
          for (int i = 0; i < V; ++i)
            if (xs + i < nx) lam_out[p0 + i] = out[i];
        }
      }
      // gCi += lam_in * l(T_n) on the inner points of plane m
      Vec<S> tym, typ;
      lds16<S>(T + ob - BW, tym);
      lds16<S>(T + ob + BW, typ);
      const S tl = T[ob - 1], tr = T[ob + V];
      const bool zi = zin(m);
      double gn[V];
      bool all_in = true;
#pragma unroll
      for (int i = 0; i < V; ++i) {
        const bool inn = xyin[i] && zi;
        all_in = all_in && inn;
        const S xm = i == 0 ? tl : tc[i - 1];
        const S xp = i == V - 1 ? tr : tc[i + 1];
        gn[i] = gci_add(G[i], inn, lc[i], tc[i], xm, xp, tym.v[i], typ.v[i], tm[i], tp[i],
                        Ops::lapw(aw));
      }
      double *gd = gCi + p0;
      if (all_in) {
#pragma unroll
        for (int i = 0; i < V; i += 2)
          *reinterpret_cast<double2 *>(gd + i) = make_double2(gn[i], gn[i + 1]);
      } else {
#pragma unroll
        for (int i = 0; i < V; ++i)
          if (xyin[i] && zi) gd[i] = gn[i];
      }
      kc = k;
      ++k;
      vbm = vbn;
      ++q;
#pragma unroll
      for (int i = 0; i < V; ++i) {
        lc[i] = lp[i];
        qc[i] = qp[i];
        tm[i] = tc[i];
        tc[i] = tp[i];
        vm[i] = vc[i];
        vc[i] = vp[i];
      }
    }
  }
  if (threadIdx.x == 0) flags[0] = issued;
  __syncthreads();
  // After a stop, wait (bounded) for loads issued but never waited for, so
  // that no bulk copy writes into this CTA's shared memory after it exits.
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

template <class S, bool CIP>
cudaError_t prepare_adj_t(int *ctas_per_sm) {
  using Sh = AdjShape<S>;
  static cudaError_t done = cudaErrorNotReady;
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  if (done == cudaErrorNotReady)
    done = cudaFuncSetAttribute(k_adjoint_tma<S, CIP>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, Sh::SMEM);
  if (done != cudaSuccess) return done;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k_adjoint_tma<S, CIP>,
                                                       32 * Sh::WARPS, Sh::SMEM);
}

template <class S, bool CIP>
cudaError_t launch_adj_t(int nx, int ny, int nz, void *lam_out, const void *lam_in, const void *Tn,
                         const void *Ci, const void *ci_box, double *gCi, const Coef &c,
                         unsigned *dev_err, cudaStream_t s) {
  using Sh = AdjShape<S>;
  CUtensorMap mL, mC, mT, mG;
  // the Ci box: FP64 values, or their pairs (8 bytes each, the same box)
  if (!encode<S>(&mL, lam_in, nx, ny, nz, Sh::BW, Sh::BH, 1) ||
      !encode<S>(&mC, ci_box, nx, ny, nz, Sh::BW, Sh::BH, 1) ||
      !encode<S>(&mT, Tn, nx, ny, nz, Sh::BW, Sh::BH, 1) ||
      !encode<double>(&mG, gCi, nx, ny, nz, Sh::W, Sh::H, 1))
    return cudaErrorInvalidValue;
  int per_sm = 0, dev = 0, sms = 0;
  cudaError_t e = prepare_adj_t<S, CIP>(&per_sm);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int ncx = (nx + Sh::W - 1) / Sh::W, ncy = (ny + Sh::H - 1) / Sh::H;
  const long long U = (long long)ncx * ncy * nz;
  // every CTA gets at least a few planes; at most the resident CTAs
  const long long G = std::min<long long>((long long)per_sm * sms, std::max<long long>(1, U / 4));
  k_adjoint_tma<S, CIP><<<(unsigned)G, 32 * Sh::WARPS, Sh::SMEM, s>>>(
      mL, mC, mT, mG, nx, ny, nz, ncx, ncx * ncy, (S *)lam_out, (const S *)lam_in,
      (const S *)Ci, gCi, c, dev_err);
  return cudaGetLastError();
}

// Ci as pairs (pair_ci), once per checkpointed run
__global__ void __launch_bounds__(256) k_pair_ci(const double *__restrict__ Ci, FF *__restrict__ out,
                                                 long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = pair_ci(__ldg(Ci + i));
}

}  // namespace

bool adjoint_tma_applies(igg_dtype dt, int nx, const void *lam_out, const void *lam_in,
                         const void *Tn, const void *Ci, const double *gCi) {
  if (!tma_available()) return false;
  size_t es = 0;
  if (dt == IGG_F64) es = 8;
  else if (dt == IGG_F32) es = 4;
  else return false;
  if (((size_t)nx * es) % 16 != 0) return false;
  for (const void *p : {lam_out, lam_in, Tn, Ci, (const void *)gCi})
    if (reinterpret_cast<uintptr_t>(p) % 16 != 0) return false;
  return true;
}

cudaError_t launch_adjoint_tma(igg_dtype dt, int nx, int ny, int nz, void *lam_out,
                               const void *lam_in, const void *Tn, const void *Ci, double *gCi,
                               const Coef &c, unsigned *dev_err, cudaStream_t s,
                               const void *ci_pairs) {
  switch (dt) {
    case IGG_F64:
      if (ci_pairs)
        return launch_adj_t<double, true>(nx, ny, nz, lam_out, lam_in, Tn, Ci, ci_pairs, gCi, c,
                                          dev_err, s);
      return launch_adj_t<double, false>(nx, ny, nz, lam_out, lam_in, Tn, Ci, Ci, gCi, c,
                                         dev_err, s);
    case IGG_F32:
      return launch_adj_t<float, false>(nx, ny, nz, lam_out, lam_in, Tn, Ci, Ci, gCi, c,
                                        dev_err, s);
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pair_ci(const void *Ci, void *pairs, long long n, cudaStream_t s) {
  long long blocks = (n + 255) / 256;
  if (blocks > 8 * 152) blocks = 8 * 152;
  if (blocks < 1) blocks = 1;
  k_pair_ci<<<(unsigned)blocks, 256, 0, s>>>((const double *)Ci, (FF *)pairs, n);
  return cudaGetLastError();
}

}  // namespace igg
