// TMA-pipelined stencil kernel for the regular boxes of the step (the full
// step, its face and inner tile sets, and the boxes of the split), and the
// fix-up launch of the emulated FP64 cell: a producer warp streams, plane by
// plane along z, a tile of T with a one-vector / one-row halo and the
// matching tile of Ci from HBM into a ring of shared-memory stages with
// cp.async.bulk.tensor (TMA); eight consumer warps compute from shared
// memory and write T2 with 16-byte stores. The bytes in flight per SM are
// set by the ring (several stages of ~18 KB per CTA), not by registers, which
// keeps HBM busy.
//
// Ring protocol (per stage s: mbarrier full[s], count 1 + transaction bytes;
// mbarrier empty[s], count = consumer warps): load k goes to stage k % NS;
// the producer waits empty[s] before reusing a stage, arms full[s] with the
// byte count and issues the copies; consumers wait full[s], read, and each
// warp arrives on empty[s]. Load k holds T plane z0-1+k and Ci plane
// z0-2+k; step z uses T planes z (neighbours) and z+1, Ci plane z, and keeps
// T plane z-1 of its own points in registers.
//
// Every wait is bounded (about 2 s of globaltimer); on a timeout the kernel
// records IGG_DEV_ERR_TIMEOUT in the device error word, stops, waits (again
// bounded) for the copies it issued, and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cstring>
#include <mutex>

#include "cell.cuh"
#include "igg_internal.h"
#include "tma_util.cuh"

// resident CTAs per SM the TMA kernels are compiled for (register budget)
#ifndef IGG_TMA_MIN_BLOCKS
#define IGG_TMA_MIN_BLOCKS 3
#endif

namespace igg {
namespace {

// Tile shapes: lanes per row LPR (W = LPR*V points), H rows.
template <class S>
struct WideShape {
  static constexpr int LPR = sizeof(S) == 2 ? 16 : 32;
  static constexpr int H = 16;
};

template <class S, int LPR_, int H_>
struct TmaShape {
  static constexpr int V = 16 / (int)sizeof(S);
  static constexpr int LPR = LPR_;                      // lanes per row
  static constexpr int W = LPR * V;                     // computed points per row
  static constexpr int BW = W + 2 * V;                  // T box width (vector halo each side)
  static constexpr int H = H_;                          // rows per tile
  static constexpr int BH = H + 2;                      // T box height (row halo)
  static constexpr int NS = 4;                          // stages
  static constexpr int CONSUMERS = 8;                   // consumer warps
  static constexpr int ROWS_PER_PASS = CONSUMERS * (32 / LPR);
  static constexpr int RPT = H / ROWS_PER_PASS;         // rows per consumer thread
  static constexpr int TB = BW * BH * (int)sizeof(S);   // T box bytes
  static constexpr int TBA = (TB + 127) / 128 * 128;
  static constexpr int CB = W * H * (int)sizeof(S);     // Ci box bytes
  static constexpr int STAGE = (TBA + CB + 127) / 128 * 128;
  // FP64 (emulated cell): per consumer warp, kFixPend fix-up entries staged
  // before they are appended to the tile set's list
  static constexpr int PEND = NS * STAGE + 2 * NS * 8 + 64;
  static constexpr int SMEM = PEND + (sizeof(S) == 8 ? CONSUMERS * 16 * 16 : 0);  // + flags, staging
  static_assert(H % ROWS_PER_PASS == 0, "rows per tile");
  static_assert(BW <= 256 && BH <= 256, "TMA box dims");
};

template <class S>
__device__ __forceinline__ void lds_vec(const S *p, Vec<S> &o) {
  unpack(*reinterpret_cast<const uint4 *>(p), o);
}
// A tile set's fix-up buffer (layout in igg_internal.h): the entries, then
// the entry count and a block counter.
struct FixEntry {
  long long p;    // index of the first of 32 consecutive points of a row
  unsigned bits;  // bit l: point p + l left to the fix-up
  unsigned pad;
};
// Entries a consumer warp stages in shared memory before it reserves their
// slots in the list with one atomic (a warp waited for each atomic's
// return, row after row, on fields with many such points).
constexpr unsigned kFixPend = 16;
struct FixList {
  FixEntry *e;
  unsigned *count, *done;
  unsigned long long *totals;  // segments and points fixed up since the buffer was made
};
__device__ __forceinline__ FixList fix_list(void *fix, size_t cap) {
  FixEntry *e = reinterpret_cast<FixEntry *>(fix);
  unsigned *c = reinterpret_cast<unsigned *>(e + cap);
  return {e, c, c + 1, reinterpret_cast<unsigned long long *>(c + 2)};
}
constexpr int kFixupBlocks = 8 * 152;

// bit i of x (i < 16) to bit 2i
__device__ __forceinline__ unsigned spread16(unsigned x) {
  x = (x | (x << 8)) & 0x00FF00FFu;
  x = (x | (x << 4)) & 0x0F0F0F0Fu;
  x = (x | (x << 2)) & 0x33333333u;
  x = (x | (x << 1)) & 0x55555555u;
  return x;
}

// How a TMA kernel computes its points: MODE_CELL = the shared cell() of the
// storage type (FP32, BF16); for FP64 fields, MODE_F64 = the FP64 cell and
// MODE_EMU + (3 - NG) = the emulated cell's fast path with NG weight groups
// (the grid's weight_groups); the points its fast path does not take are
// listed for the fix-up launch (k_fixup_f64), which applies cell().
enum { MODE_CELL = 0, MODE_F64 = 1, MODE_EMU = 2, MODE_EMU_LAST = 4 };
__host__ __device__ constexpr bool is_emu(int mode) {
  return mode >= MODE_EMU && mode <= MODE_EMU_LAST;
}
constexpr int emu_mode(int ng) { return MODE_EMU + 3 - ng; }

// V points of one row: centre vector c, x neighbours from c and the points
// beyond it (left, right), y and z neighbour vectors. ok gets bit i for each
// point written to out.
template <class S, int MODE>
__device__ __forceinline__ void compute_vec(const Vec<S> &c, typename Num<S>::C left,
                                            typename Num<S>::C right, const Vec<S> &ym,
                                            const Vec<S> &yp, const Vec<S> &zm, const Vec<S> &zp,
                                            const Vec<S> &ci, const W<typename Num<S>::C> &w,
                                            Vec<S> &out, unsigned &ok) {
  constexpr int V = Vec<S>::V;
  ok = (1u << V) - 1u;
#pragma unroll
  for (int i = 0; i < V; ++i) {
    const auto xm = i == 0 ? left : c.v[i - 1];
    const auto xp = i == V - 1 ? right : c.v[i + 1];
    out.v[i] = cell(c.v[i], xm, xp, ym.v[i], yp.v[i], zm.v[i], zp.v[i], ci.v[i], w);
  }
}

template <>
__device__ __forceinline__ void compute_vec<double, MODE_F64>(
    const Vec<double> &c, double left, double right, const Vec<double> &ym, const Vec<double> &yp,
    const Vec<double> &zm, const Vec<double> &zp, const Vec<double> &ci, const W<double> &w,
    Vec<double> &out, unsigned &ok) {
  ok = 3u;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const double xm = i == 0 ? left : c.v[0];
    const double xp = i == 1 ? right : c.v[1];
    out.v[i] = cell_f64(c.v[i], xm, xp, ym.v[i], yp.v[i], zm.v[i], zp.v[i], ci.v[i], w);
  }
}

// Emulated fast path for both points, computed unconditionally (no branch
// in the common case); ok marks the points whose fast path applies, the
// others are listed for the fix-up launch (the aligned path across powers of
// two or zero, else the FP64 cell).
template <int NG>
__device__ __forceinline__ void compute_vec_emu(
    const Vec<double> &c, double left, double right, const Vec<double> &ym, const Vec<double> &yp,
    const Vec<double> &zm, const Vec<double> &zp, const Vec<double> &ci, const W<double> &w,
    Vec<double> &out, unsigned &ok) {
  const unsigned long long b0 = dbits(c.v[0]), b1 = dbits(c.v[1]);
  const unsigned long long nb0[6] = {dbits(left),     b1,             dbits(ym.v[0]),
                                     dbits(yp.v[0]),  dbits(zm.v[0]), dbits(zp.v[0])};
  const unsigned long long nb1[6] = {b0,              dbits(right),   dbits(ym.v[1]),
                                     dbits(yp.v[1]),  dbits(zm.v[1]), dbits(zp.v[1])};
  unsigned gh0[NG], gh1[NG], gm0[NG], gm1[NG];
  // sign and exponent from the pair's first point (shared by every point of
  // the pair whose stencil passes)
  const unsigned hc = (unsigned)(b0 >> 32);
  const bool okc = emu2_centre_ok(hc);
  bool ok0 = emu2_int<NG>(b0, nb0, gh0, gm0) && okc;
  bool ok1 = emu2_int<NG>(b1, nb1, gh1, gm1) && okc;
  // the FP32 sums of both points as float2 (one instruction per pair)
  float2 fh[NG], fl[NG];
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    // Gh of both points: 1.5 2^23 + Gh minus 1.5 2^23 (exact where ok)
    fh[g] = vadd(make_float2(__uint_as_float(gh0[g]), __uint_as_float(gh1[g])),
                 vset(-kMagic, float2()));
    fl[g] = make_float2(__uint_as_float(gm0[g]), __uint_as_float(gm1[g]));
  }
  float2 S, C;
  emu2_sum<NG>(fh, fl, w, S, C);
  const float2 Kr = vfma(make_float2(emu2_cif(ci.v[0]), emu2_cif(ci.v[1])), C,
                         vset(kMagic, float2()));
  out.v[0] = emu2_apply(b0, hc, ci.v[0], S.x, Kr.x, ok0);
  out.v[1] = emu2_apply(b1, hc, ci.v[1], S.y, Kr.y, ok1);
  ok = (ok0 ? 1u : 0u) | (ok1 ? 2u : 0u);
}
template <>
__device__ __forceinline__ void compute_vec<double, MODE_EMU>(
    const Vec<double> &c, double left, double right, const Vec<double> &ym, const Vec<double> &yp,
    const Vec<double> &zm, const Vec<double> &zp, const Vec<double> &ci, const W<double> &w,
    Vec<double> &out, unsigned &ok) {
  compute_vec_emu<3>(c, left, right, ym, yp, zm, zp, ci, w, out, ok);
}
template <>
__device__ __forceinline__ void compute_vec<double, MODE_EMU + 1>(
    const Vec<double> &c, double left, double right, const Vec<double> &ym, const Vec<double> &yp,
    const Vec<double> &zm, const Vec<double> &zp, const Vec<double> &ci, const W<double> &w,
    Vec<double> &out, unsigned &ok) {
  compute_vec_emu<2>(c, left, right, ym, yp, zm, zp, ci, w, out, ok);
}
template <>
__device__ __forceinline__ void compute_vec<double, MODE_EMU + 2>(
    const Vec<double> &c, double left, double right, const Vec<double> &ym, const Vec<double> &yp,
    const Vec<double> &zm, const Vec<double> &zp, const Vec<double> &ci, const W<double> &w,
    Vec<double> &out, unsigned &ok) {
  compute_vec_emu<1>(c, left, right, ym, yp, zm, zp, ci, w, out, ok);
}

// SWAP = false: rows along y, march along z (box {BW, BH, 1}); SWAP = true:
// rows along z, march along y (box {BW, 1, BH}), for boxes thin in y. The
// cell arithmetic gets the y and z neighbour pairs in their own slots either
// way, so both orientations give the same bits.
//
// BATCH: independent problems of the batched form; a tile's problem (pad[0])
// gives its tensor maps, row pitch, ny and coefficients (TmaBatch) in place
// of mapT, mapC, nx, ny and c0.
template <class S, int LPR_, int H_, bool SWAP, int MODE, bool BATCH = false>
__global__ void __launch_bounds__(32 * 9, IGG_TMA_MIN_BLOCKS)
    k_stencil_tma(const __grid_constant__ CUtensorMap mapT, const __grid_constant__ CUtensorMap mapC,
                  const TmaTile *__restrict__ tiles, S *__restrict__ T2, int nx, int ny, Coef c0,
                  unsigned *__restrict__ dev_err, void *__restrict__ fix, size_t fix_cap,
                  const TmaBatch batch = TmaBatch()) {
  using Sh = TmaShape<S, LPR_, H_>;
  using C = typename Num<S>::C;
  constexpr int V = Sh::V, NS = Sh::NS, LPR = Sh::LPR;
  extern __shared__ __align__(128) unsigned char smem[];
  const unsigned sbase = smem_u32(smem);
  const unsigned full0 = sbase + NS * Sh::STAGE;
  const unsigned empty0 = full0 + NS * 8;
  volatile int *flags = reinterpret_cast<volatile int *>(smem + NS * Sh::STAGE + 2 * NS * 8);
  // flags[0]: abort; flags[1]: loads issued; flags[2]: loads consumed

  const TmaTile t = tiles[blockIdx.x];
  const int K = (t.m1 - t.m0) + 2;
  const CUtensorMap *pmT = &mapT, *pmC = &mapC;
  if constexpr (BATCH) {
    pmT = reinterpret_cast<const CUtensorMap *>(batch.maps + 2 * t.pad[0]);
    pmC = pmT + 1;
    nx = batch.geom[2 * t.pad[0]];  // row pitch
    ny = batch.geom[2 * t.pad[0] + 1];
    c0 = batch.coef[t.pad[0]];
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, Sh::CONSUMERS);
    }
    flags[0] = 0;
    flags[1] = 0;
    flags[2] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();

  if (warp == Sh::CONSUMERS) {
    // ---------------- producer ----------------
    if (lane == 0) {
      int k = 0;
      for (; k < K; ++k) {
        const int s = k % NS;
        if (k >= NS && !mbar_wait(empty0 + 8 * s, ((k / NS) - 1) & 1)) {
          atomicOr(dev_err, IGG_DEV_ERR_TIMEOUT);
          flags[0] = 1;
          break;
        }
        if (flags[0]) break;
        const unsigned bar = full0 + 8 * s;
        const unsigned dst = sbase + s * Sh::STAGE;
        // loads 0 and 1 carry no Ci plane (their planes z0 - 2, z0 - 1 are
        // never used)
        mbar_expect_tx(bar, k >= 2 ? Sh::TB + Sh::CB : Sh::TB);
        const int mT = t.m0 - 1 + k, mC = t.m0 - 2 + k;  // march index of the T / Ci plane
        if (!SWAP) {
          tma_load_3d(dst, pmT, t.x0 - V, t.r0 - 1, t.zoff + mT, bar);
          if (k >= 2) tma_load_3d(dst + Sh::TBA, pmC, t.x0, t.r0, t.zoff + mC, bar);
        } else {
          tma_load_3d(dst, pmT, t.x0 - V, mT, t.zoff + t.r0 - 1, bar);
          if (k >= 2) tma_load_3d(dst + Sh::TBA, pmC, t.x0, mC, t.zoff + t.r0, bar);
        }
      }
      flags[1] = k;
    }
  } else {
    // ---------------- consumers ----------------
    const int sl = lane % LPR;
    const int xs = t.x0 + sl * V;
    const W<C> w = make_w(c0, C(0));
    int rowi[Sh::RPT];
    bool comp[Sh::RPT];
#pragma unroll
    for (int j = 0; j < Sh::RPT; ++j) {
      rowi[j] = warp * (32 / LPR) + lane / LPR + j * Sh::ROWS_PER_PASS;  // row in the tile
      comp[j] = (t.r0 + rowi[j] < t.re) && xs + V > t.xb && xs < t.xe;
    }
    const bool full_vec = xs >= t.xb && xs + V <= t.xe;
    // points of this lane's vector inside the tile's box
    unsigned inm = 0u;
#pragma unroll
    for (int i = 0; i < V; ++i)
      if (xs + i >= t.xb && xs + i < t.xe) inm |= 1u << i;
    // row end cells stored with their T values (Coef::ends; full-step tiles)
    unsigned endm = 0u;
    if (!BATCH && !SWAP && c0.ends) {
#pragma unroll
      for (int i = 0; i < V; ++i)
        if (xs + i == 0 || xs + i == nx - 1) endm |= 1u << i;
    }
    const bool full_st = full_vec || (inm | endm) == (1u << V) - 1u;
    const long long sy = nx, sz = (long long)nx * ny;
    const long long srow = SWAP ? sz : sy, smarch = SWAP ? sy : sz;
    Vec<S> zm[Sh::RPT];
    // loads 0 and 1 (K >= 2 always); afterwards step k waits load k + 1 only,
    // load k having been waited by step k - 1
    // wait results are made warp-uniform: the warp's votes and __syncwarp
    // need every lane in the loop
    bool ok = __all_sync(0xffffffffu, mbar_wait(full0, 0) && mbar_wait(full0 + 8, 0));
    if (!ok) {
      atomicOr(dev_err, IGG_DEV_ERR_TIMEOUT);
      flags[0] = 1;
    } else {
      const S *Tb = reinterpret_cast<const S *>(smem);
#pragma unroll
      for (int j = 0; j < Sh::RPT; ++j) lds_vec(Tb + (rowi[j] + 1) * Sh::BW + V + sl * V, zm[j]);
      __syncwarp();
      if (lane == 0) mbar_arrive(empty0);
    }
    int consumed = 2;
    // the warp's staged fix-up entries (emulated FP64 cell)
    FixEntry *pend = reinterpret_cast<FixEntry *>(smem + Sh::PEND) + warp * kFixPend;
    unsigned npend = 0u;  // warp-uniform
    auto flush = [&]() {
      __syncwarp();
      if (npend) {
        const FixList fl = fix_list(fix, fix_cap);
        unsigned base = 0u;
        if (lane == 0) base = atomicAdd(fl.count, npend);
        base = __shfl_sync(0xffffffffu, base, 0);
        // always within fix_cap: one entry per segment, plane and row at most
        if (lane < npend && base + lane < fix_cap) fl.e[base + lane] = pend[lane];
        npend = 0u;
      }
      __syncwarp();
    };
    // FP64: two march steps per iteration (the z-plane registers alternate
    // instead of being copied; measured faster by a few percent)
    constexpr int kUnroll = sizeof(S) == 8 ? 2 : 1;
#pragma unroll kUnroll
    for (int m = t.m0; ok && m < t.m1; ++m) {
      const int k = m - t.m0 + 1;
      const int s = k % NS, s1 = (k + 1) % NS;
      if (!__all_sync(0xffffffffu, mbar_wait(full0 + 8 * s1, ((k + 1) / NS) & 1))) {
        atomicOr(dev_err, IGG_DEV_ERR_TIMEOUT);
        flags[0] = 1;
        ok = false;
        break;
      }
      consumed = k + 2;
      const S *Tc = reinterpret_cast<const S *>(smem + s * Sh::STAGE);
      const S *Tn = reinterpret_cast<const S *>(smem + s1 * Sh::STAGE);
      const S *Cn = reinterpret_cast<const S *>(smem + s1 * Sh::STAGE + Sh::TBA);
#pragma unroll
      for (int j = 0; j < Sh::RPT; ++j) {
        const int r = rowi[j];
        const S *row = Tc + (r + 1) * Sh::BW + V + sl * V;
        Vec<S> c, up, dn, zp, ci;
        lds_vec(row, c);
        lds_vec(row - Sh::BW, up);
        lds_vec(row + Sh::BW, dn);
        lds_vec(Tn + (r + 1) * Sh::BW + V + sl * V, zp);
        lds_vec(Cn + r * Sh::W + sl * V, ci);
        C left, right;
        if constexpr (sizeof(S) == 8) {
          // FP64: the x neighbours from shared memory (the box's vector
          // halo covers the row ends)
          left = row[-1];
          right = row[V];
        } else {
          left = __shfl_up_sync(0xffffffffu, c.v[V - 1], 1, LPR);
          right = __shfl_down_sync(0xffffffffu, c.v[0], 1, LPR);
          if (sl == 0) left = Num<S>::cv(row[-1]);
          if (sl == LPR - 1) right = Num<S>::cv(row[V]);
        }
        Vec<S> out;
        unsigned okm = (1u << V) - 1u;
        if (comp[j]) {
          // (up, dn) are the row pair, (zm, zp) the march pair
          Vec<S> ym = SWAP ? zm[j] : up, yp = SWAP ? zp : dn;
          Vec<S> zmm = SWAP ? up : zm[j], zpp = SWAP ? dn : zp;
          compute_vec<S, MODE>(c, left, right, ym, yp, zmm, zpp, ci, w, out, okm);
        }
        if (comp[j]) {
          // every point of the box is stored; points the fast path did not
          // take are stored again by the fix-up launch
          const long long di = t.base + xs + srow * (t.r0 + r) + smarch * m;
          S *dst = T2 + di;
          if (!BATCH && !(in_bounds(di, c0.npts) && in_bounds(di + V - 1, c0.npts))) {
            // bounds-checked build only: the store is skipped
          } else if (full_st) {
            if (endm) {
#pragma unroll
              for (int i = 0; i < V; ++i)
                if (endm >> i & 1u) out.v[i] = c.v[i];
            }
            *reinterpret_cast<uint4 *>(dst) = pack(out);
          } else {
#pragma unroll
            for (int i = 0; i < V; ++i)
              if (inm >> i & 1u) Num<S>::st(dst + i, out.v[i]);
          }
        }
        if constexpr (is_emu(MODE)) {
          // The warp owns the whole row (one row per warp, two points per
          // lane): it lists each 32-point segment of the row with points
          // the fast path did not take (its first point and a bit mask).
          static_assert(LPR == 32 && V == 2, "one FP64 row per warp");
          const unsigned defm = comp[j] ? (~okm & inm) : 0u;
          if (__any_sync(0xffffffffu, defm != 0u)) {
            const unsigned b0 = __ballot_sync(0xffffffffu, defm & 1u);
            const unsigned b1 = __ballot_sync(0xffffffffu, defm & 2u);
            // points 32*lane .. 32*lane + 31 (lanes 0, 1): lanes 16*lane ..
            // 16*lane + 15 of the row
            const unsigned h0 = (b0 >> (16 * (lane & 1))) & 0xFFFFu;
            const unsigned h1 = (b1 >> (16 * (lane & 1))) & 0xFFFFu;
            const unsigned word = lane < 2 ? spread16(h0) | (spread16(h1) << 1) : 0u;
            const unsigned has = __ballot_sync(0xffffffffu, word != 0u);  // bits 0, 1
            if (word) {
              FixEntry en;
              en.p = t.base + t.x0 + 32 * lane + srow * (t.r0 + r) + smarch * m;
              en.bits = word;
              en.pad = 0u;
              pend[npend + __popc(has & ((1u << lane) - 1u))] = en;
            }
            npend += __popc(has);
            if (npend > kFixPend - 2) flush();
          }
        }
        zm[j] = c;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(empty0 + 8 * s);
    }
    if constexpr (is_emu(MODE)) flush();
    if (warp == 0 && lane == 0) flags[2] = consumed;
  }
  __syncthreads();
  // After an abort, wait (bounded) for copies issued but never consumed, so
  // that no bulk copy writes into this CTA's shared memory after it exits.
  if (threadIdx.x == 0 && flags[0]) {
    for (int k = flags[2]; k < flags[1]; ++k) {
      if (!mbar_wait(full0 + 8 * (k % NS), (k / NS) & 1)) {
        atomicOr(dev_err, IGG_DEV_ERR_DRAIN);
        break;
      }
    }
  }
}

// Fix-up of an emulated-cell launch: the points whose fast path the kernel
// did not take get what cell() gives them (the same choice and arithmetic
// as every kernel: the aligned path for stencils across powers of two or
// zero, else the FP64 cell). The kernel listed every 32-point row segment
// with such points (its first point and a bit mask). Each warp takes
// kFixBatch entries at a time (one per lane of lanes 0..kFixBatch-1) and
// deals their listed points out to its lanes, 32 at a time, in the order of
// the entries and their bits, so that lanes are not left idle by sparse
// masks. Each block adds its segments and points to the list's totals; the
// last block to finish resets the list.
constexpr unsigned kFixBatch = 4;
__global__ void __launch_bounds__(256)
    k_fixup_f64(void *__restrict__ fix, size_t cap, double *__restrict__ T2,
                const double *__restrict__ T, const double *__restrict__ Ci, int nx, int ny,
                Coef c0) {
  const FixList fl = fix_list(fix, cap);
  const unsigned count = (unsigned)min((size_t)*(volatile unsigned *)fl.count, cap);
  const W<double> w = make_w(c0, 0.0);
  const long long sy = nx, sz = (long long)nx * ny;
  const int lane = threadIdx.x & 31;
  const unsigned warps = gridDim.x * (blockDim.x >> 5);
  const unsigned gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  unsigned segs = 0u, pts = 0u;
  for (unsigned b = gw * kFixBatch; b < count; b += warps * kFixBatch) {
    FixEntry en = {};
    if (lane < (int)kFixBatch && b + lane < count) en = fl.e[b + lane];
    // inclusive prefix of the entries' point counts over lanes 0..kFixBatch-1
    unsigned pre = __popc(en.bits);
#pragma unroll
    for (unsigned d = 1; d < kFixBatch; d <<= 1) {
      const unsigned v = __shfl_up_sync(0xffffffffu, pre, d);
      if ((unsigned)lane >= d) pre += v;
    }
    const unsigned total = __shfl_sync(0xffffffffu, pre, kFixBatch - 1);
    segs += __popc(__ballot_sync(0xffffffffu, en.bits != 0u));
    pts += total;
    unsigned pk[kFixBatch], bk[kFixBatch];
    long long qk[kFixBatch];
#pragma unroll
    for (unsigned q = 0; q < kFixBatch; ++q) {
      pk[q] = __shfl_sync(0xffffffffu, pre, q);
      bk[q] = __shfl_sync(0xffffffffu, en.bits, q);
      qk[q] = __shfl_sync(0xffffffffu, en.p, q);
    }
    for (unsigned r = 0; r < total; r += 32u) {
      const unsigned rank = r + lane;
      if (rank >= total) break;
      // the entry holding the point of this rank and the point's bit
      unsigned q = 0u;
#pragma unroll
      for (unsigned k = 0; k + 1 < kFixBatch; ++k) q += rank >= pk[k] ? 1u : 0u;
      unsigned bits = bk[0], excl = 0u;
      long long p0 = qk[0];
#pragma unroll
      for (unsigned k = 1; k < kFixBatch; ++k)
        if (q == k) {
          bits = bk[k];
          excl = pk[k - 1];
          p0 = qk[k];
        }
      const long long p = p0 + __fns(bits, 0u, (int)(rank - excl + 1u));
      if (in_bounds(p - sz, c0.npts) && in_bounds(p + sz, c0.npts)) {
        const double tc = __ldg(T + p);
        const double tn[6] = {__ldg(T + p - 1),  __ldg(T + p + 1),  __ldg(T + p - sy),
                              __ldg(T + p + sy), __ldg(T + p - sz), __ldg(T + p + sz)};
        T2[p] = cell_emu_not_fast(tc, tn, __ldg(Ci + p), w);
      }
    }
  }
  __shared__ unsigned bsum[2];
  if (threadIdx.x == 0) bsum[0] = bsum[1] = 0u;
  __syncthreads();
  if (lane == 0 && segs) {
    atomicAdd(&bsum[0], segs);
    atomicAdd(&bsum[1], pts);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (bsum[0]) {
      atomicAdd(fl.totals, (unsigned long long)bsum[0]);
      atomicAdd(fl.totals + 1, (unsigned long long)bsum[1]);
    }
    __threadfence();
    if (atomicAdd(fl.done, 1u) == gridDim.x - 1) {
      *fl.count = 0u;
      *fl.done = 0u;
    }
  }
}

template <class S, class Shp, bool SWAP, int MODE>
cudaError_t prepare_t(int *ctas_per_sm) {
  using Sh = TmaShape<S, Shp::LPR, Shp::H>;
  auto kern = k_stencil_tma<S, Shp::LPR, Shp::H, SWAP, MODE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Sh::SMEM);
  if (e == cudaSuccess && ctas_per_sm)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, kern, 32 * (Sh::CONSUMERS + 1),
                                                      Sh::SMEM);
  return e;
}

template <class S, class Shp, bool SWAP, int MODE>
cudaError_t launch_t(const TmaTile *tiles, int ntiles, void *T2, const void *T, const void *Ci,
                     int nx, int ny, long long nzt, const Coef &c, unsigned *dev_err,
                     FixBuf fix, cudaStream_t s) {
  using Sh = TmaShape<S, Shp::LPR, Shp::H>;
  CUtensorMap mT, mC;
  const bool ok = SWAP ? encode<S>(&mT, T, nx, ny, nzt, Sh::BW, 1, Sh::BH) &&
                             encode<S>(&mC, Ci, nx, ny, nzt, Sh::W, 1, Sh::H)
                       : encode<S>(&mT, T, nx, ny, nzt, Sh::BW, Sh::BH, 1) &&
                             encode<S>(&mC, Ci, nx, ny, nzt, Sh::W, Sh::H, 1);
  if (!ok) return cudaErrorInvalidValue;
  Coef cc = c;
  cc.npts = (long long)nx * ny * nzt;
  k_stencil_tma<S, Shp::LPR, Shp::H, SWAP, MODE>
      <<<ntiles, 32 * (Sh::CONSUMERS + 1), Sh::SMEM, s>>>(mT, mC, tiles, (S *)T2, nx, ny, cc,
                                                          dev_err, fix.p, fix.cap);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && is_emu(MODE)) {
    k_fixup_f64<<<kFixupBlocks, 256, 0, s>>>(fix.p, fix.cap, (double *)T2, (const double *)T,
                                            (const double *)Ci, nx, ny, cc);
    e = cudaGetLastError();
  }
  return e;
}

// FP64 fields pick the kernel of the grid's FP64 mode; other types the cell.
template <class S>
cudaError_t prepare_v(int variant, int *ctas) {
  if (variant != TMA_WIDE && variant != TMA_WIDE_SWAP) return cudaErrorInvalidValue;
  const bool swap = variant == TMA_WIDE_SWAP;
  if constexpr (sizeof(S) == 8) {
    cudaError_t e = swap ? prepare_t<S, WideShape<S>, true, MODE_F64>(nullptr)
                         : prepare_t<S, WideShape<S>, false, MODE_F64>(nullptr);
    if (e == cudaSuccess)
      e = swap ? prepare_t<S, WideShape<S>, true, MODE_EMU + 1>(nullptr)
               : prepare_t<S, WideShape<S>, false, MODE_EMU + 1>(nullptr);
    if (e == cudaSuccess)
      e = swap ? prepare_t<S, WideShape<S>, true, MODE_EMU + 2>(nullptr)
               : prepare_t<S, WideShape<S>, false, MODE_EMU + 2>(nullptr);
    if (e != cudaSuccess) return e;
    return swap ? prepare_t<S, WideShape<S>, true, MODE_EMU>(ctas)
                : prepare_t<S, WideShape<S>, false, MODE_EMU>(ctas);
  } else {
    return swap ? prepare_t<S, WideShape<S>, true, MODE_CELL>(ctas)
                : prepare_t<S, WideShape<S>, false, MODE_CELL>(ctas);
  }
}

template <class S, bool SWAP>
cudaError_t launch_m(const TmaTile *tiles, int ntiles, void *T2, const void *T, const void *Ci,
                     int nx, int ny, long long nzt, const Coef &c, unsigned *dev_err,
                     FixBuf fix, cudaStream_t s) {
  if constexpr (sizeof(S) == 8) {
    if (c.f64_emu) {
      if (!fix.p) return cudaErrorInvalidValue;
      switch (weight_groups(c.wx, c.wy, c.wz)) {
        case 1:
          return launch_t<S, WideShape<S>, SWAP, emu_mode(1)>(tiles, ntiles, T2, T, Ci, nx, ny,
                                                              nzt, c, dev_err, fix, s);
        case 2:
          return launch_t<S, WideShape<S>, SWAP, emu_mode(2)>(tiles, ntiles, T2, T, Ci, nx, ny,
                                                              nzt, c, dev_err, fix, s);
        default:
          return launch_t<S, WideShape<S>, SWAP, emu_mode(3)>(tiles, ntiles, T2, T, Ci, nx, ny,
                                                              nzt, c, dev_err, fix, s);
      }
    }
    return launch_t<S, WideShape<S>, SWAP, MODE_F64>(tiles, ntiles, T2, T, Ci, nx, ny, nzt, c,
                                                     dev_err, fix, s);
  } else {
    return launch_t<S, WideShape<S>, SWAP, MODE_CELL>(tiles, ntiles, T2, T, Ci, nx, ny, nzt, c,
                                                      dev_err, fix, s);
  }
}

template <class S>
cudaError_t launch_v(int variant, const TmaTile *tiles, int ntiles, void *T2, const void *T,
                     const void *Ci, int nx, int ny, long long nzt, const Coef &c,
                     unsigned *dev_err, FixBuf fix, cudaStream_t s) {
  switch (variant) {
    case TMA_WIDE:
      return launch_m<S, false>(tiles, ntiles, T2, T, Ci, nx, ny, nzt, c, dev_err, fix, s);
    case TMA_WIDE_SWAP:
      return launch_m<S, true>(tiles, ntiles, T2, T, Ci, nx, ny, nzt, c, dev_err, fix, s);
  }
  return cudaErrorInvalidValue;
}

// The batched form's launch: non-swapped wide tiles, the storage type's cell
// (FP64 batches: the FP64 cell), maps from the TmaBatch table.
template <class S>
cudaError_t launch_batch_t(const TmaTile *tiles, int ntiles, void *T2, const TmaBatch &b,
                           unsigned *dev_err, cudaStream_t s) {
  using Shp = WideShape<S>;
  using Sh = TmaShape<S, Shp::LPR, Shp::H>;
  constexpr int MODE = sizeof(S) == 8 ? MODE_F64 : MODE_CELL;
  CUtensorMap none;
  std::memset(&none, 0, sizeof none);
  k_stencil_tma<S, Shp::LPR, Shp::H, false, MODE, true>
      <<<ntiles, 32 * (Sh::CONSUMERS + 1), Sh::SMEM, s>>>(none, none, tiles, (S *)T2, 0, 0,
                                                          Coef(), dev_err, nullptr, 0, b);
  return cudaGetLastError();
}

template <class S>
cudaError_t prepare_batch_t() {
  using Shp = WideShape<S>;
  using Sh = TmaShape<S, Shp::LPR, Shp::H>;
  constexpr int MODE = sizeof(S) == 8 ? MODE_F64 : MODE_CELL;
  return cudaFuncSetAttribute(k_stencil_tma<S, Shp::LPR, Shp::H, false, MODE, true>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, Sh::SMEM);
}

template <class S>
bool batch_maps_t(const void *T, const void *Ci, int nprob, const long long *off, const int *sz,
                  const int *pitch, TmaMapBytes *out) {
  using Shp = WideShape<S>;
  using Sh = TmaShape<S, Shp::LPR, Shp::H>;
  auto fn = encode_fn();
  if (!fn) return false;
  const CUtensorMapDataType t = sizeof(S) == 8   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                : sizeof(S) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  for (int p = 0; p < nprob; ++p) {
    const cuuint64_t dims[3] = {(cuuint64_t)sz[3 * p], (cuuint64_t)sz[3 * p + 1],
                                (cuuint64_t)sz[3 * p + 2]};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch[p] * sizeof(S),
                                   (cuuint64_t)pitch[p] * sz[3 * p + 1] * sizeof(S)};
    const cuuint32_t estr[3] = {1, 1, 1};
    const cuuint32_t boxT[3] = {(cuuint32_t)Sh::BW, (cuuint32_t)Sh::BH, 1};
    const cuuint32_t boxC[3] = {(cuuint32_t)Sh::W, (cuuint32_t)Sh::H, 1};
    const char *tb = static_cast<const char *>(T) + off[p] * (long long)sizeof(S);
    const char *cb = static_cast<const char *>(Ci) + off[p] * (long long)sizeof(S);
    for (int k = 0; k < 2; ++k)
      if (fn(reinterpret_cast<CUtensorMap *>(&out[2 * p + k]), t, 3,
             const_cast<char *>(k == 0 ? tb : cb), dims, strides, k == 0 ? boxT : boxC, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
  }
  return true;
}

}  // namespace

int tma_tile_width(igg_dtype dt, int) {
  switch (dt) {
    case IGG_F64: return WideShape<double>::LPR * 2;
    case IGG_F32: return WideShape<float>::LPR * 4;
    case IGG_BF16: return WideShape<__nv_bfloat16>::LPR * 8;
  }
  return 0;
}

int tma_tile_rows(igg_dtype dt, int) {
  switch (dt) {
    case IGG_F64: return WideShape<double>::H;
    case IGG_F32: return WideShape<float>::H;
    case IGG_BF16: return WideShape<__nv_bfloat16>::H;
  }
  return 0;
}

bool tma_available() { return encode_fn() != nullptr; }

static_assert(sizeof(TmaMapBytes) == sizeof(CUtensorMap) && alignof(TmaMapBytes) >= 64,
              "tensor map storage");

bool tma_batch_maps(igg_dtype dt, const void *T, const void *Ci, int nprob, const long long *off,
                    const int *sizes, const int *pitch, TmaMapBytes *out) {
  switch (dt) {
    case IGG_F64: return batch_maps_t<double>(T, Ci, nprob, off, sizes, pitch, out);
    case IGG_F32: return batch_maps_t<float>(T, Ci, nprob, off, sizes, pitch, out);
    case IGG_BF16: return batch_maps_t<__nv_bfloat16>(T, Ci, nprob, off, sizes, pitch, out);
  }
  return false;
}

cudaError_t tma_batch_prepare(igg_dtype dt) {
  switch (dt) {
    case IGG_F64: return prepare_batch_t<double>();
    case IGG_F32: return prepare_batch_t<float>();
    case IGG_BF16: return prepare_batch_t<__nv_bfloat16>();
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_stencil_tma_batch(igg_dtype dt, const TmaTile *tiles, int ntiles, void *T2,
                                     const TmaBatch &b, unsigned *dev_err, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  switch (dt) {
    case IGG_F64: return launch_batch_t<double>(tiles, ntiles, T2, b, dev_err, s);
    case IGG_F32: return launch_batch_t<float>(tiles, ntiles, T2, b, dev_err, s);
    case IGG_BF16: return launch_batch_t<__nv_bfloat16>(tiles, ntiles, T2, b, dev_err, s);
  }
  return cudaErrorInvalidValue;
}


size_t tma_fix_cap(const TmaTile *tiles, int ntiles) {
  size_t cap = 0;
  for (int i = 0; i < ntiles; ++i) {
    const TmaTile &t = tiles[i];
    const size_t segs = (size_t)(t.xe - t.x0 + 31) / 32;  // 32-point segments of a row
    cap += segs * (size_t)(t.re - t.r0) * (size_t)(t.m1 - t.m0);
  }
  return cap;
}

cudaError_t tma_prepare(igg_dtype dt, int variant, int *ctas_per_sm) {
  switch (dt) {
    case IGG_F64: return prepare_v<double>(variant, ctas_per_sm);
    case IGG_F32: return prepare_v<float>(variant, ctas_per_sm);
    case IGG_BF16: return prepare_v<__nv_bfloat16>(variant, ctas_per_sm);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_stencil_tma(igg_dtype dt, int variant, const TmaTile *tiles, int ntiles,
                               void *T2, const void *T, const void *Ci, int nx, int ny,
                               long long nzt, const Coef &c, unsigned *dev_err,
                               FixBuf fix, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  switch (dt) {
    case IGG_F64:
      return launch_v<double>(variant, tiles, ntiles, T2, T, Ci, nx, ny, nzt, c, dev_err, fix,
                              s);
    case IGG_F32:
      return launch_v<float>(variant, tiles, ntiles, T2, T, Ci, nx, ny, nzt, c, dev_err, fix,
                             s);
    case IGG_BF16:
      return launch_v<__nv_bfloat16>(variant, tiles, ntiles, T2, T, Ci, nx, ny, nzt, c, dev_err,
                                     fix, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t tma_bounds_flag(unsigned *out, bool clear) { return read_bounds_flag(out, clear); }

}  // namespace igg
