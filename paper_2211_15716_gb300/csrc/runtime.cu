// Host runtime of the library: the implicit global grid (Sec. Approach;
// Fig. 1 init_global_grid / nx_g / finalize_global_grid), its halo-copy
// descriptor tables, the tile tables of the full step and of the
// boundary/inner split, the high- and low-priority streams of the hidden
// step, and the CUDA graphs of the time loop.
#include <algorithm>
#include <array>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "igg_internal.h"

namespace igg {

static thread_local std::string g_err;

int set_error(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_error(cudaError_t e, const char *what) {
  return set_error(IGG_ECUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

void clear_error() { g_err.clear(); }

size_t dtype_size(igg_dtype t) {
  switch (t) {
    case IGG_F64: return 8;
    case IGG_F32: return 4;
    case IGG_BF16: return 2;
  }
  return 0;
}

Coef make_coef(double lam, double dt, double dx, double dy, double dz) {
  const double k = dt * lam;
  Coef c;
  c.wx = k / (dx * dx);
  c.wy = k / (dy * dy);
  c.wz = k / (dz * dz);
  c.wc = -2.0 * (c.wx + c.wy + c.wz);
  c.f64_emu = 0;
  c.ends = 0;
  c.npts = 0;
  return c;
}

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
namespace {

struct DeviceGuard {
  int prev = -1;
  bool changed = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
      changed = cudaSetDevice(dev) == cudaSuccess;
    }
  }
  ~DeviceGuard() {
    if (changed) cudaSetDevice(prev);
  }
};

// Device tile table of one launch: Tile (scalar kernel, V = 1), VTile
// (vector kernel) or TmaTile (TMA kernel variant tma >= 0).
struct TileSet {
  void *dev = nullptr;
  int n = 0;
  int V = 1;
  int tma = -1;
  FixBuf fix;  // fix-up list (FP64 TMA tile sets)
};

// The split: boundary set (one launch per tile kind) and inner block.
struct SplitTiles {
  std::vector<TileSet> boundary;
  TileSet inner;
};

// The full step's TMA tiles in two sets: face tiles (reading a halo cell or
// computing a point of a sent plane) and the rest (IGG_OPT_HIDE_HALO).
struct PartTiles {
  TileSet face, inner;
};

using GraphKey = std::tuple<const void *, const void *, const void *, int, int, int, int, int,
                            double, double, double, double>;

bool aligned16(const void *p) { return p != nullptr && ((uintptr_t)p & 15u) == 0; }

// MPI_Dims_create's rule: the free entries multiply to the remaining factor,
// are as balanced as possible (smallest largest factor, then smallest spread)
// and non-increasing.
bool dims_create(int nsub, int dims[3]) {
  int fixed = 1, nfree = 0, free_idx[3];
  for (int d = 0; d < 3; ++d) {
    if (dims[d] < 0) return false;
    if (dims[d] == 0) free_idx[nfree++] = d;
    else fixed *= dims[d];
  }
  if (nsub <= 0 || nsub % fixed) return false;
  const int rest = nsub / fixed;
  if (nfree == 0) return rest == 1;
  int best[3] = {0, 0, 0}, best_max = 0, best_spread = 0;
  bool found = false;
  const int lim1 = nfree >= 2 ? rest : 1, lim2 = nfree >= 3 ? rest : 1;
  for (int a = 1; a <= rest; ++a) {
    if (rest % a) continue;
    for (int b = 1; b <= lim1; ++b) {
      if ((rest / a) % b) continue;
      for (int c = 1; c <= lim2; ++c) {
        const long long prod = (long long)a * b * c;
        if (prod != rest) continue;
        const int f[3] = {a, b, c};
        bool nonincr = true;
        for (int i = 1; i < nfree; ++i) nonincr = nonincr && f[i - 1] >= f[i];
        if (!nonincr) continue;
        int mx = 0, mn = 1 << 30;
        for (int i = 0; i < nfree; ++i) mx = std::max(mx, f[i]), mn = std::min(mn, f[i]);
        if (!found || mx < best_max || (mx == best_max && mx - mn < best_spread)) {
          found = true;
          best_max = mx;
          best_spread = mx - mn;
          for (int i = 0; i < 3; ++i) best[i] = f[i];
        }
      }
    }
  }
  if (!found) return false;
  for (int i = 0; i < nfree; ++i) dims[free_idx[i]] = best[i];
  return true;
}

// Rows of z planes per tile: enough tiles to fill the GPU several times over,
// but long z sweeps (each tile re-reads two extra planes).
int choose_zb(long long xy_tiles, int zext) {
  int zb = 64;
  while (zb > 8 && xy_tiles * ((zext + zb - 1) / zb) < 8 * 152 * 4) zb /= 2;
  return std::max(1, std::min(zb, zext));
}

void add_box(std::vector<Tile> &v, long long base, int nx, int ny, int x0, int x1, int y0,
             int y1, int z0, int z1, int zb, int param) {
  if (x0 >= x1 || y0 >= y1 || z0 >= z1) return;
  for (int zc = z0; zc < z1; zc += zb)
    for (int y = y0; y < y1; y += kTileY)
      for (int x = x0; x < x1; x += kTileX) {
        Tile t;
        t.base = base;
        t.nx = nx;
        t.ny = ny;
        t.x0 = x;
        t.y0 = y;
        t.xe = x1;
        t.ye = y1;
        t.z0 = zc;
        t.z1 = std::min(zc + zb, z1);
        t.param = param;
        t.xb = x;
        v.push_back(t);
      }
}

// Tiles of the vector kernel for the box [x0,x1) x [y0,y1) x [z0,z1) of one
// array. Rows run along y and the tiles march along z, unless the box is thin
// in y (fewer than kVecWarps rows) and longer in z: then rows run along z and
// the tiles march along y. A row of a tile is a segment of lpr lanes, the
// smallest power of two (<= 32) that covers the box's width in vectors.
}  // namespace

void add_box_vec_pitched(std::vector<VTile> &v, long long base, int nx, int pitch, int ny, int x0,
                         int x1, int y0, int y1, int z0, int z1, int zb, int param, int V) {
  if (x0 >= x1 || y0 >= y1 || z0 >= z1) return;
  const long long sxy = (long long)pitch * ny;
  const bool swap = (y1 - y0) < kVecWarps && (z1 - z0) > (y1 - y0);
  const int r0 = swap ? z0 : y0, r1 = swap ? z1 : y1;
  const int m0 = swap ? y0 : z0, m1 = swap ? y1 : z1;
  const long long sr = swap ? sxy : pitch, sm = swap ? pitch : sxy;
  const int mb = swap ? (m1 - m0) : zb;
  const int a0 = (x0 / V) * V;
  const int nvec = (x1 - a0 + V - 1) / V;
  int lg = 0;
  while ((1 << lg) < nvec && lg < 5) ++lg;
  const int lpr = 1 << lg;
  const int rows_per_cta = kVecWarps * (32 / lpr);
  const int span = lpr * V;
  for (int mc = m0; mc < m1; mc += mb)
    for (int r = r0; r < r1; r += rows_per_cta)
      for (int xa = a0; xa < x1; xa += span) {
        VTile t;
        t.base = base;
        t.sr = sr;
        t.sm = sm;
        t.nx = nx;
        t.x0 = xa;
        t.xb = std::max(x0, xa);
        t.xe = std::min(x1, xa + span);
        t.r0 = r;
        t.re = std::min(r + rows_per_cta, r1);
        t.m0 = mc;
        t.m1 = std::min(mc + mb, m1);
        t.param = param;
        t.lpr_log2 = (unsigned short)lg;
        t.swap = swap ? 1 : 0;
        v.push_back(t);
      }
}

namespace {

void add_box_vec(std::vector<VTile> &v, long long base, int nx, int ny, int x0, int x1, int y0,
                 int y1, int z0, int z1, int zb, int param, int V) {
  add_box_vec_pitched(v, base, nx, nx, ny, x0, x1, y0, y1, z0, z1, zb, param, V);
}

// dtype whose vector width is V (V = 16 / element size)
igg_dtype dtype_of_vec(int V) { return V == 2 ? IGG_F64 : V == 4 ? IGG_F32 : IGG_BF16; }

// z depth of TMA tiles: each tile loads two extra planes of T and of Ci, so
// deeper is cheaper, but the tile count should fill whole waves of resident
// CTAs; minimise (extra-plane cost) / (wave efficiency).
int choose_zb_tma(long long xy_tiles, int zext, long long slots) {
  int best = std::min(64, zext);
  double best_cost = 1e30;
  for (int zb : {16, 24, 32, 40, 48, 64, 96, 128}) {
    const int z = std::min(zb, zext);
    const long long nt = xy_tiles * ((zext + z - 1) / z);
    const long long waves = (nt + slots - 1) / slots;
    const double eff = (double)nt / (double)(waves * slots);
    const double cost = (1.0 + (2.0 / z) * (2.0 / 3.0)) / eff;
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best = z;
    }
    if (zb >= zext) break;
  }
  return best;
}

long long tma_xy_tiles(int x0, int x1, int y0, int y1, int V, int Wt, int Ht) {
  if (x0 >= x1 || y0 >= y1) return 0;
  const int a0 = (x0 / V) * V;
  return (long long)((x1 - a0 + Wt - 1) / Wt) * ((y1 - y0 + Ht - 1) / Ht);
}

// resident-CTA slots of a TMA kernel variant for the dtype of vector width V
long long tma_slots(int V, int variant = TMA_WIDE) {
  int per_sm = 1, sms = 152, dev = 0;
  if (tma_prepare(dtype_of_vec(V), variant, &per_sm) != cudaSuccess || per_sm < 1) per_sm = 1;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return (long long)per_sm * sms;
}

}  // namespace

// Tiles of a TMA kernel variant for one box of the subdomain whose planes
// start at zoff. Rows run over [r0, r1) in blocks of Ht, the march over
// [m0, m1) in chunks of mb: rows y / march z, or (swapped variant) rows z /
// march y.
void add_box_tma(std::vector<TmaTile> &v, long long base, long long zoff, int x0, int x1, int r0,
                 int r1, int m0, int m1, int mb, int V, int Wt, int Ht) {
  if (x0 >= x1 || r0 >= r1 || m0 >= m1) return;
  for (int mc = m0; mc < m1; mc += mb)
    for (int r = r0; r < r1; r += Ht)
      for (int xa = (x0 / V) * V; xa < x1; xa += Wt) {
        TmaTile t;
        t.base = base;
        t.x0 = xa;
        t.xb = std::max(x0, xa);
        t.xe = std::min(x1, xa + Wt);
        t.r0 = r;
        t.re = std::min(r + Ht, r1);
        t.m0 = mc;
        t.m1 = std::min(mc + mb, m1);
        t.zoff = (int)zoff;
        t.pad[0] = t.pad[1] = 0;
        v.push_back(t);
      }
}

namespace {

// Tiles of one box for the kernel of the set: scalar (V = 1), vector or TMA.
struct TileLists {
  std::vector<Tile> scalar;
  std::vector<VTile> vec;
  std::vector<TmaTile> tma;
};
void add_tiles(TileLists &v, int V, long long base, int nx, int ny, int x0, int x1, int y0,
               int y1, int z0, int z1, int zb, int param) {
  if (V > 1) add_box_vec(v.vec, base, nx, ny, x0, x1, y0, y1, z0, z1, zb, param, V);
  else add_box(v.scalar, base, nx, ny, x0, x1, y0, y1, z0, z1, zb, param);
}

long long xy_tiles_of(int x0, int x1, int y0, int y1) {
  if (x0 >= x1 || y0 >= y1) return 0;
  return (long long)((x1 - x0 + kTileX - 1) / kTileX) * ((y1 - y0 + kTileY - 1) / kTileY);
}

template <class TT>
int upload_vec(const std::vector<TT> &v, TileSet *out) {
  out->n = (int)v.size();
  out->dev = nullptr;
  if (v.empty()) return IGG_OK;
  cudaError_t e = cudaMalloc(&out->dev, v.size() * sizeof(TT));
  if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(tiles)");
  e = cudaMemcpy(out->dev, v.data(), v.size() * sizeof(TT), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_error(e, "cudaMemcpy(tiles)");
  return IGG_OK;
}

int upload_tiles(const TileLists &v, int V, TileSet *out, int tma = -1) {
  out->V = V;
  out->tma = tma;
  out->fix = FixBuf();
  if (tma >= 0) {
    if (int rc = upload_vec(v.tma, out)) return rc;
    if (V == 2 && out->n > 0) {  // FP64: list of the emulated cell's fix-up
      out->fix.cap = tma_fix_cap(v.tma.data(), out->n);
      const size_t bytes = tma_fix_bytes(out->fix.cap);
      cudaError_t e = cudaMalloc(&out->fix.p, bytes);
      if (e == cudaSuccess) e = cudaMemset(out->fix.p, 0, bytes);
      if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(fix-up list)");
    }
    return IGG_OK;
  }
  return V > 1 ? upload_vec(v.vec, out) : upload_vec(v.scalar, out);
}

void free_tiles(TileSet &t) {
  cudaFree(t.dev);
  cudaFree(t.fix.p);
  t.dev = nullptr;
  t.fix = FixBuf();
}

}  // namespace
}  // namespace igg

using namespace igg;

struct igg_grid {
  int n[3], dims[3], overlap[3], periods[3], ng[3];
  int nsub = 0;
  int device = 0;
  long long nloc = 0;
  std::vector<int> left, right;  // [nsub*3]
  cudaStream_t hi = nullptr, lo = nullptr, cap = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_hi = nullptr, ev_lo = nullptr, ev_face = nullptr;
  std::map<int, TileSet> full;                     // keyed by V (1 = scalar tiles)
  std::map<int, PartTiles> part;                   // keyed by V (TMA tiles only)
  std::map<std::array<int, 4>, SplitTiles> split;  // keyed by widths and V
  PlaneCopy *copies[3] = {nullptr, nullptr, nullptr};
  int ncopies[3] = {0, 0, 0};
  // plane-copy tables of staggered field sizes (igg_update_halo_staggered)
  struct Tables {
    PlaneCopy *copies[3] = {nullptr, nullptr, nullptr};
    int ncopies[3] = {0, 0, 0};
  };
  std::map<std::array<int, 3>, Tables> staggered;
  std::map<GraphKey, cudaGraphExec_t> graphs;
  unsigned *dev_err = nullptr;  // device error word of the pipelined kernels
  int *nbr = nullptr;           // device copy of left/right per subdomain and dimension
  bool tma_enabled = true;      // TMA kernel for the regular boxes when available
  int f64_emu = 1;              // FP64 fields: emulated FP64 cell (1) or FP64 cell (0)
  bool fused_halo = true;       // hidden steps: full-step tiles (else the boundary/inner split)
  bool hide_halo = false;       // full-step tiles in face/inner sets, halo update beside the inner
  // IGG_OPT_PHASE_TIMES: three events per step queued outside graph
  // capture (start, end of the stencil launches, end of the step)
  bool phase_times = false;
  std::vector<cudaEvent_t> pev;
  int pev_used = 0;
};

namespace {

int check_grid(const igg_grid *g) {
  if (!g) return set_error(IGG_EINVAL, "grid handle is NULL");
  return IGG_OK;
}

int check_field(const igg_grid *g, const void *p, const char *name) {
  if (!p) return set_error(IGG_EINVAL, "%s is NULL", name);
  if (!aligned16(p)) return set_error(IGG_EINVAL, "%s is not 16-byte aligned", name);
  (void)g;
  return IGG_OK;
}

int check_dtype(igg_dtype t) {
  if (dtype_size(t) == 0) return set_error(IGG_EINVAL, "unknown dtype %d", (int)t);
  return IGG_OK;
}

int check_coef(double lam, double dt, double dx, double dy, double dz) {
  if (!(dx > 0) || !(dy > 0) || !(dz > 0))
    return set_error(IGG_EINVAL, "grid spacings must be positive");
  if (!(lam == lam) || !(dt == dt)) return set_error(IGG_EINVAL, "lam or dt is NaN");
  return IGG_OK;
}

// The TMA kernel takes the regular boxes (full step, inner block) of grids
// whose rows are 16-byte multiples, unless disabled on the grid.
// A dimension of size 1 is absent (2-D and 1-D grids): its only index is
// inner, its neighbour stride 0 (zero second difference), its weight 0.
bool low_dim(const igg_grid *g) { return g->n[1] == 1 || g->n[2] == 1; }
int lo_in(int n) { return n > 1 ? 1 : 0; }
int hi_in(int n) { return n > 1 ? n - 1 : 1; }

// Zero neighbour strides of absent dimensions in vector tiles (rows along y
// and march along z, or swapped).
void zero_absent_strides(const igg_grid *g, std::vector<VTile> &v) {
  for (VTile &t : v) {
    const bool ya = g->n[1] == 1, za = g->n[2] == 1;
    if (t.swap ? za : ya) t.sr = 0;
    if (t.swap ? ya : za) t.sm = 0;
  }
}

bool use_tma(const igg_grid *g, int V) {
  return V > 1 && g->tma_enabled && tma_available() && !low_dim(g);
}

// Vector width used for dtype dt on this grid (1 = scalar kernel): the
// 16-byte vector kernel needs rows of a multiple of V points.
int grid_vec(const igg_grid *g, igg_dtype dt) {
  const int V = vec_width(dt);
  return (V > 1 && g->n[0] % V == 0) ? V : 1;
}

// Tiles of one box per subdomain, for the full step.
// The full step's TMA tiles of every subdomain. Tile order: for each (z
// chunk, row block) the tiles of the subdomains that are neighbours in x
// side by side (measured faster than subdomain after subdomain).
void full_tma_list(const igg_grid *g, int V, int zbt, int Wt, int Ht, std::vector<TmaTile> &out) {
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  std::vector<std::vector<TmaTile>> per(g->nsub);
  for (int s = 0; s < g->nsub; ++s)
    add_box_tma(per[s], (long long)s * g->nloc, (long long)s * nz, 1, nx - 1, 1, ny - 1, 1,
                nz - 1, zbt, V, Wt, Ht);
  const int nrow = (int)((nx - 1 + Wt - 1) / Wt);  // tiles per row block (x0 = 0 .. nx - 2)
  const int dx = g->dims[0];
  for (int syz = 0; syz < g->nsub / dx; ++syz)
    for (size_t b = 0; b < per[syz * dx].size(); b += nrow)
      for (int sx = 0; sx < dx; ++sx) {
        const std::vector<TmaTile> &p = per[sx + dx * syz];
        out.insert(out.end(), p.begin() + b, p.begin() + std::min(p.size(), b + nrow));
      }
}

// Whether a full-step tile reads a halo cell or computes a point of a sent
// plane in a dimension with exchanges: computed range [lo, hi) of a
// dimension of n points, overlap o; the halo cells are 0 and n - 1, the
// sent planes o - 1 and n - o.
bool touches_faces(const igg_grid *g, const TmaTile &t) {
  auto side = [](int lo, int hi, int n, int o) { return lo <= o - 1 || hi > n - o; };
  const bool ex[3] = {g->ncopies[0] > 0, g->ncopies[1] > 0, g->ncopies[2] > 0};
  return (ex[0] && side(t.xb, t.xe, g->n[0], g->overlap[0])) ||
         (ex[1] && side(t.r0, t.re, g->n[1], g->overlap[1])) ||
         (ex[2] && side(t.m0, t.m1, g->n[2], g->overlap[2]));
}

int build_full_tiles(igg_grid *g, int V, TileSet **out) {
  auto it = g->full.find(V);
  if (it != g->full.end()) {
    *out = &it->second;
    return IGG_OK;
  }
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  const long long xy = xy_tiles_of(1, nx - 1, lo_in(ny), hi_in(ny)) * g->nsub;
  const int zb = choose_zb(xy, hi_in(nz) - lo_in(nz));
  TileLists v;
  const bool tma = use_tma(g, V);
  const int Wt = tma ? tma_tile_width(dtype_of_vec(V), TMA_WIDE) : 0;
  const int Ht = tma ? tma_tile_rows(dtype_of_vec(V), TMA_WIDE) : 0;
  const int zbt = tma ? choose_zb_tma(tma_xy_tiles(1, nx - 1, 1, ny - 1, V, Wt, Ht) * g->nsub,
                                      nz - 2, tma_slots(V))
                      : 0;
  if (tma) {
    full_tma_list(g, V, zbt, Wt, Ht, v.tma);
  } else {
    for (int s = 0; s < g->nsub; ++s)
      add_tiles(v, V, (long long)s * g->nloc, nx, ny, 1, nx - 1, lo_in(ny), hi_in(ny), lo_in(nz),
                hi_in(nz), zb, 0);
  }
  zero_absent_strides(g, v.vec);
  TileSet ts;
  if (int rc = upload_tiles(v, V, &ts, tma ? TMA_WIDE : -1)) return rc;
  *out = &g->full.emplace(V, ts).first->second;
  return IGG_OK;
}

// The full step's TMA tiles split into face and inner sets (same tiles, same
// order within each set). Requires use_tma(g, V).
int build_part_tiles(igg_grid *g, int V, PartTiles **out) {
  auto it = g->part.find(V);
  if (it != g->part.end()) {
    *out = &it->second;
    return IGG_OK;
  }
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  const int Wt = tma_tile_width(dtype_of_vec(V), TMA_WIDE);
  const int Ht = tma_tile_rows(dtype_of_vec(V), TMA_WIDE);
  const int zbt = choose_zb_tma(tma_xy_tiles(1, nx - 1, 1, ny - 1, V, Wt, Ht) * g->nsub, nz - 2,
                                tma_slots(V));
  std::vector<TmaTile> all;
  full_tma_list(g, V, zbt, Wt, Ht, all);
  TileLists f, in;
  for (const TmaTile &t : all) (touches_faces(g, t) ? f : in).tma.push_back(t);
  PartTiles pt;
  if (int rc = upload_tiles(f, V, &pt.face, TMA_WIDE)) return rc;
  if (int rc = upload_tiles(in, V, &pt.inner, TMA_WIDE)) {
    free_tiles(pt.face);
    return rc;
  }
  *out = &g->part.emplace(V, pt).first->second;
  return IGG_OK;
}

int build_split_tiles(igg_grid *g, const int w[3], int V, SplitTiles **out) {
  std::array<int, 4> key = {w[0], w[1], w[2], V};
  auto it = g->split.find(key);
  if (it != g->split.end()) {
    *out = &it->second;
    return IGG_OK;
  }
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  // 0-based ranges: boundary-low [1, w-1], inner block [w, n-w-1],
  // boundary-high [n-w, n-2]; clamp so that empty ranges stay empty.
  auto lo_end = [](int wd, int nd) { return std::min(wd, nd - 1); };      // end of low slab
  auto hi_beg = [](int wd, int nd) { return std::max(nd - wd, 1); };      // start of high slab
  const int xl = lo_end(w[0], nx), xh = std::max(hi_beg(w[0], nx), xl);
  const int yl = lo_end(w[1], ny), yh = std::max(hi_beg(w[1], ny), yl);
  const int zl = lo_end(w[2], nz), zh = std::max(hi_beg(w[2], nz), zl);
  TileLists vb, vi;
  // z slabs: all inner x, y; y slabs: z in the inner block range; x slabs:
  // y and z in the inner block ranges. The six boxes are disjoint and their
  // union with the inner block is the set of inner points.
  long long xy_b = 0, xy_i = 0;
  xy_b += 2 * xy_tiles_of(1, nx - 1, 1, ny - 1);
  xy_b += 2 * xy_tiles_of(1, nx - 1, 1, yl) + 2 * xy_tiles_of(1, xl, yl, yh);
  xy_i += xy_tiles_of(xl, xh, yl, yh);
  // boundary slabs are thin: short z sweeps give many tiles that run side by
  // side instead of a few long latency-bound sweeps on the critical path
  const int zb_b = std::min(8, choose_zb(xy_b * g->nsub, zh - zl > 0 ? zh - zl : 1));
  const int zb_i = choose_zb(xy_i * g->nsub, zh - zl > 0 ? zh - zl : 1);
  SplitTiles st;
  int rc = IGG_OK;
  if (use_tma(g, V)) {
    // TMA: z slabs with wide tiles, y slabs with wide tiles marching along y
    // (rows along z). The x slabs are widened to whole wide tiles at both
    // ends of each row (narrow boxes make short TMA rows); the inner-block
    // points inside those tiles are computed there, before the halo update,
    // and the inner-block launch covers the rest. Every point is computed
    // exactly once with the same arithmetic, so the result is unchanged.
    const igg_dtype d = dtype_of_vec(V);
    const int Ww = tma_tile_width(d, TMA_WIDE), Hw = tma_tile_rows(d, TMA_WIDE);
    int xlw = std::min(std::max(xl, (xl + Ww - 1) / Ww * Ww), nx - 1);
    int xhw = std::max(xlw, std::min(xh, std::max(1, ((nx - Ww) / V) * V)));
    TileLists wzx, sy;  // z slabs and x ends (one launch), y slabs
    const int zbt_i = choose_zb_tma(tma_xy_tiles(xlw, xhw, yl, yh, V, Ww, Hw) * g->nsub,
                                    zh - zl > 0 ? zh - zl : 1, tma_slots(V));
    const int zbt_x = choose_zb_tma(
        (tma_xy_tiles(1, xlw, yl, yh, V, Ww, Hw) + tma_xy_tiles(xhw, nx - 1, yl, yh, V, Ww, Hw)) *
            g->nsub,
        zh - zl > 0 ? zh - zl : 1, tma_slots(V));
    for (int s = 0; s < g->nsub; ++s) {
      const long long base = (long long)s * g->nloc, zoff = (long long)s * nz;
      add_box_tma(wzx.tma, base, zoff, 1, xlw, yl, yh, zl, zh, zbt_x, V, Ww, Hw);          // x low
      add_box_tma(wzx.tma, base, zoff, xhw, nx - 1, yl, yh, zl, zh, zbt_x, V, Ww, Hw);     // x high
      add_box_tma(sy.tma, base, zoff, 1, nx - 1, zl, zh, 1, yl, 64, V, Ww, Hw);            // y low
      add_box_tma(sy.tma, base, zoff, 1, nx - 1, zl, zh, yh, ny - 1, 64, V, Ww, Hw);       // y high
      add_box_tma(vi.tma, base, zoff, xlw, xhw, yl, yh, zl, zh, zbt_i, V, Ww, Hw);         // inner
    }
    // the short z-slab tiles after the long x-end tiles in the same launch
    for (int s = 0; s < g->nsub; ++s) {
      const long long base = (long long)s * g->nloc, zoff = (long long)s * nz;
      add_box_tma(wzx.tma, base, zoff, 1, nx - 1, 1, ny - 1, 1, zl, 64, V, Ww, Hw);         // z low
      add_box_tma(wzx.tma, base, zoff, 1, nx - 1, 1, ny - 1, zh, nz - 1, 64, V, Ww, Hw);    // z high
    }
    const std::pair<TileLists *, int> parts[2] = {{&wzx, TMA_WIDE}, {&sy, TMA_WIDE_SWAP}};
    for (auto &pt : parts) {
      if (pt.first->tma.empty()) continue;
      // each kernel variant needs its shared-memory attribute before launch
      cudaError_t e = tma_prepare(d, pt.second, nullptr);
      if (e != cudaSuccess) {
        rc = cuda_error(e, "TMA kernel set-up");
        break;
      }
      TileSet ts;
      if ((rc = upload_tiles(*pt.first, V, &ts, pt.second)) != IGG_OK) break;
      st.boundary.push_back(ts);
    }
    if (rc == IGG_OK) rc = upload_tiles(vi, V, &st.inner, TMA_WIDE);
  } else {
    for (int s = 0; s < g->nsub; ++s) {
      const long long base = (long long)s * g->nloc;
      add_tiles(vb, V, base, nx, ny, 1, nx - 1, 1, ny - 1, 1, zl, 64, 0);          // z low
      add_tiles(vb, V, base, nx, ny, 1, nx - 1, 1, ny - 1, zh, nz - 1, 64, 0);     // z high
      add_tiles(vb, V, base, nx, ny, 1, nx - 1, 1, yl, zl, zh, zb_b, 0);           // y low
      add_tiles(vb, V, base, nx, ny, 1, nx - 1, yh, ny - 1, zl, zh, zb_b, 0);      // y high
      add_tiles(vb, V, base, nx, ny, 1, xl, yl, yh, zl, zh, zb_b, 0);              // x low
      add_tiles(vb, V, base, nx, ny, xh, nx - 1, yl, yh, zl, zh, zb_b, 0);         // x high
      add_tiles(vi, V, base, nx, ny, xl, xh, yl, yh, zl, zh, zb_i, 0);             // inner block
    }
    TileSet tb;
    rc = upload_tiles(vb, V, &tb);
    if (rc == IGG_OK) {
      st.boundary.push_back(tb);
      rc = upload_tiles(vi, V, &st.inner);
    }
  }
  if (rc != IGG_OK) {
    for (auto &b : st.boundary) free_tiles(b);
    free_tiles(st.inner);
    return rc;
  }
  auto res = g->split.emplace(key, st);
  *out = &res.first->second;
  return IGG_OK;
}

cudaError_t launch_tiles(const igg_grid *g, int V, igg_dtype dt, const TileSet &ts, void *T2,
                         const void *T, const void *Ci, const Coef &c, cudaStream_t s) {
  if (ts.tma >= 0)
    return launch_stencil_tma(dt, ts.tma, (const TmaTile *)ts.dev, ts.n, T2, T, Ci, g->n[0],
                              g->n[1], (long long)g->nsub * g->n[2], c, g->dev_err, ts.fix, s);
  if (V > 1) return launch_stencil_vec(dt, (const VTile *)ts.dev, ts.n, T2, T, Ci, c, nullptr, s);
  return launch_stencil(dt, (const Tile *)ts.dev, ts.n, T2, T, Ci, c, nullptr, s);
}

// Plane-copy tables of the halo update of a field of local size nf (the
// grid's own size, or a staggered one), one per dimension. The field's
// overlap is o + (nf - n) (staggered points on a shared face are shared);
// a dimension whose overlap is below 2 exchanges nothing.
int build_halo_tables(const igg_grid *g, const int nf[3], PlaneCopy *copies[3], int ncopies[3]) {
  const long long nloc = (long long)nf[0] * nf[1] * nf[2];
  const long long plane_stride[3] = {1, nf[0], (long long)nf[0] * nf[1]};
  for (int d = 0; d < 3; ++d) {
    std::vector<PlaneCopy> v;
    const int nd = nf[d], o = g->overlap[d] + nf[d] - g->n[d];
    for (int s = 0; s < g->nsub && o >= 2; ++s) {
      const int l = g->left[3 * s + d], r = g->right[3 * s + d];
      if (l >= 0)
        v.push_back({(long long)s * nloc + 0 * plane_stride[d],
                     (long long)l * nloc + (long long)(nd - o) * plane_stride[d]});
      if (r >= 0)
        v.push_back({(long long)s * nloc + (long long)(nd - 1) * plane_stride[d],
                     (long long)r * nloc + (long long)(o - 1) * plane_stride[d]});
    }
    ncopies[d] = (int)v.size();
    copies[d] = nullptr;
    if (v.empty()) continue;
    cudaError_t e = cudaMalloc(&copies[d], v.size() * sizeof(PlaneCopy));
    if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(halo table)");
    e = cudaMemcpy(copies[d], v.data(), v.size() * sizeof(PlaneCopy), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpy(halo table)");
  }
  return IGG_OK;
}

int build_halo_tables(igg_grid *g) { return build_halo_tables(g, g->n, g->copies, g->ncopies); }

// The plane copies of a field of local size nf, dimensions x, y, z in order.
cudaError_t enqueue_halo(PlaneCopy *const copies[3], const int ncopies[3], const int nf[3],
                         void *field, size_t es, cudaStream_t s) {
  const int nx = nf[0], ny = nf[1], nz = nf[2];
  const long long sxy = (long long)nx * ny;
  cudaError_t e = launch_halo(es, copies[0], ncopies[0], field, ny, nz, nx, sxy, s);
  if (e == cudaSuccess) e = launch_halo(es, copies[1], ncopies[1], field, nx, nz, 1, sxy, s);
  if (e == cudaSuccess) e = launch_halo(es, copies[2], ncopies[2], field, nx, ny, 1, nx, s);
  return e;
}

// The transpose of the halo update of a field of the grid's own size (F64
// or F32): the plane copies' transposes, dimensions z, y, x.
cudaError_t enqueue_halo_adjoint(igg_grid *g, void *field, size_t es, cudaStream_t s) {
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  const long long sxy = (long long)nx * ny;
  cudaError_t e = launch_halo_adjoint(es, g->copies[2], g->ncopies[2], field, nx, ny, 1, nx, s);
  if (e == cudaSuccess) e = launch_halo_adjoint(es, g->copies[1], g->ncopies[1], field, nx, nz, 1, sxy, s);
  if (e == cudaSuccess) e = launch_halo_adjoint(es, g->copies[0], g->ncopies[0], field, ny, nz, nx, sxy, s);
  return e;
}

// The halo update of a field of the grid's own size: on 3-D grids one
// gather launch, else the plane copies dimension by dimension.
cudaError_t enqueue_halo(igg_grid *g, void *field, size_t es, cudaStream_t s,
                         bool skipx = false) {
  if (g->n[0] > 1 && g->n[1] > 1 && g->n[2] > 1) {
    HaloGather h;
    h.skipx = skipx ? 1 : 0;
    h.nbr = g->nbr;
    for (int d = 0; d < 3; ++d) {
      h.n[d] = g->n[d];
      h.o[d] = g->overlap[d];
    }
    h.nloc = g->nloc;
    h.nsub = g->nsub;
    return launch_halo_gather(es, field, h, s);
  }
  return enqueue_halo(g->copies, g->ncopies, g->n, field, es, s);
}

// Plane tables for fields of local size nf: the grid's own, or a staggered
// size's (built on first use).
int halo_tables(igg_grid *g, const int nf[3], PlaneCopy *const **copies, const int **ncopies) {
  if (nf[0] == g->n[0] && nf[1] == g->n[1] && nf[2] == g->n[2]) {
    *copies = g->copies;
    *ncopies = g->ncopies;
    return IGG_OK;
  }
  const std::array<int, 3> key = {nf[0], nf[1], nf[2]};
  auto it = g->staggered.find(key);
  if (it == g->staggered.end()) {
    igg_grid::Tables t;
    if (int rc = build_halo_tables(g, nf, t.copies, t.ncopies)) {
      for (int d = 0; d < 3; ++d) cudaFree(t.copies[d]);
      return rc;
    }
    it = g->staggered.emplace(key, t).first;
  }
  *copies = it->second.copies;
  *ncopies = it->second.ncopies;
  return IGG_OK;
}

// Halo update of several fields (field i of local size nf[3i..3i+2]): per
// dimension x, y, z one launch for all fields (chunks of kMaxHaloJobs).
int enqueue_halo_fields(igg_grid *g, void *const fields[], const int *nf, int nfields, size_t es,
                        cudaStream_t s, unsigned dims = 7u) {
  std::vector<PlaneCopy *const *> tc(nfields);
  std::vector<const int *> tn(nfields);
  for (int i = 0; i < nfields; ++i)
    if (int rc = halo_tables(g, nf + 3 * i, &tc[i], &tn[i])) return rc;
  for (int d = 0; d < 3; ++d) {
    if (!(dims >> d & 1u)) continue;
    HaloJobs jobs;
    int nj = 0;
    for (int i = 0; i <= nfields; ++i) {
      if (nj == kMaxHaloJobs || (i == nfields && nj > 0)) {
        cudaError_t e = launch_halo_jobs(es, jobs, nj, s);
        if (e != cudaSuccess) return cuda_error(e, "halo launch");
        nj = 0;
      }
      if (i == nfields) break;
      if (tn[i][d] == 0) continue;
      const int *n = nf + 3 * i;
      const long long sxy = (long long)n[0] * n[1];
      HaloJob &j = jobs.j[nj++];
      j.copies = tc[i][d];
      j.ncopies = tn[i][d];
      j.field = fields[i];
      j.na = d == 0 ? n[1] : n[0];
      j.nb = d == 2 ? n[1] : n[2];
      j.sa = d == 0 ? n[0] : 1;
      j.sb = d == 2 ? n[0] : sxy;
      j.vec = 0;
    }
  }
  return IGG_OK;
}

bool any_halo(const igg_grid *g) { return g->ncopies[0] + g->ncopies[1] + g->ncopies[2] > 0; }

// Whether hidden steps run as the full step launch followed by the halo
// update (the option; the alternative is the boundary/inner split).
bool use_fused_halo(const igg_grid *g) { return g->fused_halo; }

// Whether a step with its halo update runs the full step's TMA tiles as face
// and inner sets with the halo update beside the inner set (3-D grids on
// the TMA kernel, with the grid's option).
bool hide_applies(const igg_grid *g, int V, bool with_halo) {
  return with_halo && g->hide_halo && use_fused_halo(g) && !low_dim(g) && use_tma(g, V) &&
         any_halo(g);
}

// NVTX range over a host scope: the enqueue of one phase of the step (the
// profiler places the GPU work it launches beneath it).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

// Event k of the current step's phase triple when phase timing is on and s
// is not being captured into a graph (nullptr otherwise); the triples are
// made on demand, at most kMaxPhaseSteps steps between two queries.
constexpr int kMaxPhaseSteps = 4096;
cudaEvent_t phase_event(igg_grid *g, cudaStream_t s, int k) {
  if (!g->phase_times) return nullptr;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
    return nullptr;
  if (k == 0 && g->pev_used >= 3 * kMaxPhaseSteps) return nullptr;
  const int i = k == 0 ? g->pev_used : g->pev_used - 3 + k;
  if (i < 0) return nullptr;
  while ((int)g->pev.size() <= i) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    g->pev.push_back(e);
  }
  if (k == 0) g->pev_used += 3;
  return g->pev[i];
}

// One step of Fig. 1's loop, queued on s: plain (full step, then halo update
// of T2 on s) or hidden (boundary set + halo on the high-priority stream,
// inner block on the low-priority stream, s joins both).
int enqueue_step(igg_grid *g, const int *widths, void *T2, const void *T, const void *Ci,
                 igg_dtype dt, const Coef &c0, bool with_halo, cudaStream_t s) {
  cudaError_t e;
  Coef c = c0;
  c.f64_emu = g->f64_emu && emu_weights_ok(c);
  const int V = grid_vec(g, dt);
  // 2-D and 1-D grids: the hidden step runs as the plain step and the halo
  // update (same result; no boundary/inner split of an absent dimension);
  // by default (the grid's option) every hidden step does: with all
  // subdomains in one device's memory there is no transfer to overlap, and
  // the full step launch followed by the one-launch halo update is faster
  // than the split's extra launches
  if (low_dim(g) || use_fused_halo(g)) widths = nullptr;
  NvtxRange step_range(with_halo ? "igg step + halo" : "igg step");
  cudaEvent_t p0 = phase_event(g, s, 0);
  if (p0 && (e = cudaEventRecord(p0, s)) != cudaSuccess) return cuda_error(e, "record");
  if (!widths && hide_applies(g, V, with_halo)) {
    // face tiles, then the halo update, on the high-priority stream; the
    // inner tiles (which neither read halo cells nor compute sent points)
    // beside them on the low-priority stream; s joins both
    PartTiles *pt = nullptr;
    if (int rc = build_part_tiles(g, V, &pt)) return rc;
    c.ends = 1;
    if ((e = cudaEventRecord(g->ev_fork, s)) != cudaSuccess) return cuda_error(e, "record");
    if ((e = cudaStreamWaitEvent(g->hi, g->ev_fork, 0)) != cudaSuccess) return cuda_error(e, "wait");
    if ((e = cudaStreamWaitEvent(g->lo, g->ev_fork, 0)) != cudaSuccess) return cuda_error(e, "wait");
    {
      NvtxRange r("face tiles (high priority)");
      if (pt->face.n > 0 && (e = launch_tiles(g, V, dt, pt->face, T2, T, Ci, c, g->hi)) != cudaSuccess)
        return cuda_error(e, "face tiles launch");
    }
    cudaEvent_t pf = p0 ? g->ev_face : nullptr;
    if (pf && (e = cudaEventRecord(pf, g->hi)) != cudaSuccess) return cuda_error(e, "record");
    {
      NvtxRange r("inner tiles (low priority)");
      if (pt->inner.n > 0 && (e = launch_tiles(g, V, dt, pt->inner, T2, T, Ci, c, g->lo)) != cudaSuccess)
        return cuda_error(e, "inner tiles launch");
    }
    {
      NvtxRange r("halo update (high priority)");
      if ((e = enqueue_halo(g, T2, dtype_size(dt), g->hi)) != cudaSuccess)
        return cuda_error(e, "halo launch");
    }
    if ((e = cudaEventRecord(g->ev_hi, g->hi)) != cudaSuccess) return cuda_error(e, "record");
    if ((e = cudaEventRecord(g->ev_lo, g->lo)) != cudaSuccess) return cuda_error(e, "record");
    if (pf) {  // phase events: the end of both tile sets, then the end of the step
      if ((e = cudaStreamWaitEvent(s, pf, 0)) != cudaSuccess) return cuda_error(e, "wait");
      if ((e = cudaStreamWaitEvent(s, g->ev_lo, 0)) != cudaSuccess) return cuda_error(e, "wait");
      if (cudaEvent_t p1 = phase_event(g, s, 1))
        if ((e = cudaEventRecord(p1, s)) != cudaSuccess) return cuda_error(e, "record");
    }
    if ((e = cudaStreamWaitEvent(s, g->ev_hi, 0)) != cudaSuccess) return cuda_error(e, "wait");
    if ((e = cudaStreamWaitEvent(s, g->ev_lo, 0)) != cudaSuccess) return cuda_error(e, "wait");
    if (cudaEvent_t p2 = p0 ? phase_event(g, s, 2) : nullptr)
      if ((e = cudaEventRecord(p2, s)) != cudaSuccess) return cuda_error(e, "record");
    return IGG_OK;
  }
  if (!widths) {
    TileSet *full = nullptr;
    if (int rc = build_full_tiles(g, V, &full)) return rc;
    c.ends = with_halo && any_halo(g) ? 1 : 0;
    {
      NvtxRange r("stencil");
      e = launch_tiles(g, V, dt, *full, T2, T, Ci, c, s);
    }
    if (e != cudaSuccess) return cuda_error(e, "stencil launch");
    if (cudaEvent_t p1 = p0 ? phase_event(g, s, 1) : nullptr)
      if ((e = cudaEventRecord(p1, s)) != cudaSuccess) return cuda_error(e, "record");
    if (with_halo && any_halo(g)) {
      NvtxRange r("halo update");
      e = enqueue_halo(g, T2, dtype_size(dt), s);
      if (e != cudaSuccess) return cuda_error(e, "halo launch");
    }
    if (cudaEvent_t p2 = p0 ? phase_event(g, s, 2) : nullptr)
      if ((e = cudaEventRecord(p2, s)) != cudaSuccess) return cuda_error(e, "record");
    return IGG_OK;
  }
  SplitTiles *st = nullptr;
  int rc = build_split_tiles(g, widths, V, &st);
  if (rc != IGG_OK) return rc;
  if ((e = cudaEventRecord(g->ev_fork, s)) != cudaSuccess) return cuda_error(e, "cudaEventRecord");
  if ((e = cudaStreamWaitEvent(g->hi, g->ev_fork, 0)) != cudaSuccess) return cuda_error(e, "wait");
  if ((e = cudaStreamWaitEvent(g->lo, g->ev_fork, 0)) != cudaSuccess) return cuda_error(e, "wait");
  e = cudaSuccess;
  {
    NvtxRange r("boundary slabs + halo update (high priority)");
    for (const TileSet &b : st->boundary)
      if (e == cudaSuccess) e = launch_tiles(g, V, dt, b, T2, T, Ci, c, g->hi);
    if (e == cudaSuccess && with_halo && any_halo(g))
      e = enqueue_halo(g, T2, dtype_size(dt), g->hi);
  }
  if (e != cudaSuccess) return cuda_error(e, "boundary/halo launch");
  {
    NvtxRange r("inner block (low priority)");
    e = launch_tiles(g, V, dt, st->inner, T2, T, Ci, c, g->lo);
  }
  if (e != cudaSuccess) return cuda_error(e, "inner launch");
  if ((e = cudaEventRecord(g->ev_hi, g->hi)) != cudaSuccess) return cuda_error(e, "record");
  if (cudaEvent_t p1 = p0 ? phase_event(g, s, 1) : nullptr)
    if ((e = cudaEventRecord(p1, g->hi)) != cudaSuccess) return cuda_error(e, "record");
  if ((e = cudaEventRecord(g->ev_lo, g->lo)) != cudaSuccess) return cuda_error(e, "record");
  if ((e = cudaStreamWaitEvent(s, g->ev_hi, 0)) != cudaSuccess) return cuda_error(e, "wait");
  if ((e = cudaStreamWaitEvent(s, g->ev_lo, 0)) != cudaSuccess) return cuda_error(e, "wait");
  if (cudaEvent_t p2 = p0 ? phase_event(g, s, 2) : nullptr)
    if ((e = cudaEventRecord(p2, s)) != cudaSuccess) return cuda_error(e, "record");
  return IGG_OK;
}

int check_widths(const igg_grid *g, const int *w) {
  if (!w) return IGG_OK;
  for (int d = 0; d < 3; ++d) {
    if (g->n[d] == 1) continue;  // absent dimension
    if (w[d] < g->overlap[d])
      return set_error(IGG_EINVAL, "widths[%d]=%d is smaller than overlap %d", d, w[d],
                       g->overlap[d]);
  }
  return IGG_OK;
}

void destroy_grid(igg_grid *g) {
  if (!g) return;
  for (auto &kv : g->graphs) cudaGraphExecDestroy(kv.second);
  for (auto &kv : g->split) {
    for (auto &b : kv.second.boundary) free_tiles(b);
    free_tiles(kv.second.inner);
  }
  for (auto &kv : g->full) free_tiles(kv.second);
  for (auto &kv : g->part) {
    free_tiles(kv.second.face);
    free_tiles(kv.second.inner);
  }
  for (int d = 0; d < 3; ++d) cudaFree(g->copies[d]);
  for (auto &kv : g->staggered)
    for (int d = 0; d < 3; ++d) cudaFree(kv.second.copies[d]);
  cudaFree(g->dev_err);
  cudaFree(g->nbr);
  for (cudaEvent_t e : g->pev) cudaEventDestroy(e);
  if (g->ev_fork) cudaEventDestroy(g->ev_fork);
  if (g->ev_face) cudaEventDestroy(g->ev_face);
  if (g->ev_hi) cudaEventDestroy(g->ev_hi);
  if (g->ev_lo) cudaEventDestroy(g->ev_lo);
  if (g->hi) cudaStreamDestroy(g->hi);
  if (g->lo) cudaStreamDestroy(g->lo);
  if (g->cap) cudaStreamDestroy(g->cap);
  delete g;
}

// most partial sums of igg_reduce (blocks of its first kernel)
constexpr int kMaxRedBlocks = 1024;

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char *igg_last_error(void) { return g_err.c_str(); }

int igg_abi_version(void) { return IGG_ABI_VERSION; }

int igg_init_global_grid(int nx, int ny, int nz, const int dims_in[3], int nsub,
                         const int overlap[3], const int periods[3], igg_grid **out) {
  clear_error();
  if (!out) return set_error(IGG_EINVAL, "out is NULL");
  *out = nullptr;
  const int n[3] = {nx, ny, nz};
  int dims[3] = {0, 0, 0}, o[3] = {2, 2, 2}, per[3] = {0, 0, 0};
  if (dims_in) std::memcpy(dims, dims_in, sizeof dims);
  if (overlap) std::memcpy(o, overlap, sizeof o);
  if (periods)
    for (int d = 0; d < 3; ++d) per[d] = periods[d] ? 1 : 0;
  for (int d = 0; d < 3; ++d) {
    if (n[d] == 1 && d > 0) {
      // an absent dimension (2-D and 1-D grids): one subdomain, not periodic
      if (dims[d] > 1) return set_error(IGG_EINVAL, "dims[%d]=%d for a dimension of size 1", d, dims[d]);
      if (per[d]) return set_error(IGG_EINVAL, "a dimension of size 1 cannot be periodic");
      dims[d] = 1;
      continue;
    }
    if (n[d] < 3) return set_error(IGG_EINVAL, "local size n[%d]=%d < 3", d, n[d]);
    if (o[d] < 2 || o[d] > n[d] - 1)
      return set_error(IGG_EINVAL, "overlap[%d]=%d outside [2, n-1]", d, o[d]);
  }
  bool has_free = dims[0] == 0 || dims[1] == 0 || dims[2] == 0;
  if (has_free) {
    if (!dims_create(nsub, dims))
      return set_error(IGG_EINVAL, "cannot factor nsub=%d over dims (%d,%d,%d)", nsub,
                       dims_in ? dims_in[0] : 0, dims_in ? dims_in[1] : 0,
                       dims_in ? dims_in[2] : 0);
  } else {
    for (int d = 0; d < 3; ++d)
      if (dims[d] < 0) return set_error(IGG_EINVAL, "negative dims");
    if (nsub > 0 && nsub != dims[0] * dims[1] * dims[2])
      return set_error(IGG_EINVAL, "dims product %d differs from nsub %d",
                       dims[0] * dims[1] * dims[2], nsub);
  }
  const long long nloc = (long long)nx * ny * nz;
  if (nloc > (1LL << 40)) return set_error(IGG_EINVAL, "local array too large");

  igg_grid *g = new (std::nothrow) igg_grid();
  if (!g) return set_error(IGG_ENOMEM, "host allocation failed");
  for (int d = 0; d < 3; ++d) {
    g->n[d] = n[d];
    g->dims[d] = dims[d];
    g->overlap[d] = o[d];
    g->periods[d] = per[d];
    g->ng[d] = n[d] == 1 ? 1 : dims[d] * (n[d] - o[d]) + (per[d] ? 0 : o[d]);
  }
  g->nsub = dims[0] * dims[1] * dims[2];
  g->nloc = nloc;
  cudaError_t e = cudaGetDevice(&g->device);
  if (e != cudaSuccess) {
    destroy_grid(g);
    return cuda_error(e, "cudaGetDevice");
  }
  // topology: coordinates x fastest; neighbours wrap in periodic dimensions
  g->left.assign(3 * g->nsub, -1);
  g->right.assign(3 * g->nsub, -1);
  for (int s = 0; s < g->nsub; ++s) {
    const int c[3] = {s % dims[0], (s / dims[0]) % dims[1], s / (dims[0] * dims[1])};
    for (int d = 0; d < 3; ++d) {
      for (int side = 0; side < 2; ++side) {
        int cc[3] = {c[0], c[1], c[2]};
        cc[d] += side == 0 ? -1 : 1;
        if (cc[d] < 0 || cc[d] >= dims[d]) {
          if (!per[d]) continue;
          cc[d] = (cc[d] + dims[d]) % dims[d];
        }
        const int nb = cc[0] + dims[0] * (cc[1] + dims[1] * cc[2]);
        (side == 0 ? g->left : g->right)[3 * s + d] = nb;
      }
    }
  }
  int lo_prio = 0, hi_prio = 0;
  e = cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&g->hi, cudaStreamNonBlocking, hi_prio);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&g->lo, cudaStreamNonBlocking, lo_prio);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_hi, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_lo, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_face, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    destroy_grid(g);
    return cuda_error(e, "stream/event creation");
  }
  e = cudaMalloc(&g->dev_err, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(g->dev_err, 0, sizeof(unsigned));
  if (e != cudaSuccess) {
    destroy_grid(g);
    return cuda_error(e, "device error word");
  }
  int rc = build_halo_tables(g);
  if (rc == IGG_OK) {
    std::vector<int> nb(6 * (size_t)g->nsub);
    for (int q = 0; q < g->nsub; ++q)
      for (int d = 0; d < 3; ++d) {
        nb[6 * q + 2 * d] = g->left[3 * q + d];
        nb[6 * q + 2 * d + 1] = g->right[3 * q + d];
      }
    e = cudaMalloc(&g->nbr, nb.size() * sizeof(int));
    if (e == cudaSuccess)
      e = cudaMemcpy(g->nbr, nb.data(), nb.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) rc = cuda_error(e, "neighbour table");
  }
  if (rc != IGG_OK) {
    destroy_grid(g);
    return rc;
  }
  *out = g;
  return IGG_OK;
}

int igg_finalize_global_grid(igg_grid *g) {
  clear_error();
  if (!g) return IGG_OK;
  DeviceGuard dg(g->device);
  cudaError_t e1 = cudaStreamSynchronize(g->hi);
  cudaError_t e2 = cudaStreamSynchronize(g->lo);
  destroy_grid(g);
  if (e1 != cudaSuccess) return cuda_error(e1, "finalize: high-priority stream");
  if (e2 != cudaSuccess) return cuda_error(e2, "finalize: low-priority stream");
  return IGG_OK;
}

int igg_global_size(const igg_grid *g, int n_g[3]) {
  clear_error();
  if (int rc = check_grid(g)) return rc;
  if (!n_g) return set_error(IGG_EINVAL, "n_g is NULL");
  for (int d = 0; d < 3; ++d) n_g[d] = g->ng[d];
  return IGG_OK;
}

int igg_grid_shape(const igg_grid *g, int n[3], int dims[3], int overlap[3], int periods[3],
                   int *nsub) {
  clear_error();
  if (int rc = check_grid(g)) return rc;
  for (int d = 0; d < 3; ++d) {
    if (n) n[d] = g->n[d];
    if (dims) dims[d] = g->dims[d];
    if (overlap) overlap[d] = g->overlap[d];
    if (periods) periods[d] = g->periods[d];
  }
  if (nsub) *nsub = g->nsub;
  return IGG_OK;
}

int igg_subdomain_info(const igg_grid *g, int sub, int coords[3], int left[3], int right[3],
                       int offset[3]) {
  clear_error();
  if (int rc = check_grid(g)) return rc;
  if (sub < 0 || sub >= g->nsub) return set_error(IGG_EINVAL, "sub %d out of range", sub);
  const int c[3] = {sub % g->dims[0], (sub / g->dims[0]) % g->dims[1],
                    sub / (g->dims[0] * g->dims[1])};
  for (int d = 0; d < 3; ++d) {
    if (coords) coords[d] = c[d];
    if (left) left[d] = g->left[3 * sub + d];
    if (right) right[d] = g->right[3 * sub + d];
    if (offset) offset[d] = c[d] * (g->n[d] - g->overlap[d]);
  }
  return IGG_OK;
}

int igg_update_halo(igg_grid *g, void *const fields[], int nfields, igg_dtype dt,
                    void *stream) {
  clear_error();
  if (int rc = check_grid(g)) return rc;
  if (int rc = check_dtype(dt)) return rc;
  if (nfields < 0 || (nfields > 0 && !fields)) return set_error(IGG_EINVAL, "bad field list");
  for (int i = 0; i < nfields; ++i)
    if (int rc = check_field(g, fields[i], "field")) return rc;
  DeviceGuard dg(g->device);
  if (g->n[0] > 1 && g->n[1] > 1 && g->n[2] > 1) {  // 3-D: one gather launch per field
    if (!any_halo(g)) return IGG_OK;
    for (int i = 0; i < nfields; ++i) {
      cudaError_t e = enqueue_halo(g, fields[i], dtype_size(dt), (cudaStream_t)stream);
      if (e != cudaSuccess) return cuda_error(e, "halo launch");
    }
    return IGG_OK;
  }
  std::vector<int> nf(3 * (size_t)nfields);
  for (int i = 0; i < nfields; ++i)
    for (int d = 0; d < 3; ++d) nf[3 * i + d] = g->n[d];
  return enqueue_halo_fields(g, fields, nf.data(), nfields, dtype_size(dt), (cudaStream_t)stream);
}

int igg_update_halo_staggered(igg_grid *g, void *const fields[], int nfields, igg_dtype dt,
                              const int nf[3], void *stream) {
  clear_error();
  if (int rc = check_grid(g)) return rc;
  if (int rc = check_dtype(dt)) return rc;
  if (!nf) return set_error(IGG_EINVAL, "nf is NULL");
  for (int d = 0; d < 3; ++d) {
    if (nf[d] < g->n[d] - 1 || nf[d] > g->n[d] + 1)
      return set_error(IGG_EINVAL, "nf[%d]=%d differs from n[%d]=%d by more than one", d, nf[d], d,
                       g->n[d]);
    if (nf[d] < 3) return set_error(IGG_EINVAL, "nf[%d]=%d < 3", d, nf[d]);
  }
  if (nfields < 0 || (nfields > 0 && !fields)) return set_error(IGG_EINVAL, "bad field list");
  for (int i = 0; i < nfields; ++i)
    if (int rc = check_field(g, fields[i], "field")) return rc;
  DeviceGuard dg(g->device);
  std::vector<int> nfs(3 * (size_t)nfields);
  for (int i = 0; i < nfields; ++i)
    for (int d = 0; d < 3; ++d) nfs[3 * i + d] = nf[d];
  return enqueue_halo_fields(g, fields, nfs.data(), nfields, dtype_size(dt), (cudaStream_t)stream);
}

int igg_update_halo_fields(igg_grid *g, void *const fields[], const int *sizes, int nfields,
                           igg_dtype dt, void *stream) {
  clear_error();
  if (int rc = check_grid(g)) return rc;
  if (int rc = check_dtype(dt)) return rc;
  if (nfields < 0 || (nfields > 0 && (!fields || !sizes)))
    return set_error(IGG_EINVAL, "bad field list");
  for (int i = 0; i < nfields; ++i) {
    for (int d = 0; d < 3; ++d) {
      const int v = sizes[3 * i + d];
      if (v < g->n[d] - 1 || v > g->n[d] + 1 || v < 3)
        return set_error(IGG_EINVAL, "field %d: size %d in dimension %d not within one of %d (or < 3)",
                         i, v, d, g->n[d]);
    }
    if (int rc = check_field(g, fields[i], "field")) return rc;
  }
  DeviceGuard dg(g->device);
  return enqueue_halo_fields(g, fields, sizes, nfields, dtype_size(dt), (cudaStream_t)stream);
}

int igg_gp_step(igg_grid *g, void *u, void *v, const void *V, igg_dtype dt, double gnl,
                double dtime, double dx, double dy, double dz, int with_halo, void *stream) {
  clear_error();
  if (int rc = check_grid(g)) return rc;
  if (dt != IGG_F64 && dt != IGG_F32) return set_error(IGG_EINVAL, "Gross-Pitaevskii: F64 or F32 only");
  for (const void *f : {(const void *)u, (const void *)v, V})
    if (int rc = check_field(g, f, "field")) return rc;
  if (u == v) return set_error(IGG_EINVAL, "u aliases v");
  if (!(dx > 0) || !(dy > 0) || !(dz > 0) || !(dtime == dtime) || !(gnl == gnl))
    return set_error(IGG_EINVAL, "Gross-Pitaevskii: spacings must be positive, dt and g numbers");
  DeviceGuard dg(g->device);
  GpCoef c;
  c.kx = -dtime / (2.0 * dx * dx);
  c.ky = -dtime / (2.0 * dy * dy);
  c.kz = -dtime / (2.0 * dz * dz);
  c.kc = -2.0 * (c.kx + c.ky + c.kz);
  c.dt = dtime;
  c.g = gnl;
  // with the halo update on a 3-D grid, the TMA half-step launch stores its
  // sent x planes into the neighbours' halo columns itself, and the halo
  // launch copies the face rows only
  c.nbr = g->nbr;
  c.ox = g->overlap[0];
  c.xsend = with_halo && any_halo(g) && !low_dim(g) ? 1 : 0;
  cudaStream_t s = (cudaStream_t)stream;
  for (int which = 0; which < 2; ++which) {
    bool xsent = false;
    cudaError_t e = launch_gp_half(dt, which, g->nsub, g->n[0], g->n[1], g->n[2], u, v, V, c,
                                   g->tma_enabled && !low_dim(g), g->dev_err, s, &xsent);
    if (e != cudaSuccess) return cuda_error(e, "Gross-Pitaevskii launch");
    if (with_halo && any_halo(g)) {
      e = enqueue_halo(g, which == 0 ? u : v, dtype_size(dt), s, xsent);
      if (e != cudaSuccess) return cuda_error(e, "halo launch");
    }
  }
  return IGG_OK;
}

int igg_acoustic_step(igg_grid *g, void *P, void *Vx, void *Vy, void *Vz, igg_dtype dt,
                      double rho, double K, double dtime, double dx, double dy, double dz,
                      int with_halo, void *stream) {
  clear_error();
  if (int rc = check_grid(g)) return rc;
  if (dt != IGG_F64 && dt != IGG_F32) return set_error(IGG_EINVAL, "acoustics: F64 or F32 only");
  if (low_dim(g)) return set_error(IGG_EINVAL, "acoustics: needs a 3-D grid");
  for (void *f : {P, Vx, Vy, Vz})
    if (int rc = check_field(g, f, "field")) return rc;
  if (!(rho > 0) || !(K > 0) || !(dx > 0) || !(dy > 0) || !(dz > 0) || !(dtime == dtime))
    return set_error(IGG_EINVAL, "acoustics: rho, K and spacings must be positive, dt a number");
  DeviceGuard dg(g->device);
  AcCoef c;
  c.ax = dtime / rho / dx;
  c.ay = dtime / rho / dy;
  c.az = dtime / rho / dz;
  c.bx = dtime * K / dx;
  c.by = dtime * K / dy;
  c.bz = dtime * K / dz;
  // with the halo update, the two launches do its x exchange themselves
  // (the x-face planes, which are strided), the y and z exchanges follow
  c.nbr = g->nbr;
  c.ox = g->overlap[0];
  c.xsend = with_halo ? 1 : 0;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = launch_acoustic(dt, g->nsub, g->n[0], g->n[1], g->n[2], P, Vx, Vy, Vz, c, s);
  if (e != cudaSuccess) return cuda_error(e, "acoustic launch");
  if (!with_halo) return IGG_OK;
  void *const fields[4] = {P, Vx, Vy, Vz};
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  const int sizes[12] = {nx, ny, nz, nx + 1, ny, nz, nx, ny + 1, nz, nx, ny, nz + 1};
  return enqueue_halo_fields(g, fields, sizes, 4, dtype_size(dt), s, 6u);
}

int igg_step(igg_grid *g, void *T2, const void *T, const void *Ci, igg_dtype dt, double lam,
             double dtime, double dx, double dy, double dz, void *stream) {
  clear_error();
  if (int rc = check_grid(g)) return rc;
  if (int rc = check_dtype(dt)) return rc;
  if (int rc = check_field(g, T2, "T2")) return rc;
  if (int rc = check_field(g, T, "T")) return rc;
  if (int rc = check_field(g, Ci, "Ci")) return rc;
  if (T2 == T || T2 == Ci) return set_error(IGG_EINVAL, "T2 aliases T or Ci");
  if (int rc = check_coef(lam, dtime, dx, dy, dz)) return rc;
  DeviceGuard dg(g->device);
  return enqueue_step(g, nullptr, T2, T, Ci, dt, make_coef(lam, dtime, dx, dy, dz), false,
                      (cudaStream_t)stream);
}

int igg_step_hidden(igg_grid *g, const int widths[3], void *T2, const void *T, const void *Ci,
                    igg_dtype dt, double lam, double dtime, double dx, double dy, double dz,
                    void *stream) {
  clear_error();
  if (int rc = check_grid(g)) return rc;
  if (!widths) return set_error(IGG_EINVAL, "widths is NULL");
  if (int rc = check_widths(g, widths)) return rc;
  if (int rc = check_dtype(dt)) return rc;
  if (int rc = check_field(g, T2, "T2")) return rc;
  if (int rc = check_field(g, T, "T")) return rc;
  if (int rc = check_field(g, Ci, "Ci")) return rc;
  if (T2 == T || T2 == Ci) return set_error(IGG_EINVAL, "T2 aliases T or Ci");
  if (int rc = check_coef(lam, dtime, dx, dy, dz)) return rc;
  DeviceGuard dg(g->device);
  return enqueue_step(g, widths, T2, T, Ci, dt, make_coef(lam, dtime, dx, dy, dz), true,
                      (cudaStream_t)stream);
}

int igg_run(igg_grid *g, int nt, const int widths[3], void *T, void *T2, const void *Ci,
            igg_dtype dt, double lam, double dtime, double dx, double dy, double dz,
            void *stream) {
  clear_error();
  if (int rc = check_grid(g)) return rc;
  if (nt < 0) return set_error(IGG_EINVAL, "nt < 0");
  if (int rc = check_widths(g, widths)) return rc;
  if (int rc = check_dtype(dt)) return rc;
  if (int rc = check_field(g, T2, "T2")) return rc;
  if (int rc = check_field(g, T, "T")) return rc;
  if (int rc = check_field(g, Ci, "Ci")) return rc;
  if (T2 == T || T2 == Ci || T == Ci) return set_error(IGG_EINVAL, "T, T2, Ci alias");
  if (int rc = check_coef(lam, dtime, dx, dy, dz)) return rc;
  DeviceGuard dg(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  const Coef c = make_coef(lam, dtime, dx, dy, dz);
  if (nt == 0) return IGG_OK;
  cudaGraphExec_t exec = nullptr;
  if (nt >= 2) {
    // tile tables are allocated before the capture starts
    const int V = grid_vec(g, dt);
    if (widths && !use_fused_halo(g) && !low_dim(g)) {
      SplitTiles *st = nullptr;
      if (int rc = build_split_tiles(g, widths, V, &st)) return rc;
    } else if (hide_applies(g, V, true)) {
      PartTiles *pt = nullptr;
      if (int rc = build_part_tiles(g, V, &pt)) return rc;
    } else {
      TileSet *full = nullptr;
      if (int rc = build_full_tiles(g, V, &full)) return rc;
    }
    const GraphKey key(T, T2, Ci, (int)dt, widths ? 1 : 0, widths ? widths[0] : 0,
                       widths ? widths[1] : 0, widths ? widths[2] : 0, c.wx, c.wy, c.wz, c.wc);
    auto it = g->graphs.find(key);
    if (it != g->graphs.end()) {
      exec = it->second;
    } else {
      cudaError_t e = cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_error(e, "cudaStreamBeginCapture");
      int rc = enqueue_step(g, widths, T2, T, Ci, dt, c, true, g->cap);
      if (rc == IGG_OK) rc = enqueue_step(g, widths, T, T2, Ci, dt, c, true, g->cap);
      cudaGraph_t graph = nullptr;
      e = cudaStreamEndCapture(g->cap, &graph);
      if (rc != IGG_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
      }
      if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
      e = cudaGraphInstantiateWithFlags(&exec, graph, cudaGraphInstantiateFlagUseNodePriority);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_error(e, "cudaGraphInstantiate");
      if (g->graphs.size() >= 16) {  // bounded cache
        cudaGraphExecDestroy(g->graphs.begin()->second);
        g->graphs.erase(g->graphs.begin());
      }
      g->graphs.emplace(key, exec);
    }
    NvtxRange r("igg_run graph launches (two steps each)");
    for (int i = 0; i < nt / 2; ++i) {
      cudaError_t e = cudaGraphLaunch(exec, s);
      if (e != cudaSuccess) return cuda_error(e, "cudaGraphLaunch");
    }
  }
  if (nt % 2) return enqueue_step(g, widths, T2, T, Ci, dt, c, true, s);
  return IGG_OK;
}

int igg_run_host(igg_grid *g, int nt, const int widths[3], void *T_host, const void *Ci_host,
                 void *T, void *T2, void *Ci, igg_dtype dt, double lam, double dtime, double dx,
                 double dy, double dz, void *stream) {
  clear_error();
  if (int rc = check_grid(g)) return rc;
  if (!T_host || !Ci_host) return set_error(IGG_EINVAL, "T_host or Ci_host is NULL");
  if (int rc = check_dtype(dt)) return rc;
  if (nt < 0) return set_error(IGG_EINVAL, "nt < 0");
  if (int rc = check_field(g, T, "T")) return rc;
  if (int rc = check_field(g, T2, "T2")) return rc;
  if (int rc = check_field(g, Ci, "Ci")) return rc;
  if (T2 == T || T2 == Ci || T == Ci) return set_error(IGG_EINVAL, "T, T2, Ci alias");
  DeviceGuard dg(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)g->nsub * (size_t)g->nloc * dtype_size(dt);
  cudaError_t e;
  {
    NvtxRange r("igg_run_host inputs (H2D, T2 = T)");
    e = cudaMemcpyAsync(T, T_host, bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(Ci, Ci_host, bytes, cudaMemcpyHostToDevice, s);
    // Fig. 1: T2 = copy(T) (the boundary values stay fixed in both buffers)
    if (e == cudaSuccess) e = cudaMemcpyAsync(T2, T, bytes, cudaMemcpyDeviceToDevice, s);
  }
  if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyAsync(inputs)");
  if (int rc = igg_run(g, nt, widths, T, T2, Ci, dt, lam, dtime, dx, dy, dz, stream)) return rc;
  NvtxRange r("igg_run_host result (D2H)");
  e = cudaMemcpyAsync(T_host, nt % 2 ? T2 : T, bytes, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyAsync(result)");
  return IGG_OK;
}

int igg_reduce(int op, const void *a, const void *b, size_t n, igg_dtype dt, double *out_dev,
               void *stream) {
  clear_error();
  if (op < IGG_RED_MAX || op > IGG_RED_SUM_SQDIFF) return set_error(IGG_EINVAL, "bad op %d", op);
  if (int rc = check_dtype(dt)) return rc;
  if (n > 0 && !a) return set_error(IGG_EINVAL, "a is NULL");
  if (n > 0 && (op == IGG_RED_SUM_DIV || op == IGG_RED_SUM_SQDIFF) && !b)
    return set_error(IGG_EINVAL, "b is NULL");
  if (!out_dev) return set_error(IGG_EINVAL, "out_dev is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  long long nb = (long long)((n + 255) / 256);
  if (nb < 1) nb = 1;
  if (nb > kMaxRedBlocks) nb = kMaxRedBlocks;
  // per-call scratch from the stream-ordered allocator: calls on different
  // streams never share it
  double *scratch = nullptr;
  cudaError_t e = cudaMallocAsync((void **)&scratch, (size_t)nb * sizeof(double), s);
  if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync(reduce scratch)");
  e = launch_reduce(op, a, b, n, dt, scratch, (int)nb, out_dev, s);
  cudaError_t ef = cudaFreeAsync(scratch, s);
  if (e != cudaSuccess) return cuda_error(e, "reduce launch");
  if (ef != cudaSuccess) return cuda_error(ef, "cudaFreeAsync(reduce scratch)");
  return IGG_OK;
}


// ---------------------------------------------------------------------------
// Adjoint (differentiated Fig. 1 loop) on a single-subdomain, non-periodic
// grid; drivers with checkpoints every `every` steps.
// ---------------------------------------------------------------------------
static int check_adjoint_grid(const igg_grid *g, igg_dtype dt) {
  if (low_dim(g)) return set_error(IGG_EINVAL, "the adjoint needs a 3-D grid");
  if (dt != IGG_F64 && dt != IGG_F32) return set_error(IGG_EINVAL, "adjoint dtype must be F64 or F32");
  return IGG_OK;
}

// The transposed step S^T on every subdomain (one launch each); the
// subdomains' fields are consecutive blocks of nloc points.
static cudaError_t adjoint_subdomains(igg_grid *g, igg_dtype dt, void *lam_out,
                                      const void *lam_in, const void *Tn, const void *Ci,
                                      double *gCi, const Coef &c, cudaStream_t s,
                                      const void *ci_pairs) {
  const size_t bytes = (size_t)g->nloc * dtype_size(dt);
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < g->nsub && e == cudaSuccess; ++k) {
    const size_t o = (size_t)k * bytes;
    e = launch_adjoint(dt, g->n[0], g->n[1], g->n[2], (char *)lam_out + o,
                       (const char *)lam_in + o, (const char *)Tn + o, (const char *)Ci + o,
                       gCi + (size_t)k * g->nloc, c, g->tma_enabled, g->dev_err, s,
                       ci_pairs ? (const char *)ci_pairs + (size_t)k * g->nloc * 8 : nullptr);
  }
  return e;
}

int igg_checkpoint_slots(int nt, int every) {
  clear_error();
  if (nt < 1 || every < 1) return set_error(IGG_EINVAL, "need nt >= 1 and every >= 1");
  return (nt + every - 1) / every;
}

int igg_adjoint_step(igg_grid *g, void *lam_out, const void *lam_in, const void *Tn,
                     const void *Ci, double *gCi, igg_dtype dt, double lam, double dtime,
                     double dx, double dy, double dz, void *stream) {
  clear_error();
  if (int rc = check_grid(g)) return rc;
  if (int rc = check_adjoint_grid(g, dt)) return rc;
  for (const void *p : {(const void *)lam_out, lam_in, Tn, Ci, (const void *)gCi})
    if (int rc = check_field(g, p, "field")) return rc;
  if (lam_out == lam_in) return set_error(IGG_EINVAL, "lam_out aliases lam_in");
  if (int rc = check_coef(lam, dtime, dx, dy, dz)) return rc;
  DeviceGuard dg(g->device);
  cudaError_t e = adjoint_subdomains(g, dt, lam_out, lam_in, Tn, Ci, gCi,
                                     make_coef(lam, dtime, dx, dy, dz), (cudaStream_t)stream,
                                     nullptr);
  if (e != cudaSuccess) return cuda_error(e, "adjoint launch");
  return IGG_OK;
}

int igg_update_halo_adjoint(igg_grid *g, void *lam, igg_dtype dt, void *stream) {
  clear_error();
  if (int rc = check_grid(g)) return rc;
  if (dt != IGG_F64 && dt != IGG_F32) return set_error(IGG_EINVAL, "dtype must be F64 or F32");
  if (int rc = check_field(g, lam, "lam")) return rc;
  DeviceGuard dg(g->device);
  cudaError_t e = enqueue_halo_adjoint(g, lam, dtype_size(dt), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_error(e, "halo adjoint launch");
  return IGG_OK;
}

int igg_residual(void *out, const void *a, const void *b, size_t n, igg_dtype dt, void *stream) {
  clear_error();
  if (dt != IGG_F64 && dt != IGG_F32) return set_error(IGG_EINVAL, "dtype must be F64 or F32");
  if (n > 0 && (!out || !a || !b)) return set_error(IGG_EINVAL, "NULL pointer");
  if (n == 0) return IGG_OK;
  cudaError_t e = launch_sub(dt, (long long)n, out, a, b, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_error(e, "residual launch");
  return IGG_OK;
}

int igg_forward_checkpointed(igg_grid *g, int nt, int every, const void *T0, const void *Ci,
                             igg_dtype dt, double lam, double dtime, double dx, double dy,
                             double dz, void *ckpt, void *work, void *T_out, void *stream) {
  clear_error();
  if (int rc = check_grid(g)) return rc;
  if (int rc = check_adjoint_grid(g, dt)) return rc;
  const int nslots = igg_checkpoint_slots(nt, every);
  if (nslots < 0) return nslots;
  for (const void *p : {T0, Ci, (const void *)ckpt, (const void *)work, (const void *)T_out})
    if (int rc = check_field(g, p, "field")) return rc;
  if (int rc = check_coef(lam, dtime, dx, dy, dz)) return rc;
  DeviceGuard dg(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t es = dtype_size(dt), bytes = (size_t)g->nsub * (size_t)g->nloc * es;
  const bool halo = any_halo(g);  // the steps of Fig. 1's loop: step!, then update_halo!
  char *A = (char *)work, *B = (char *)work + bytes, *K = (char *)ckpt;
  const Coef c = make_coef(lam, dtime, dx, dy, dz);
  cudaError_t e = cudaMemcpyAsync(A, T0, bytes, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(B, T0, bytes, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(K, T0, bytes, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_error(e, "checkpoint copy");
  char *cur = A;
  for (int n = 0; n < nt; ++n) {
    char *nxt = cur == A ? B : A;
    if (int rc = enqueue_step(g, nullptr, nxt, cur, Ci, dt, c, halo, s)) return rc;
    cur = nxt;
    if ((n + 1) % every == 0 && n + 1 < nt) {
      e = cudaMemcpyAsync(K + (size_t)((n + 1) / every) * bytes, cur, bytes,
                          cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) return cuda_error(e, "checkpoint copy");
    }
  }
  e = cudaMemcpyAsync(T_out, cur, bytes, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_error(e, "result copy");
  return IGG_OK;
}

int igg_adjoint_checkpointed(igg_grid *g, int nt, int every, const void *ckpt, const void *Ci,
                             const void *lam_nt, igg_dtype dt, double lam, double dtime,
                             double dx, double dy, double dz, void *seg, void *work, void *gT0,
                             double *gCi, void *stream) {
  clear_error();
  if (int rc = check_grid(g)) return rc;
  if (int rc = check_adjoint_grid(g, dt)) return rc;
  const int nslots = igg_checkpoint_slots(nt, every);
  if (nslots < 0) return nslots;
  for (const void *p : {ckpt, Ci, lam_nt, (const void *)work, (const void *)gT0, (const void *)gCi})
    if (int rc = check_field(g, p, "field")) return rc;
  if (every > 1)
    if (int rc = check_field(g, seg, "seg")) return rc;
  if (int rc = check_coef(lam, dtime, dx, dy, dz)) return rc;
  DeviceGuard dg(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t ntot = (size_t)g->nsub * (size_t)g->nloc;
  const size_t es = dtype_size(dt), bytes = ntot * es;
  const bool halo = any_halo(g);
  const char *K = (const char *)ckpt;
  char *S = (char *)seg, *LA = (char *)work, *LB = (char *)work + bytes;
  const Coef c = make_coef(lam, dtime, dx, dy, dz);
  // FP64 fields on the TMA kernel: Ci split into pairs once for the run
  // (stream-ordered scratch, freed on every exit)
  struct Scratch {
    void *p = nullptr;
    cudaStream_t s;
    ~Scratch() {
      if (p) cudaFreeAsync(p, s);
    }
  } ci_pairs;
  ci_pairs.s = s;
  if (dt == IGG_F64 && g->tma_enabled &&
      adjoint_tma_applies(dt, g->n[0], work, lam_nt, ckpt, Ci, gCi)) {
    // without room for the pairs the adjoint steps take the kernel that
    // reads Ci itself (the same bits): a failed allocation is not an error
    if (cudaMallocAsync(&ci_pairs.p, ntot * 8, s) != cudaSuccess) {
      ci_pairs.p = nullptr;
      (void)cudaGetLastError();
    } else {
      cudaError_t ea = launch_pair_ci(Ci, ci_pairs.p, (long long)ntot, s);
      if (ea != cudaSuccess) return cuda_error(ea, "Ci pairs");
    }
  }
  cudaError_t e = cudaMemcpyAsync(LA, lam_nt, bytes, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(gCi, 0, ntot * sizeof(double), s);
  // segment buffers carry the fixed boundary values of T0 (steps write inner points only)
  for (int j = 1; j < every && e == cudaSuccess; ++j)
    e = cudaMemcpyAsync(S + (size_t)(j - 1) * bytes, K, bytes, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_error(e, "adjoint set-up copies");
  char *cur = LA;
  for (int k = nslots - 1; k >= 0; --k) {
    const int s0 = k * every, s1 = std::min(s0 + every, nt), len = s1 - s0;
    auto state = [&](int j) -> const char * {
      return j == 0 ? K + (size_t)k * bytes : S + (size_t)(j - 1) * bytes;
    };
    for (int j = 1; j < len; ++j)
      if (int rc = enqueue_step(g, nullptr, (void *)state(j), state(j - 1), Ci, dt, c, halo, s))
        return rc;
    for (int j = len - 1; j >= 0; --j) {
      // one step is H(S(T)): lam <- H^T lam (in place), then S^T per subdomain
      char *nxt = cur == LA ? LB : LA;
      if (halo && (e = enqueue_halo_adjoint(g, cur, es, s)) != cudaSuccess)
        return cuda_error(e, "halo adjoint launch");
      e = adjoint_subdomains(g, dt, nxt, cur, state(j), Ci, gCi, c, s, ci_pairs.p);
      if (e != cudaSuccess) return cuda_error(e, "adjoint launch");
      cur = nxt;
    }
  }
  e = cudaMemcpyAsync(gT0, cur, bytes, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_error(e, "gradient copy");
  return IGG_OK;
}


int igg_device_status(igg_grid *g, unsigned *status, int clear) {
  clear_error();
  if (int rc = check_grid(g)) return rc;
  if (!status) return set_error(IGG_EINVAL, "status is NULL");
  DeviceGuard dg(g->device);
  cudaError_t e = cudaMemcpy(status, g->dev_err, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && clear) e = cudaMemset(g->dev_err, 0, sizeof(unsigned));
  if (e != cudaSuccess) return cuda_error(e, "device status");
  return IGG_OK;
}

int igg_grid_set_option(igg_grid *g, int option, int value) {
  clear_error();
  if (int rc = check_grid(g)) return rc;
  if (option != IGG_OPT_TMA && option != IGG_OPT_F64_EMU && option != IGG_OPT_FUSED_HALO &&
      option != IGG_OPT_PHASE_TIMES && option != IGG_OPT_HIDE_HALO)
    return set_error(IGG_EINVAL, "unknown option %d", option);
  DeviceGuard dg(g->device);
  cudaError_t e1 = cudaStreamSynchronize(g->hi), e2 = cudaStreamSynchronize(g->lo);
  if (e1 != cudaSuccess) return cuda_error(e1, "set_option");
  if (e2 != cudaSuccess) return cuda_error(e2, "set_option");
  if (option == IGG_OPT_PHASE_TIMES) {  // kernels, tables and graphs are unchanged
    g->phase_times = value != 0;
    g->pev_used = 0;
    return IGG_OK;
  }
  if (option == IGG_OPT_TMA) g->tma_enabled = value != 0;
  else if (option == IGG_OPT_F64_EMU) g->f64_emu = value != 0 ? 1 : 0;
  else if (option == IGG_OPT_HIDE_HALO) g->hide_halo = value != 0;
  else g->fused_halo = value != 0;
  // tile tables and graphs depend on the kernel choice
  for (auto &kv : g->graphs) cudaGraphExecDestroy(kv.second);
  g->graphs.clear();
  for (auto &kv : g->split) {
    for (auto &b : kv.second.boundary) free_tiles(b);
    free_tiles(kv.second.inner);
  }
  g->split.clear();
  for (auto &kv : g->full) free_tiles(kv.second);
  for (auto &kv : g->part) {
    free_tiles(kv.second.face);
    free_tiles(kv.second.inner);
  }
  g->full.clear();
  g->part.clear();
  return IGG_OK;
}

int igg_phase_times(igg_grid *g, double ms[3], int *steps) {
  clear_error();
  if (int rc = check_grid(g)) return rc;
  if (!ms || !steps) return set_error(IGG_EINVAL, "ms or steps is NULL");
  DeviceGuard dg(g->device);
  ms[0] = ms[1] = ms[2] = 0.0;
  const int n = g->pev_used / 3;
  *steps = n;
  g->pev_used = 0;
  if (n == 0) return IGG_OK;
  cudaError_t e = cudaEventSynchronize(g->pev[3 * n - 1]);
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    float a = 0.f, b = 0.f;
    e = cudaEventElapsedTime(&a, g->pev[3 * i], g->pev[3 * i + 1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&b, g->pev[3 * i + 1], g->pev[3 * i + 2]);
    ms[0] += a;
    ms[1] += b;
    ms[2] += (double)a + b;
  }
  if (e != cudaSuccess) return cuda_error(e, "phase times");
  return IGG_OK;
}

int igg_bounds_checked(void) {
#ifdef IGG_BOUNDS_CHECK
  return 1;
#else
  return 0;
#endif
}

int igg_bounds_status(unsigned *status, int clear) {
  clear_error();
  if (!status) return set_error(IGG_EINVAL, "status is NULL");
  unsigned a = 0u, b = 0u;
  cudaError_t e = tma_bounds_flag(&a, clear != 0);
  if (e == cudaSuccess) e = halo_bounds_flag(&b, clear != 0);
  if (e != cudaSuccess) return cuda_error(e, "bounds status");
  *status = (a | b) ? IGG_DEV_ERR_BOUNDS : 0u;
  return IGG_OK;
}

int igg_fixup_stats(igg_grid *g, unsigned long long counts[2], int clear) {
  clear_error();
  if (int rc = check_grid(g)) return rc;
  if (!counts) return set_error(IGG_EINVAL, "counts is NULL");
  DeviceGuard dg(g->device);
  counts[0] = counts[1] = 0ull;
  cudaError_t e = cudaDeviceSynchronize();
  std::vector<FixBuf *> bufs;
  for (auto &kv : g->full) bufs.push_back(&kv.second.fix);
  for (auto &kv : g->part) {
    bufs.push_back(&kv.second.face.fix);
    bufs.push_back(&kv.second.inner.fix);
  }
  for (auto &kv : g->split) {
    for (auto &b : kv.second.boundary) bufs.push_back(&b.fix);
    bufs.push_back(&kv.second.inner.fix);
  }
  for (FixBuf *f : bufs) {
    if (!f->p || e != cudaSuccess) continue;
    unsigned long long t[2];
    char *tot = (char *)f->p + tma_fix_bytes(f->cap) - 16;
    e = cudaMemcpy(t, tot, sizeof t, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && clear) e = cudaMemset(tot, 0, sizeof t);
    counts[0] += t[0];
    counts[1] += t[1];
  }
  if (e != cudaSuccess) return cuda_error(e, "fix-up stats");
  return IGG_OK;
}

}  // extern "C"
