// Batched form of the step: many independent diffusion problems of uneven
// sizes advanced together, one persistent launch per step, the nt-step loop
// captured in a CUDA graph, and an autotuner that picks the tile shape, the
// z depth of a tile and the number of CTAs per SM by timing them on the
// caller's data.
//
// Layout: all problems of a field share one device buffer; problem b is an
// array [nz_b][ny_b][pitch_b] (x fastest, rows padded to pitch_b >= nx_b
// elements, a multiple of 16 bytes) starting at element offset off[b], every
// offset aligned to 256 bytes. Each problem has its own lam, dt, dx, dy, dz
// (coefficient table on the device).
//
// Kernels: variant 4 launches the TMA-pipelined kernel over every problem's
// tiles (per-problem tensor maps in device memory; the default where the
// driver's tensor-map encoder is available); variant 3 the register-pipelined
// 16-byte vector kernel, one CTA per tile of rows;
// variants 0-2 the persistent scalar kernel with 32x8, 32x4 or 64x4 column
// tiles.
//
// Autotune cache: the tuned tiling is kept per (GPU name, dtype, problem
// sizes), in the process and, when the environment variable
// IGG_AUTOTUNE_CACHE names a file, in that file (one line per key:
// "<key> <variant> <zb> <ctas_per_sm> <ms>"), so that a later batch of the
// same shapes, in this process or another, skips the timing.
#include <algorithm>
#include <array>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "igg_internal.h"

using namespace igg;

namespace {

// the vector-kernel variant (one CTA per tile), the TMA variant; below them
// the persistent ones
constexpr int kBatchVector = kPersistentVariants;
constexpr int kBatchTma = kBatchVector + 1;

// CTAs per SM of each persistent variant for this dtype (occupancy query).
int max_ctas_per_sm(igg_dtype dt, int variant);

struct TunedCfg {
  int cfg[3];
  float ms;
};
std::mutex g_tune_mu;
std::map<std::string, TunedCfg> g_tune;  // the process's cache
bool g_tune_file_read = false;

const char *tune_file() {
  const char *p = std::getenv("IGG_AUTOTUNE_CACHE");
  return p && *p ? p : nullptr;
}

// FNV-1a over the problem sizes
unsigned long long sizes_hash(const std::vector<std::array<int, 3>> &sizes) {
  unsigned long long h = 1469598103934665603ull;
  for (const auto &s : sizes)
    for (int v : s)
      for (int k = 0; k < 4; ++k) {
        h ^= (unsigned long long)((unsigned)v >> (8 * k) & 0xFFu);
        h *= 1099511628211ull;
      }
  return h;
}

// key: GPU name (spaces as '_'), dtype, problem count, hash of the sizes
std::string tune_key(int device, igg_dtype dt, const std::vector<std::array<int, 3>> &sizes) {
  cudaDeviceProp prop;
  std::string name = cudaGetDeviceProperties(&prop, device) == cudaSuccess ? prop.name : "unknown";
  for (char &c : name)
    if (c == ' ' || c == '\t') c = '_';
  char buf[96];
  snprintf(buf, sizeof buf, "|dt%d|n%zu|%016llx", (int)dt, sizes.size(), sizes_hash(sizes));
  return name + buf;
}

// the file's entries into the process cache, once (caller holds the lock)
void read_tune_file() {
  if (g_tune_file_read) return;
  g_tune_file_read = true;
  const char *path = tune_file();
  if (!path) return;
  FILE *f = std::fopen(path, "r");
  if (!f) return;
  char key[256];
  TunedCfg t;
  while (std::fscanf(f, "%255s %d %d %d %f", key, &t.cfg[0], &t.cfg[1], &t.cfg[2], &t.ms) == 5)
    g_tune[key] = t;
  std::fclose(f);
}

bool tune_lookup(const std::string &key, TunedCfg *out) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  read_tune_file();
  auto it = g_tune.find(key);
  if (it == g_tune.end()) return false;
  *out = it->second;
  return true;
}

void tune_store(const std::string &key, const TunedCfg &t) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  read_tune_file();
  g_tune[key] = t;
  if (const char *path = tune_file()) {
    if (FILE *f = std::fopen(path, "a")) {
      std::fprintf(f, "%s %d %d %d %.6f\n", key.c_str(), t.cfg[0], t.cfg[1], t.cfg[2], t.ms);
      std::fclose(f);
    }
  }
}

}  // namespace

struct igg_batch {
  int nprob = 0;
  igg_dtype dtype = IGG_F32;
  int device = 0;
  int sm_count = 0;
  std::vector<std::array<int, 3>> sizes;
  std::vector<int> pitch;  // row pitch of each problem (elements)
  std::vector<long long> offsets;
  long long total = 0;
  Coef *coef = nullptr;
  bool have_coef = false;
  int variant = kBatchVector, zb = 32, ctas_per_sm = 0;
  Tile *tiles = nullptr;      // variants 0-2
  VTile *vtiles = nullptr;    // variant 3
  TmaTile *ttiles = nullptr;  // variant 4
  int ntiles = 0;
  // variant 4: tensor maps per (T, Ci) pointer pair, row pitch and ny per
  // problem, device error word of the TMA kernel
  std::map<std::pair<const void *, const void *>, TmaMapBytes *> maps;
  int *geom = nullptr;
  unsigned *dev_err = nullptr;
  cudaStream_t cap = nullptr;
  std::map<std::tuple<const void *, const void *, const void *>, cudaGraphExec_t> graphs;
};

namespace {

void drop_graphs(igg_batch *b) {
  for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
  b->graphs.clear();
}

int build_tiles(igg_batch *b) {
  cudaFree(b->tiles);
  cudaFree(b->vtiles);
  cudaFree(b->ttiles);
  b->tiles = nullptr;
  b->vtiles = nullptr;
  b->ttiles = nullptr;
  b->ntiles = 0;
  drop_graphs(b);
  cudaError_t e = cudaSuccess;
  if (b->variant == kBatchTma) {
    const int V = vec_width(b->dtype);
    const int Wt = tma_tile_width(b->dtype, TMA_WIDE), Ht = tma_tile_rows(b->dtype, TMA_WIDE);
    std::vector<TmaTile> v;
    for (int p = 0; p < b->nprob; ++p) {
      const int nx = b->sizes[p][0], ny = b->sizes[p][1], nz = b->sizes[p][2];
      const size_t first = v.size();
      add_box_tma(v, b->offsets[p], 0, 1, nx - 1, 1, ny - 1, 1, nz - 1,
                  b->zb > 0 ? b->zb : nz - 2, V, Wt, Ht);
      for (size_t k = first; k < v.size(); ++k) v[k].pad[0] = p;
    }
    b->ntiles = (int)v.size();
    e = cudaMalloc(&b->ttiles, v.size() * sizeof(TmaTile));
    if (e == cudaSuccess)
      e = cudaMemcpy(b->ttiles, v.data(), v.size() * sizeof(TmaTile), cudaMemcpyHostToDevice);
  } else if (b->variant == kBatchVector) {
    const int V = vec_width(b->dtype);
    std::vector<VTile> v;
    for (int p = 0; p < b->nprob; ++p) {
      const int nx = b->sizes[p][0], ny = b->sizes[p][1], nz = b->sizes[p][2];
      add_box_vec_pitched(v, b->offsets[p], nx, b->pitch[p], ny, 1, nx - 1, 1, ny - 1, 1, nz - 1,
                          b->zb > 0 ? b->zb : nz - 2, p, V);
    }
    b->ntiles = (int)v.size();
    e = cudaMalloc(&b->vtiles, v.size() * sizeof(VTile));
    if (e == cudaSuccess)
      e = cudaMemcpy(b->vtiles, v.data(), v.size() * sizeof(VTile), cudaMemcpyHostToDevice);
  } else {
    int tx = 32, ty = 8;
    persistent_tile_shape(b->variant, &tx, &ty);
    std::vector<Tile> v;
    for (int p = 0; p < b->nprob; ++p) {
      const int nx = b->sizes[p][0], ny = b->sizes[p][1], nz = b->sizes[p][2];
      const int zb = b->zb > 0 ? b->zb : nz - 2;
      for (int z = 1; z < nz - 1; z += zb)
        for (int y = 1; y < ny - 1; y += ty)
          for (int x = 1; x < nx - 1; x += tx) {
            Tile t;
            t.base = b->offsets[p];
            t.nx = b->pitch[p];  // row stride
            t.ny = ny;
            t.x0 = x;
            t.y0 = y;
            t.xe = nx - 1;
            t.ye = ny - 1;
            t.z0 = z;
            t.z1 = std::min(z + zb, nz - 1);
            t.param = p;
            t.xb = x;
            v.push_back(t);
          }
    }
    b->ntiles = (int)v.size();
    e = cudaMalloc(&b->tiles, v.size() * sizeof(Tile));
    if (e == cudaSuccess)
      e = cudaMemcpy(b->tiles, v.data(), v.size() * sizeof(Tile), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) return cuda_error(e, "batch tile table");
  return IGG_OK;
}

int check_fields(const igg_batch *b, const void *T2, const void *T, const void *Ci) {
  for (const void *p : {T2, T, Ci}) {
    if (!p) return set_error(IGG_EINVAL, "field pointer is NULL");
    if ((uintptr_t)p & 15u) return set_error(IGG_EINVAL, "field pointer is not 16-byte aligned");
  }
  if (T2 == T || T2 == Ci) return set_error(IGG_EINVAL, "T2 aliases T or Ci");
  if (!b->have_coef) return set_error(IGG_ESTATE, "igg_batch_set_coefs was not called");
  return IGG_OK;
}

// Tensor maps of (T, Ci) for the TMA variant, encoded and uploaded on first
// use (before any capture: igg_batch_run prepares both pointer pairs).
int batch_maps(igg_batch *b, const void *T, const void *Ci, const TmaMapBytes **out) {
  const auto key = std::make_pair(T, Ci);
  auto it = b->maps.find(key);
  if (it != b->maps.end()) {
    *out = it->second;
    return IGG_OK;
  }
  std::vector<TmaMapBytes> h(2 * (size_t)b->nprob);
  std::vector<int> sz(3 * (size_t)b->nprob);
  for (int p = 0; p < b->nprob; ++p)
    for (int d = 0; d < 3; ++d) sz[3 * p + d] = b->sizes[p][d];
  if (!tma_batch_maps(b->dtype, T, Ci, b->nprob, b->offsets.data(), sz.data(), b->pitch.data(),
                      h.data()))
    return set_error(IGG_ECUDA, "tensor map encoding failed for the batch");
  TmaMapBytes *d = nullptr;
  cudaError_t e = cudaMalloc(&d, h.size() * sizeof(TmaMapBytes));
  if (e == cudaSuccess) e = cudaMemcpy(d, h.data(), h.size() * sizeof(TmaMapBytes), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d);
    return cuda_error(e, "batch tensor maps");
  }
  if (b->maps.size() >= 8) {  // keep a few pointer pairs
    cudaFree(b->maps.begin()->second);
    b->maps.erase(b->maps.begin());
  }
  b->maps.emplace(key, d);
  *out = d;
  return IGG_OK;
}

int enqueue(igg_batch *b, void *T2, const void *T, const void *Ci, cudaStream_t s) {
  cudaError_t e;
  if (b->variant == kBatchTma) {
    const TmaMapBytes *m = nullptr;
    if (int rc = batch_maps(b, T, Ci, &m)) return rc;
    TmaBatch tb;
    tb.maps = m;
    tb.geom = b->geom;
    tb.coef = b->coef;
    e = launch_stencil_tma_batch(b->dtype, b->ttiles, b->ntiles, T2, tb, b->dev_err, s);
  } else if (b->variant == kBatchVector) {
    e = launch_stencil_vec(b->dtype, b->vtiles, b->ntiles, T2, T, Ci, Coef(), b->coef, s);
  } else {
    const int nctas = b->sm_count * b->ctas_per_sm;
    e = launch_stencil_persistent(b->dtype, b->variant, b->tiles, b->ntiles, nctas, T2, T, Ci,
                                  b->coef, s);
  }
  if (e != cudaSuccess) return cuda_error(e, "batched stencil launch");
  return IGG_OK;
}

struct DevGuard {
  int prev = -1;
  bool changed = false;
  explicit DevGuard(int d) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != d) changed = cudaSetDevice(d) == cudaSuccess;
  }
  ~DevGuard() {
    if (changed) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" {

int igg_batch_create(int nprob, const int *sizes, igg_dtype dt, igg_batch **out) {
  clear_error();
  if (!out) return set_error(IGG_EINVAL, "out is NULL");
  *out = nullptr;
  if (nprob <= 0 || !sizes) return set_error(IGG_EINVAL, "need nprob > 0 and sizes");
  if (dtype_size(dt) == 0) return set_error(IGG_EINVAL, "unknown dtype %d", (int)dt);
  igg_batch *b = new (std::nothrow) igg_batch();
  if (!b) return set_error(IGG_ENOMEM, "host allocation failed");
  b->nprob = nprob;
  b->dtype = dt;
  const long long align = 256 / (long long)dtype_size(dt);
  const int V = vec_width(dt);
  long long off = 0;
  for (int p = 0; p < nprob; ++p) {
    std::array<int, 3> n = {sizes[3 * p], sizes[3 * p + 1], sizes[3 * p + 2]};
    for (int d = 0; d < 3; ++d)
      if (n[d] < 3) {
        delete b;
        return set_error(IGG_EINVAL, "problem %d: size %d < 3 in dim %d", p, n[d], d);
      }
    b->sizes.push_back(n);
    b->pitch.push_back((n[0] + V - 1) / V * V);
    b->offsets.push_back(off);
    off += (long long)b->pitch.back() * n[1] * n[2];
    off = (off + align - 1) / align * align;
  }
  b->total = off;
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device);
  if (e == cudaSuccess) e = cudaMalloc(&b->coef, nprob * sizeof(Coef));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cudaFree(b->coef);
    delete b;
    return cuda_error(e, "batch set-up");
  }
  b->ctas_per_sm = 0;
  b->variant = tma_available() ? kBatchTma : kBatchVector;
  {
    std::vector<int> geom(2 * (size_t)nprob);
    for (int p = 0; p < nprob; ++p) {
      geom[2 * p] = b->pitch[p];
      geom[2 * p + 1] = b->sizes[p][1];
    }
    e = cudaMalloc(&b->geom, geom.size() * sizeof(int));
    if (e == cudaSuccess)
      e = cudaMemcpy(b->geom, geom.data(), geom.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&b->dev_err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(b->dev_err, 0, sizeof(unsigned));
    if (e == cudaSuccess && tma_available()) e = tma_batch_prepare(dt);
    if (e != cudaSuccess) {
      cudaFree(b->geom);
      cudaFree(b->dev_err);
      cudaFree(b->coef);
      cudaStreamDestroy(b->cap);
      delete b;
      return cuda_error(e, "batch set-up");
    }
  }
  if (int rc = build_tiles(b)) {
    cudaFree(b->coef);
    cudaStreamDestroy(b->cap);
    delete b;
    return rc;
  }
  *out = b;
  return IGG_OK;
}

int igg_batch_destroy(igg_batch *b) {
  clear_error();
  if (!b) return IGG_OK;
  DevGuard g(b->device);
  cudaError_t e = cudaStreamSynchronize(b->cap);
  drop_graphs(b);
  cudaFree(b->tiles);
  cudaFree(b->vtiles);
  cudaFree(b->ttiles);
  for (auto &kv : b->maps) cudaFree(kv.second);
  cudaFree(b->geom);
  cudaFree(b->dev_err);
  cudaFree(b->coef);
  cudaStreamDestroy(b->cap);
  delete b;
  if (e != cudaSuccess) return cuda_error(e, "batch destroy");
  return IGG_OK;
}

int igg_batch_layout(const igg_batch *b, long long *offsets, long long *total) {
  clear_error();
  if (!b) return set_error(IGG_EINVAL, "batch is NULL");
  if (offsets) std::memcpy(offsets, b->offsets.data(), b->nprob * sizeof(long long));
  if (total) *total = b->total;
  return IGG_OK;
}

int igg_batch_pitches(const igg_batch *b, int *pitches) {
  clear_error();
  if (!b) return set_error(IGG_EINVAL, "batch is NULL");
  if (!pitches) return set_error(IGG_EINVAL, "pitches is NULL");
  std::memcpy(pitches, b->pitch.data(), b->nprob * sizeof(int));
  return IGG_OK;
}

int igg_batch_set_coefs(igg_batch *b, const double *lam, const double *dt, const double *dx,
                        const double *dy, const double *dz) {
  clear_error();
  if (!b) return set_error(IGG_EINVAL, "batch is NULL");
  if (!lam || !dt || !dx || !dy || !dz) return set_error(IGG_EINVAL, "coefficient array is NULL");
  std::vector<Coef> c(b->nprob);
  for (int p = 0; p < b->nprob; ++p) {
    if (!(dx[p] > 0) || !(dy[p] > 0) || !(dz[p] > 0))
      return set_error(IGG_EINVAL, "problem %d: spacings must be positive", p);
    c[p] = make_coef(lam[p], dt[p], dx[p], dy[p], dz[p]);
  }
  DevGuard g(b->device);
  cudaError_t e = cudaMemcpy(b->coef, c.data(), c.size() * sizeof(Coef), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_error(e, "cudaMemcpy(batch coefficients)");
  b->have_coef = true;
  drop_graphs(b);
  return IGG_OK;
}

int igg_batch_configure(igg_batch *b, int variant, int zb, int ctas_per_sm) {
  clear_error();
  if (!b) return set_error(IGG_EINVAL, "batch is NULL");
  if (variant < 0 || variant > kBatchTma)
    return set_error(IGG_EINVAL, "variant %d outside [0, %d]", variant, kBatchTma);
  if (variant == kBatchTma && !tma_available())
    return set_error(IGG_EINVAL, "the TMA variant needs the driver's tensor-map encoder");
  if (zb < 0) return set_error(IGG_EINVAL, "zb < 0");
  DevGuard g(b->device);
  if (variant >= kBatchVector) {
    if (ctas_per_sm != 0)
      return set_error(IGG_EINVAL, "ctas_per_sm must be 0 for the vector variant (one CTA per tile)");
  } else {
    const int cmax = max_ctas_per_sm(b->dtype, variant);
    if (ctas_per_sm <= 0) ctas_per_sm = cmax;
    if (ctas_per_sm > cmax)
      return set_error(IGG_EINVAL, "ctas_per_sm %d above the resident maximum %d", ctas_per_sm,
                       cmax);
  }
  b->variant = variant;
  b->zb = zb;
  b->ctas_per_sm = ctas_per_sm;
  return build_tiles(b);
}

int igg_batch_get_config(const igg_batch *b, int cfg[3], int *ntiles) {
  clear_error();
  if (!b) return set_error(IGG_EINVAL, "batch is NULL");
  if (cfg) {
    cfg[0] = b->variant;
    cfg[1] = b->zb;
    cfg[2] = b->ctas_per_sm;
  }
  if (ntiles) *ntiles = b->ntiles;
  return IGG_OK;
}

int igg_batch_step(igg_batch *b, void *T2, const void *T, const void *Ci, void *stream) {
  clear_error();
  if (!b) return set_error(IGG_EINVAL, "batch is NULL");
  if (int rc = check_fields(b, T2, T, Ci)) return rc;
  DevGuard g(b->device);
  return enqueue(b, T2, T, Ci, (cudaStream_t)stream);
}

int igg_batch_run(igg_batch *b, int nt, void *T, void *T2, const void *Ci, void *stream) {
  clear_error();
  if (!b) return set_error(IGG_EINVAL, "batch is NULL");
  if (nt < 0) return set_error(IGG_EINVAL, "nt < 0");
  if (int rc = check_fields(b, T2, T, Ci)) return rc;
  if (T == Ci) return set_error(IGG_EINVAL, "T aliases Ci");
  DevGuard g(b->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (b->variant == kBatchTma) {  // tensor maps are built outside any capture
    const TmaMapBytes *m = nullptr;
    if (int rc = batch_maps(b, T, Ci, &m)) return rc;
    if (int rc = batch_maps(b, T2, Ci, &m)) return rc;
  }
  if (nt >= 2) {
    auto key = std::make_tuple((const void *)T, (const void *)T2, Ci);
    cudaGraphExec_t exec = nullptr;
    auto it = b->graphs.find(key);
    if (it != b->graphs.end()) {
      exec = it->second;
    } else {
      cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_error(e, "cudaStreamBeginCapture");
      int rc = enqueue(b, T2, T, Ci, b->cap);
      if (rc == IGG_OK) rc = enqueue(b, T, T2, Ci, b->cap);
      cudaGraph_t graph = nullptr;
      e = cudaStreamEndCapture(b->cap, &graph);
      if (rc != IGG_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
      }
      if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
      e = cudaGraphInstantiateWithFlags(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_error(e, "cudaGraphInstantiate");
      if (b->graphs.size() >= 8) {
        cudaGraphExecDestroy(b->graphs.begin()->second);
        b->graphs.erase(b->graphs.begin());
      }
      b->graphs.emplace(key, exec);
    }
    for (int i = 0; i < nt / 2; ++i) {
      cudaError_t e = cudaGraphLaunch(exec, s);
      if (e != cudaSuccess) return cuda_error(e, "cudaGraphLaunch");
    }
  }
  if (nt % 2) return enqueue(b, T2, T, Ci, s);
  return IGG_OK;
}

int igg_batch_autotune(igg_batch *b, void *T2, const void *T, const void *Ci, int reps,
                       void *stream, int best_cfg[3], float *best_ms) {
  clear_error();
  if (!b) return set_error(IGG_EINVAL, "batch is NULL");
  if (int rc = check_fields(b, T2, T, Ci)) return rc;
  DevGuard g(b->device);
  const std::string key = tune_key(b->device, b->dtype, b->sizes);
  TunedCfg hit;
  if (reps >= 0 && tune_lookup(key, &hit)) {
    b->variant = hit.cfg[0];
    b->zb = hit.cfg[1];
    b->ctas_per_sm = hit.cfg[2];
    if (int rc = build_tiles(b)) return rc;
    if (best_cfg) std::memcpy(best_cfg, hit.cfg, sizeof hit.cfg);
    if (best_ms) *best_ms = hit.ms;
    return IGG_OK;
  }
  if (reps <= 0) reps = 3;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return cuda_error(e, "cudaEventCreate");
  const int zbs[] = {8, 16, 32, 64, 0};
  float best = 1e30f;
  int bv = b->variant, bz = b->zb, bc = b->ctas_per_sm;
  int rc = IGG_OK;
  for (int v = 0; v <= kBatchTma && rc == IGG_OK; ++v) {
    if (v == kBatchTma && !tma_available()) break;
    const bool one_cta_per_tile = v >= kBatchVector;
    const int cmax = one_cta_per_tile ? 0 : max_ctas_per_sm(b->dtype, v);
    const int cands[2] = {cmax, std::max(1, cmax / 2)};
    for (int zb : zbs) {
      for (int ci = 0; ci < (cmax > 1 ? 2 : 1); ++ci) {
        b->variant = v;
        b->zb = zb;
        b->ctas_per_sm = cands[ci];
        if ((rc = build_tiles(b)) != IGG_OK) break;
        if ((rc = enqueue(b, T2, T, Ci, s)) != IGG_OK) break;  // warm-up
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && rc == IGG_OK; ++r) rc = enqueue(b, T2, T, Ci, s);
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
          rc = cuda_error(e, "autotune timing");
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        if (ms < best) {
          best = ms;
          bv = v;
          bz = zb;
          bc = cands[ci];
        }
      }
      if (rc != IGG_OK) break;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->variant = bv;
  b->zb = bz;
  b->ctas_per_sm = bc;
  int rc2 = build_tiles(b);
  if (rc != IGG_OK) return rc;
  if (rc2 != IGG_OK) return rc2;
  if (best_cfg) {
    best_cfg[0] = bv;
    best_cfg[1] = bz;
    best_cfg[2] = bc;
  }
  if (best_ms) *best_ms = best;
  tune_store(key, TunedCfg{{bv, bz, bc}, best});
  return IGG_OK;
}

}  // extern "C"

namespace {
int max_ctas_per_sm(igg_dtype dt, int variant) {
  int n = persistent_occupancy(dt, variant);
  return n > 0 ? n : 1;
}
}  // namespace
