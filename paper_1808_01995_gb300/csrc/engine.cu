// Host side of the propagator library: contexts with a budgeted caching device
// allocator, the pitched field layout, TMA descriptors, sparse-point setup,
// the time loops (forward, adjoint, forward with snapshots, backward with
// recompute + fused gradient), and the C ABI declared in wavprop.h.
#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include "../../include/wavprop.h"
#include "kernels.cuh"
#include "stencil3d.cuh"
#include "stencil3d_hi.cuh"

using namespace wp;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

static int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CU(x)                                                                                  \
  do {                                                                                         \
    cudaError_t e_ = (x);                                                                      \
    if (e_ != cudaSuccess) return fail(WP_ECUDA, "%s failed: %s", #x, cudaGetErrorString(e_)); \
  } while (0)

#define TRY(x)              \
  do {                      \
    int rc_ = (x);          \
    if (rc_ != WP_OK) return rc_; \
  } while (0)

// NVTX range over a host scope (the phases of a call: forward, adjoint,
// recompute, ...); free when no profiler is attached.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct wp_ctx {
  int device = 0;
  int num_sms = 0;
  size_t budget = 0;
  size_t in_use = 0;                       // live + cached device bytes
  std::multimap<size_t, void *> cache;     // free blocks by size
  std::map<void *, size_t> live;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_done = nullptr;
  double timeout_s = 600.0;
  int *d_scalars = nullptr;                // [0] error word, [1] bad-input bits, [2] max(1/m) bits, [8..14] box
  int *h_scalars = nullptr;                // pinned mirror
  uint64_t launches = 0;
  int smem3d[2][9] = {};
  int occ3d[2][9] = {};
  int ty3d[2][9] = {};
  uint64_t wait_ns = kWaitLimitNs;        // limit of the kernels' ring waits
  bool broken = false;
  // profiling: an event pair around every prof_every-th stencil launch, summed on read
  bool profiling = false;
  int prof_every = 1;
  uint64_t prof_seq = 0;  // stencil launches seen (restarts for every graph hash/capture pass)
  bool prof_open = false; // the last stencil launch was bracketed
  std::vector<cudaEvent_t> prof_events;   // 2 per launch
  size_t prof_used = 0;
  double prof_ms = 0.0;
  uint64_t prof_count = 0;
  std::vector<cudaEvent_t> *prof_ev = nullptr;  // where the next stencil events go
  size_t *prof_n = nullptr;
  // Programmatic dependent launch inside the time loop: a step kernel whose
  // predecessor on the stream is another step kernel (chain) may start launching
  // while that one still runs (its blocks wait for it on the device), hiding the
  // launch gaps between the stencil, injection and interpolation of a step.
  // pdl_mode: 0 never, 1 (default) at every order, 2 only with the stencil kernel
  // of half-orders up to 4.  Measured: the 280^3 SO8 gradient (plain launches)
  // 437 -> 412 ms; 336^3 shots of 1000 steps (replayed graphs) SO16 1.5 us less
  // per step, SO8 within the noise of 1 us.
  int pdl_mode = 1;
  bool pdl_scope = false;  // inside a time loop that uses it
  bool chain = false;      // the last operation enqueued was a step kernel
  // CUDA graphs of time-loop blocks (see graph_replay)
  bool use_graphs = true;
  bool hashing = false, capturing = false;
  uint64_t hash = 0;
  size_t hash_marks = 0;
  long long *d_rows = nullptr;            // device row bases read by the sparse kernels
  std::vector<struct GraphEntry *> graphs;
  uint64_t graph_stamp = 0;
  // states handed out by wp_forward_save and not yet freed: wp_destroy releases
  // their device memory and detaches them, so a state freed after its context
  // touches nothing of it
  std::set<struct wp_state *> states;
};

// One instantiated graph of a block of time steps, replayable while every
// kernel argument (hashed into `key`) is unchanged.
struct GraphEntry {
  uint64_t key = 0;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaEvent_t> ev;  // events recorded by the graph's profiling nodes
  size_t nev = 0;
  uint64_t kernels = 0;         // kernel nodes per replay
  uint64_t stamp = 0;
};

static void graph_destroy(GraphEntry *e) {
  if (e->exec) cudaGraphExecDestroy(e->exec);
  for (cudaEvent_t ev : e->ev) cudaEventDestroy(ev);
  delete e;
}

static size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Device blocks are stream-ordered allocations on the context's stream, so
// releasing them never waits for work of other contexts (cudaFree would
// synchronise the whole device).
static void release_cache(wp_ctx *c, size_t need) {
  while (!c->cache.empty() && (need == 0 || c->in_use + need > c->budget)) {
    auto it = std::prev(c->cache.end());
    cudaFreeAsync(it->second, c->stream);
    c->in_use -= it->first;
    c->cache.erase(it);
  }
}

static int dev_alloc(wp_ctx *c, size_t bytes, void **out) {
  bytes = round_up(std::max<size_t>(bytes, 1), 256);
  auto it = c->cache.lower_bound(bytes);
  if (it != c->cache.end() && it->first <= bytes + bytes / 4) {  // reuse a block at most 25 % larger
    *out = it->second;
    c->live[*out] = it->first;
    c->cache.erase(it);
    return WP_OK;
  }
  if (c->in_use + bytes > c->budget) release_cache(c, bytes);
  if (c->in_use + bytes > c->budget)
    return fail(WP_ENOMEM, "request of %zu bytes exceeds the context budget (%zu of %zu bytes in use)",
                bytes, c->in_use, c->budget);
  cudaError_t e = cudaMallocAsync(out, bytes, c->stream);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    release_cache(c, 0);
    cudaStreamSynchronize(c->stream);
    e = cudaMallocAsync(out, bytes, c->stream);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    *out = nullptr;
    return fail(e == cudaErrorMemoryAllocation ? WP_ENOMEM : WP_ECUDA, "cudaMallocAsync(%zu) failed: %s", bytes,
                cudaGetErrorString(e));
  }
  c->in_use += bytes;
  c->live[*out] = bytes;
  return WP_OK;
}

static void dev_free(wp_ctx *c, void *p) {
  if (!p) return;
  auto it = c->live.find(p);
  if (it == c->live.end()) return;
  c->cache.emplace(it->second, p);
  c->live.erase(it);
}

// Allocations released (to the context cache) at scope exit.
struct Arena {
  wp_ctx *c;
  std::vector<void *> ptrs;
  explicit Arena(wp_ctx *c_) : c(c_) {}
  ~Arena() {
    for (void *p : ptrs) dev_free(c, p);
  }
  template <class T>
  int alloc(T **out, size_t count) {
    void *p = nullptr;
    TRY(dev_alloc(c, count * sizeof(T), &p));
    ptrs.push_back(p);
    *out = static_cast<T *>(p);
    return WP_OK;
  }
  void release_all_to(std::vector<void *> &dst) {
    dst.insert(dst.end(), ptrs.begin(), ptrs.end());
    ptrs.clear();
  }
};

// Wait for everything queued on the context stream, with a deadline; `what`
// names the phase in error messages.
static int ctx_wait(wp_ctx *c, const char *what = "device work") {
  CU(cudaEventRecord(c->ev_done, c->stream));
  const auto t0 = std::chrono::steady_clock::now();
  int spins = 0;
  while (true) {
    cudaError_t e = cudaEventQuery(c->ev_done);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) return fail(WP_ECUDA, "%s failed: %s", what, cudaGetErrorString(e));
    const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (dt > c->timeout_s) {
      c->broken = true;
      return fail(WP_ETIMEOUT, "%s did not finish within %.1f s", what, c->timeout_s);
    }
    if (++spins > 64) std::this_thread::sleep_for(std::chrono::microseconds(spins > 1000 ? 200 : 20));
  }
  return WP_OK;
}

static const char *device_error_text(int code) {
  switch (code) {
    case kErrWaitFull: return "a wait inside a kernel gave up (its limit ran out)";
    case kErrLaunch: return "a kernel was launched with an unsupported shape";
    case kErrBounds: return "a bounds check failed (debug build)";
    default: return "unknown device error";
  }
}

static int check_device_error(wp_ctx *c) {
  CU(cudaMemcpyAsync(c->h_scalars, c->d_scalars, 4 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  TRY(ctx_wait(c));
  if (c->h_scalars[0] != 0)
    return fail(WP_EDEVICE, "a kernel reported device error %d: %s", c->h_scalars[0],
                device_error_text(c->h_scalars[0]));
  return WP_OK;
}

// ---------------------------------------------------------------------------
// geometry, weights, CFL
// ---------------------------------------------------------------------------
struct Geom {
  int ndim = 3;
  int nz = 0, ny = 1, nx = 0;
  int pitch = 0;
  long long plane = 0;     // ny * pitch
  long long nfield = 0;    // nz * plane (elements of a pitched field)
  long long npoints = 0;   // nz * ny * nx
  double h[3] = {1, 1, 1}; // z, y, x
  double o[3] = {0, 0, 0};
  int k = 0, R = 0;
  double dt = 0;
  int nt = 0;
  int tiles_x = 1, tiles_y = 1;  // damping-flag tiles (32 x 16)
  int nzw = 1;                    // 32-bit words of a tile's z bitmask
  FieldGeom fg() const {
    FieldGeom g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.pitch = pitch;
    g.plane = plane;
    return g;
  }
  size_t field_bytes() const { return static_cast<size_t>(nfield) * sizeof(float); }
};

// a_j = 2 (-1)^{j+1} C(2p, p-j) / (j^2 C(2p, p)),  a_0 = -2 sum a_j   (p = k/2)
static bool weights(int k, double *alpha) {
  if (k < 2 || k > 16 || (k & 1)) return false;
  const int p = k / 2;
  auto binom = [](int n, int r) {
    double v = 1.0;
    for (int i = 1; i <= r; ++i) v = v * (n - r + i) / i;
    return v;
  };
  const double cpp = binom(2 * p, p);
  double sum = 0.0;
  for (int j = 1; j <= p; ++j) {
    alpha[j] = ((j & 1) ? 2.0 : -2.0) * binom(2 * p, p - j) / (double(j) * j * cpp);
    sum += alpha[j];
  }
  alpha[0] = -2.0 * sum;
  return true;
}

static double cfl_limit(const Geom &G, double vmax) {
  double a[9];
  weights(G.k, a);
  double A = std::fabs(a[0]);
  for (int j = 1; j <= G.R; ++j) A += 2.0 * std::fabs(a[j]);
  double s = A / (G.h[0] * G.h[0]) + A / (G.h[2] * G.h[2]);
  if (G.ndim == 3) s += A / (G.h[1] * G.h[1]);
  return 2.0 / (vmax * std::sqrt(s));
}

static int make_geom(const wp_grid *g, Geom *G, bool need_dt = true) {
  if (!g) return fail(WP_EINVAL, "grid is NULL");
  if (g->ndim != 2 && g->ndim != 3) return fail(WP_EINVAL, "ndim must be 2 or 3 (got %d)", g->ndim);
  if (g->space_order < 2 || g->space_order > 16 || (g->space_order & 1))
    return fail(WP_EINVAL, "space_order must be even in [2, 16] (got %d)", g->space_order);
  for (int a = 0; a < g->ndim; ++a) {
    if (g->shape[a] < 2 || g->shape[a] > (1 << 24))
      return fail(WP_EINVAL, "shape[%d] = %lld out of range [2, 2^24]", a, (long long)g->shape[a]);
    if (!(g->spacing[a] > 0) || !std::isfinite(g->spacing[a]))
      return fail(WP_EINVAL, "spacing[%d] must be positive and finite", a);
    if (!std::isfinite(g->origin[a])) return fail(WP_EINVAL, "origin[%d] must be finite", a);
  }
  if (g->nt < 0) return fail(WP_EINVAL, "nt must be >= 0");
  if (need_dt && (!(g->dt > 0) || !std::isfinite(g->dt))) return fail(WP_EINVAL, "dt must be positive");
  G->ndim = g->ndim;
  G->k = g->space_order;
  G->R = g->space_order / 2;
  G->dt = g->dt;
  G->nt = g->nt;
  if (g->ndim == 3) {
    G->nz = int(g->shape[0]);
    G->ny = int(g->shape[1]);
    G->nx = int(g->shape[2]);
    for (int a = 0; a < 3; ++a) {
      G->h[a] = g->spacing[a];
      G->o[a] = g->origin[a];
    }
  } else {
    G->nz = int(g->shape[0]);
    G->ny = 1;
    G->nx = int(g->shape[1]);
    G->h[0] = g->spacing[0];
    G->o[0] = g->origin[0];
    G->h[1] = 1.0;
    G->o[1] = 0.0;
    G->h[2] = g->spacing[1];
    G->o[2] = g->origin[1];
  }
  G->pitch = int(round_up(size_t(G->nx), 32));
  G->plane = static_cast<long long>(G->ny) * G->pitch;
  G->nfield = G->plane * G->nz;
  G->npoints = static_cast<long long>(G->nx) * G->ny * G->nz;
  if (G->nfield > (1ll << 36)) return fail(WP_EINVAL, "grid too large");
  G->tiles_x = (G->nx + kFlagTX - 1) / kFlagTX;  // damping-flag columns
  G->tiles_y = (G->ny + kTileFlagTY - 1) / kTileFlagTY;  // damping-flag rows
  G->nzw = (G->nz + 31) / 32;
  return WP_OK;
}

static LapCoef lap_coef(const Geom &G) {
  double a[9];
  weights(G.k, a);
  LapCoef c;
  memset(&c, 0, sizeof c);
  const double iz = 1.0 / (G.h[0] * G.h[0]), iy = G.ndim == 3 ? 1.0 / (G.h[1] * G.h[1]) : 0.0,
               ix = 1.0 / (G.h[2] * G.h[2]);
  c.c0 = static_cast<float>(a[0] * (iz + iy + ix));
  for (int j = 1; j <= G.R; ++j) {
    c.cz[j] = static_cast<float>(a[j] * iz);
    c.cy[j] = static_cast<float>(a[j] * iy);
    c.cx[j] = static_cast<float>(a[j] * ix);
  }
  c.p0 = make_float2(c.c0, c.c0);
  for (int j = 0; j < 9; ++j) {
    c.pz[j] = make_float2(c.cz[j], c.cz[j]);
    c.py[j] = make_float2(c.cy[j], c.cy[j]);
    c.px[j] = make_float2(c.cx[j], c.cx[j]);
  }
  return c;
}

// ---------------------------------------------------------------------------
// sparse points: multilinear corners (double precision decisions), pitched
// ---------------------------------------------------------------------------
struct PointSet {
  int npts = 0, nc = 0;
  std::vector<long long> idx;  // [npts][nc]
  std::vector<float> w;        // [npts][nc]
};

static int build_points(const Geom &G, int npts, const double *coords, PointSet *ps, const char *what) {
  ps->npts = npts;
  ps->nc = G.ndim == 3 ? 8 : 4;
  ps->idx.assign(size_t(npts) * ps->nc, 0);
  ps->w.assign(size_t(npts) * ps->nc, 0.f);
  if (npts > 0 && !coords) return fail(WP_EINVAL, "%s coordinates are NULL", what);
  const int axes3[3] = {0, 1, 2}, axes2[2] = {0, 2};
  const int *axes = G.ndim == 3 ? axes3 : axes2;
  const int n_of[3] = {G.nz, G.ny, G.nx};
  for (int i = 0; i < npts; ++i) {
    long long base[3] = {0, 0, 0};
    double frac[3] = {0, 0, 0};
    for (int q = 0; q < G.ndim; ++q) {
      const int d = axes[q];
      const double c = coords[size_t(i) * G.ndim + q];
      if (!std::isfinite(c)) return fail(WP_ENONFINITE, "%s %d has a non-finite coordinate", what, i);
      double t = (c - G.o[d]) / G.h[d];
      if (!(t >= -1e-9) || !(t <= double(n_of[d] - 1) + 1e-9))
        return fail(WP_EINVAL, "%s %d lies outside the grid on axis %d", what, i, q);
      t = std::min(std::max(t, 0.0), double(n_of[d] - 1));
      long long b = static_cast<long long>(std::floor(t));
      if (b > n_of[d] - 2) b = n_of[d] - 2;
      if (b < 0) b = 0;
      base[d] = b;
      frac[d] = t - double(b);
    }
    int c = 0;
    for (int cz = 0; cz < 2; ++cz)
      for (int cy = 0; cy < (G.ndim == 3 ? 2 : 1); ++cy)
        for (int cx = 0; cx < 2; ++cx) {
          double w = (cz ? frac[0] : 1.0 - frac[0]);
          if (G.ndim == 3) w *= (cy ? frac[1] : 1.0 - frac[1]);
          w *= (cx ? frac[2] : 1.0 - frac[2]);
          const long long z = base[0] + cz, y = base[1] + cy, x = base[2] + cx;
          ps->idx[size_t(i) * ps->nc + c] = z * G.plane + y * G.pitch + x;
          ps->w[size_t(i) * ps->nc + c] = static_cast<float>(w);
          ++c;
        }
  }
  return WP_OK;
}

// Device copy of a point set: gather form (interpolation) and CSR scatter form
// (injection, entries of one target in (point, corner) order).
struct DevPoints {
  int npts = 0, nc = 0, ntarget = 0;
  long long *idx = nullptr;
  float *w = nullptr;
  long long *target = nullptr;
  int *rowptr = nullptr;
  int *pid = nullptr;
  float *cw = nullptr;
};

static int upload_points(wp_ctx *c, Arena &ar, const PointSet &ps, bool gather, bool scatter, DevPoints *dp) {
  dp->npts = ps.npts;
  dp->nc = ps.nc;
  if (ps.npts == 0) return WP_OK;
  const size_t ne = size_t(ps.npts) * ps.nc;
  if (gather) {
    TRY(ar.alloc(&dp->idx, ne));
    TRY(ar.alloc(&dp->w, ne));
    CU(cudaMemcpyAsync(dp->idx, ps.idx.data(), ne * sizeof(long long), cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemcpyAsync(dp->w, ps.w.data(), ne * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  }
  if (scatter) {
    std::vector<size_t> order(ne);
    for (size_t e = 0; e < ne; ++e) order[e] = e;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return ps.idx[a] < ps.idx[b]; });
    std::vector<long long> target;
    std::vector<int> rowptr, pid;
    std::vector<float> cw;
    for (size_t k = 0; k < ne; ++k) {
      const size_t e = order[k];
      if (target.empty() || target.back() != ps.idx[e]) {
        target.push_back(ps.idx[e]);
        rowptr.push_back(int(k));
      }
      pid.push_back(int(e / ps.nc));
      cw.push_back(ps.w[e]);
    }
    rowptr.push_back(int(ne));
    dp->ntarget = int(target.size());
    TRY(ar.alloc(&dp->target, target.size()));
    TRY(ar.alloc(&dp->rowptr, rowptr.size()));
    TRY(ar.alloc(&dp->pid, pid.size()));
    TRY(ar.alloc(&dp->cw, cw.size()));
    // pageable sources: these copies complete before returning, so the vectors may go
    CU(cudaMemcpy(dp->target, target.data(), target.size() * sizeof(long long), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(dp->rowptr, rowptr.data(), rowptr.size() * sizeof(int), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(dp->pid, pid.data(), pid.size() * sizeof(int), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(dp->cw, cw.data(), cw.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  return WP_OK;
}

// ---------------------------------------------------------------------------
// TMA descriptors
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static int get_encode() {
  if (g_encode) return WP_OK;
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
    return fail(WP_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return WP_OK;
}

// 3D map over a pitched field, box (bx, by, 1); out-of-range elements read as 0.
static int make_map(CUtensorMap *m, const float *base, const Geom &G, int bx, int by) {
  TRY(get_encode());
  cuuint64_t dims[3] = {cuuint64_t(G.nx), cuuint64_t(G.ny), cuuint64_t(G.nz)};
  cuuint64_t strides[2] = {cuuint64_t(G.pitch) * 4, cuuint64_t(G.plane) * 4};
  cuuint32_t box[3] = {cuuint32_t(bx), cuuint32_t(by), 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(WP_ECUDA, "cuTensorMapEncodeTiled failed (%d)", int(r));
  return WP_OK;
}

static int halo_box_w(int R, int mode) { return stencil3d_tile_x(R, mode) + 2 * ((R + 3) / 4 * 4); }

// A field and its TMA descriptors: the halo'd plane box of the forward and of the
// adjoint+gradient stencil (their tiles differ in height).
struct Field3 {
  float *p = nullptr;
  bool mapped = false;  // descriptors encoded for p
  CUtensorMap halo[2], tile[2];
};

static int make_field_maps(Field3 *f, const Geom &G) {
  if (G.ndim != 3) return WP_OK;
  for (int mode = 0; mode < 2; ++mode) {
    const int tx = stencil3d_tile_x(G.R, mode), ty = stencil3d_tile_y(G.R, mode);
    TRY(make_map(&f->halo[mode], f->p, G, halo_box_w(G.R, mode), ty + 2 * G.R));
    TRY(make_map(&f->tile[mode], f->p, G, tx, ty));
  }
  f->mapped = true;
  return WP_OK;
}

// Persistent launch plan of the 3D stencil: (tile, z-chunk) work items walked
// round-robin by ctas = SMs x occupancy CTAs.  The chunk count minimises
// rounds x (chunk + R), the planes streamed by the busiest CTA.
struct Plan3d {
  int tiles_x = 1, tiles_y = 1, zchunk = 1, nzc = 1, nitems = 0;
  dim3 grid;
};

// tx x ty tiles; every item streams its chunk plus `extra` planes
// tx x ty tiles over an nx x ny x nz box; every item streams its chunk plus `extra` planes
static Plan3d plan_items(int nx, int ny, int nz, int R, int tx, int ty, int extra, int num_sms, int occ) {
  Plan3d p;
  p.tiles_x = (nx + tx - 1) / tx;
  p.tiles_y = (ny + ty - 1) / ty;
  const long long tiles = static_cast<long long>(p.tiles_x) * p.tiles_y;
  const long long ctas = static_cast<long long>(num_sms) * std::max(occ, 1);
  double best = 1e300;
  const int min_chunk = std::min(nz, std::max(2 * R, 8));
  for (int nzc = 1; nzc <= nz; ++nzc) {
    const int zc = (nz + nzc - 1) / nzc;
    if (zc < min_chunk) break;
    const int n_eff = (nz + zc - 1) / zc;
    const long long items = tiles * n_eff;
    const long long rounds = (items + ctas - 1) / ctas;
    const double used = std::min(1.0, double(items) / double(ctas));
    // fewer CTAs than slots leave bandwidth unused: charge the idle fraction
    const double cost = double(rounds) * (zc + extra) / std::min(1.0, used / 0.9);
    if (cost < best * 0.999) {
      best = cost;
      p.zchunk = zc;
      p.nzc = n_eff;
    }
  }
  const char *env = getenv("WP_ZCHUNK");
  if (env && atoi(env) > 0) {
    p.zchunk = std::min(nz, atoi(env));
    p.nzc = (nz + p.zchunk - 1) / p.zchunk;
  }
  p.nitems = int(tiles * p.nzc);
  p.grid = dim3(unsigned(std::min<long long>(p.nitems, ctas)));
  return p;
}
static Plan3d plan_items(const Geom &G, int tx, int ty, int extra, int num_sms, int occ) {
  return plan_items(G.nx, G.ny, G.nz, G.R, tx, ty, extra, num_sms, occ);
}

static Plan3d plan3d(const Geom &G, int mode, int num_sms, int occ) {
  return plan_items(G, stencil3d_tile_x(G.R, mode), stencil3d_tile_y(G.R, mode), G.R, num_sms, occ);
}

// ---------------------------------------------------------------------------
// the propagator of one call: coefficients, launch configuration, step launches
// ---------------------------------------------------------------------------
struct Prop {
  wp_ctx *c = nullptr;
  Geom G;
  LapCoef lc;
  float neg_inv_dt2 = 0;
  Field3 b, s;
  unsigned *tbits = nullptr;
  Plan3d plan[2];
  bool sub = false;  // a sub-box for prop_step(..., sub = true): box (x0 a multiple of 4) and its plans
  Box box;
  Plan3d plan_sub[2];
};

// dt, dt^2 and dt/2 for the coefficient kernel, each as a float pair hi + lo
static void coef_set_dt(CoefArgs *a, double dt) {
  auto split = [](double v, float *hi, float *lo) {
    *hi = static_cast<float>(v);
    *lo = static_cast<float>(v - static_cast<double>(*hi));
  };
  a->dt = dt;
  split(dt, &a->dt_hi, &a->dt_lo);
  split(dt * dt, &a->dt2_hi, &a->dt2_lo);
  split(0.5 * dt, &a->hdt_hi, &a->hdt_lo);
}

static int prop_setup(wp_ctx *c, Arena &ar, const Geom &G, const float *m, const float *eta, Prop *P) {
  P->c = c;
  P->G = G;
  P->lc = lap_coef(G);
  P->neg_inv_dt2 = static_cast<float>(-1.0 / (G.dt * G.dt));
  TRY(ar.alloc(&P->b.p, G.nfield));
  TRY(ar.alloc(&P->s.p, G.nfield));
  CU(cudaMemsetAsync(c->d_scalars, 0, 4 * sizeof(int), c->stream));
  CoefArgs a;
  memset(&a, 0, sizeof a);
  a.m = m;
  a.eta = eta;
  a.g = G.fg();
  coef_set_dt(&a, G.dt);
  a.b = P->b.p;
  a.s = P->s.p;
  if (G.ndim == 3) {
    const size_t nflag = size_t(G.nz) * G.tiles_y * G.tiles_x;
    unsigned char *tflag = nullptr;
    TRY(ar.alloc(&tflag, nflag));
    CU(cudaMemsetAsync(tflag, 0, nflag, c->stream));
    TRY(ar.alloc(&P->tbits, size_t(G.tiles_y) * G.tiles_x * G.nzw));
    a.tflag = tflag;
    a.tbits = P->tbits;
    a.nzw = G.nzw;
    a.tiles_x = G.tiles_x;
    a.tiles_y = G.tiles_y;
    a.tile_w = kFlagTX;
    a.tile_h = kTileFlagTY;
  }
  a.max_inv_m_bits = reinterpret_cast<unsigned int *>(c->d_scalars + 2);
  a.bad = c->d_scalars + 1;
  CU(launch_coef(c->stream, a));
  c->launches += G.ndim == 3 ? 2 : 1;
  CU(cudaMemcpyAsync(c->h_scalars, c->d_scalars, 4 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  TRY(ctx_wait(c, "coefficient setup"));
  if (c->h_scalars[1] & 1) return fail(WP_ENONFINITE, "m or eta holds NaN or Inf");
  if (c->h_scalars[1] & 2) return fail(WP_EINVAL, "m must be > 0 and eta >= 0 everywhere");
  float max_inv_m;
  memcpy(&max_inv_m, &c->h_scalars[2], 4);
  const double vmax = std::sqrt(double(max_inv_m));
  const double lim = cfl_limit(G, vmax);
  if (G.dt > lim * (1.0 + 1e-5))
    return fail(WP_ECFL, "dt = %.6g exceeds the stability limit %.6g for vmax = %.6g", G.dt, lim, vmax);
  if (G.ndim == 3) {
    TRY(make_field_maps(&P->b, G));
    TRY(make_field_maps(&P->s, G));
    for (int mode = 0; mode < 2; ++mode) P->plan[mode] = plan3d(G, mode, c->num_sms, c->occ3d[mode][G.R]);
  }
  return WP_OK;
}

// One stencil step: out = update(u, um) (out may alias um).  Adjoint+gradient
// mode also accumulates into grad using the forward field uj.
// While c->hashing is set the launch helpers fold their complete kernel
// arguments (TMA descriptors included) into c->hash instead of launching: two
// blocks of work with the same hash enqueue identical kernels.
static void hash_bytes(wp_ctx *c, const void *p, size_t n) {
  const unsigned char *b = static_cast<const unsigned char *>(p);
  uint64_t h = c->hash;
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  c->hash = h;
}

// Whether the next step kernel may use a programmatic launch; every step-kernel
// launcher calls it once and then marks the chain (in hashing mode too, so that
// the hashed and the captured block decide alike).
static bool pdl_next(wp_ctx *c) {
  const bool p = c->pdl_scope && c->chain;
  c->chain = true;
  return p;
}

// Scope of one time loop of half-order R: programmatic launches only between its
// step kernels, as pdl_mode allows.
struct PdlScope {
  wp_ctx *c;
  PdlScope(wp_ctx *ctx, int R) : c(ctx) {
    c->pdl_scope = c->pdl_mode == 1 || (c->pdl_mode == 2 && R <= 4);
    c->chain = false;
  }
  ~PdlScope() {
    c->pdl_scope = false;
    c->chain = false;
  }
};

static int prof_mark(wp_ctx *c) {
  c->chain = false;  // an event record sits between the kernels around it
  if (!c->profiling) return WP_OK;
  if (c->hashing) {
    c->hash_marks++;
    return WP_OK;
  }
  std::vector<cudaEvent_t> &ev = *c->prof_ev;
  size_t &n = *c->prof_n;
  if (n == ev.size()) {
    cudaEvent_t e;
    CU(cudaEventCreate(&e));
    ev.push_back(e);
  }
  // inside a capture only an "external" record becomes a graph node the host can time
  if (c->capturing) CU(cudaEventRecordWithFlags(ev[n++], c->stream, cudaEventRecordExternal));
  else CU(cudaEventRecord(ev[n++], c->stream));
  return WP_OK;
}

// Fold recorded (start, end) event pairs into the totals (the events must have completed).
static int prof_fold(wp_ctx *c, const std::vector<cudaEvent_t> &ev, size_t n) {
  for (size_t i = 0; i + 1 < n; i += 2) {
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, ev[i], ev[i + 1]));
    c->prof_ms += ms;
    c->prof_count++;
  }
  return WP_OK;
}

static int prof_collect(wp_ctx *c) {
  TRY(prof_fold(c, c->prof_events, c->prof_used));
  c->prof_used = 0;
  return WP_OK;
}

// Wait (with the context deadline) for one event.
static int wait_event(wp_ctx *c, cudaEvent_t ev, const char *what) {
  const auto t0 = std::chrono::steady_clock::now();
  int spins = 0;
  while (true) {
    cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return WP_OK;
    if (e != cudaErrorNotReady) return fail(WP_ECUDA, "%s failed: %s", what, cudaGetErrorString(e));
    if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > c->timeout_s) {
      c->broken = true;
      return fail(WP_ETIMEOUT, "%s did not finish within %.1f s", what, c->timeout_s);
    }
    if (++spins > 64) std::this_thread::sleep_for(std::chrono::microseconds(spins > 1000 ? 200 : 20));
  }
}

static int prop_step(Prop &P, const Field3 &u, const Field3 &um, float *out, int mode, const Field3 *uj,
                     const Field3 *grad, bool sub = false) {
  const Geom &G = P.G;
  P.c->prof_open = P.c->profiling && (P.c->prof_seq++ % uint64_t(P.c->prof_every)) == 0;
  if (P.c->prof_open) TRY(prof_mark(P.c));
  if (G.ndim == 3) {
    // never hand the kernel a descriptor that was not encoded for its buffer
    if (!u.mapped || !um.mapped || !P.b.mapped || !P.s.mapped || (uj && !uj->mapped) || (grad && !grad->mapped))
      return fail(WP_ECUDA, "internal error: a field of the 3D stencil has no TMA descriptor");
    const bool in_box = sub && P.sub;
    const Plan3d &pl = in_box ? P.plan_sub[mode] : P.plan[mode];
    Stencil3dArgs a;
    memset(&a, 0, sizeof a);
    if (in_box) {
      a.bx0 = P.box.x0;
      a.by0 = P.box.y0;
      a.bz0 = P.box.z0;
      a.bx1 = P.box.x1;
      a.by1 = P.box.y1;
      a.bz1 = P.box.z1;
    } else {
      a.bx1 = G.nx;
      a.by1 = G.ny;
      a.bz1 = G.nz;
    }
    a.g = G.fg();
    a.c = P.lc;
    a.u = u.p;
    a.out = out;
    a.grad = grad ? grad->p : nullptr;
    a.neg_inv_dt2 = P.neg_inv_dt2;
    a.tbits = P.tbits;
    a.nzw = G.nzw;
    a.tiles_x = pl.tiles_x;
    a.tiles_y = pl.tiles_y;
    a.flag_tiles_x = G.tiles_x;
    a.flag_tiles_y = G.tiles_y;
    a.zchunk = pl.zchunk;
    a.nzc = pl.nzc;
    a.nitems = pl.nitems;
    a.err = P.c->d_scalars;
    a.wait_ns = P.c->wait_ns;
    a.pdl = pdl_next(P.c);
    const CUtensorMap maps[7] = {u.halo[mode], um.tile[mode], P.b.tile[mode], P.s.tile[mode],
                                 uj ? uj->tile[mode] : P.b.tile[mode], grad ? grad->tile[mode] : P.b.tile[mode],
                                 u.tile[mode]};
    if (P.c->hashing) {
      hash_bytes(P.c, &mode, sizeof mode);
      hash_bytes(P.c, &a, sizeof a);
      hash_bytes(P.c, maps, sizeof maps);
      hash_bytes(P.c, &pl.grid, sizeof pl.grid);
      return P.c->prof_open ? prof_mark(P.c) : WP_OK;
    }
    cudaError_t e = mode == kModeAdjGrad ? launch_stencil3d_adj(G.R, pl.grid, P.c->stream, maps, a)
                                         : launch_stencil3d_fwd(G.R, pl.grid, P.c->stream, maps, a);
    if (e != cudaSuccess) return fail(WP_ECUDA, "stencil3d launch failed: %s", cudaGetErrorString(e));
  } else {
    Stencil2dArgs a;
    memset(&a, 0, sizeof a);
    a.g = G.fg();
    a.c = P.lc;
    a.u = u.p;
    a.um = um.p;
    a.b = P.b.p;
    a.s = P.s.p;
    a.out = out;
    a.grad = grad ? grad->p : nullptr;
    a.uj = uj ? uj->p : nullptr;
    a.neg_inv_dt2 = P.neg_inv_dt2;
    a.pdl = pdl_next(P.c);
    if (P.c->hashing) {
      hash_bytes(P.c, &mode, sizeof mode);
      hash_bytes(P.c, &a, sizeof a);
      return P.c->prof_open ? prof_mark(P.c) : WP_OK;
    }
    cudaError_t e = launch_stencil2d(G.R, mode, P.c->stream, a);
    if (e != cudaSuccess) return fail(WP_ECUDA, "stencil2d launch failed: %s", cudaGetErrorString(e));
  }
  P.c->launches++;
  if (P.c->prof_open) TRY(prof_mark(P.c));
  if (!P.c->capturing && P.c->prof_used >= 4096) {  // bound the event pool: fold what has completed
    TRY(ctx_wait(P.c));
    TRY(prof_collect(P.c));
  }
  return WP_OK;
}

static int prop_inject(Prop &P, const DevPoints &dp, const float *data, long long row, float *u, float *grad,
                       const float *uj, const long long *row_base = nullptr) {
  if (dp.ntarget == 0) return WP_OK;
  InjectArgs a;
  memset(&a, 0, sizeof a);
  a.ntarget = dp.ntarget;
  a.target = dp.target;
  a.rowptr = dp.rowptr;
  a.pid = dp.pid;
  a.w = dp.cw;
  a.data = data;
  a.npts = dp.npts;
  a.row_base = row_base;
  a.row = row;
  a.u = u;
  a.b = P.b.p;
  a.grad = grad;
  a.uj = uj;
  a.neg_inv_dt2 = P.neg_inv_dt2;
  a.nfield = P.G.nfield;
  a.err = P.c->d_scalars;
  a.pdl = pdl_next(P.c);
  if (P.c->hashing) {
    hash_bytes(P.c, &a, sizeof a);
    return WP_OK;
  }
  CU(launch_inject(P.c->stream, a));
  P.c->launches++;
  return WP_OK;
}

static int prop_sample(Prop &P, const DevPoints &dp, const float *u, float *out, long long row,
                       const long long *row_base = nullptr) {
  if (dp.npts == 0) return WP_OK;
  InterpArgs a;
  memset(&a, 0, sizeof a);
  a.npts = dp.npts;
  a.ncorner = dp.nc;
  a.idx = dp.idx;
  a.w = dp.w;
  a.u = u;
  a.out = out;
  a.row_base = row_base;
  a.row = row;
  a.nfield = P.G.nfield;
  a.err = P.c->d_scalars;
  a.pdl = pdl_next(P.c);
  if (P.c->hashing) {
    hash_bytes(P.c, &a, sizeof a);
    return WP_OK;
  }
  CU(launch_interp(P.c->stream, a));
  P.c->launches++;
  return WP_OK;
}

static int prop_add_row(wp_ctx *c, long long *p, long long d) {
  const bool pdl = pdl_next(c);
  if (c->hashing) {
    hash_bytes(c, &p, sizeof p);
    hash_bytes(c, &d, sizeof d);
    hash_bytes(c, &pdl, sizeof pdl);
    return WP_OK;
  }
  CU(launch_add_row(c->stream, p, d, pdl));
  c->launches++;
  return WP_OK;
}

// Run `block` (a callable that enqueues one block of work through the helpers
// above) `replays` times as a cached CUDA graph.  The block is first run in
// hashing mode; a cached graph with the same hash is replayed, otherwise the
// block is captured and instantiated (at most 16 graphs per context, least
// recently used evicted).  With profiling on, the stencil event pairs inside the
// graph are folded after every replay.
template <class F>
static int graph_replay(wp_ctx *c, F &&block, int replays) {
  if (replays <= 0) return WP_OK;
  c->hashing = true;
  c->hash = 1469598103934665603ull ^ (c->profiling ? 0x9e3779b97f4a7c15ull : 0ull);
  c->hash_marks = 0;
  const uint64_t seq0 = c->prof_seq;
  c->prof_seq = 0;
  c->chain = false;  // a graph's first kernel has no kernel before it inside the graph
  int rc = block();
  c->hashing = false;
  TRY(rc);
  const uint64_t key = c->hash;
  GraphEntry *e = nullptr;
  for (GraphEntry *g : c->graphs)
    if (g->key == key) e = g;
  if (!e) {
    e = new GraphEntry();
    e->key = key;
    for (size_t i = 0; i < c->hash_marks; ++i) {  // events exist before capture starts
      cudaEvent_t ev;
      if (cudaEventCreate(&ev) != cudaSuccess) {
        graph_destroy(e);
        return fail(WP_ECUDA, "cudaEventCreate failed");
      }
      e->ev.push_back(ev);
    }
    std::vector<cudaEvent_t> *sev = c->prof_ev;
    size_t *sn = c->prof_n;
    c->prof_ev = &e->ev;
    c->prof_n = &e->nev;
    const uint64_t l0 = c->launches;
    c->capturing = true;
    cudaGraph_t g = nullptr;
    c->prof_seq = 0;
    c->chain = false;
    cudaError_t be = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    int brc = be == cudaSuccess ? block() : WP_OK;
    cudaError_t ee = be == cudaSuccess ? cudaStreamEndCapture(c->stream, &g) : be;
    c->capturing = false;
    c->prof_ev = sev;
    c->prof_n = sn;
    e->kernels = c->launches - l0;
    c->launches = l0;
    cudaError_t ie = cudaSuccess;
    if (brc == WP_OK && ee == cudaSuccess) ie = cudaGraphInstantiate(&e->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (brc != WP_OK || ee != cudaSuccess || ie != cudaSuccess) {
      graph_destroy(e);
      if (brc != WP_OK) return brc;
      return fail(WP_ECUDA, "graph capture failed: %s", cudaGetErrorString(ee != cudaSuccess ? ee : ie));
    }
    if (c->graphs.size() >= 16) {
      auto it = std::min_element(c->graphs.begin(), c->graphs.end(),
                                 [](GraphEntry *x, GraphEntry *y) { return x->stamp < y->stamp; });
      graph_destroy(*it);
      c->graphs.erase(it);
    }
    c->graphs.push_back(e);
  }
  c->prof_seq = seq0;
  e->stamp = ++c->graph_stamp;
  c->chain = false;  // the work after the replays follows a graph launch
  for (int r = 0; r < replays; ++r) {
    CU(cudaGraphLaunch(e->exec, c->stream));
    c->launches += e->kernels;
    if (c->profiling && e->nev) {
      TRY(wait_event(c, e->ev[e->nev - 1], "graph replay"));
      TRY(prof_fold(c, e->ev, e->nev));
    }
  }
  return WP_OK;
}

// Steps per graph replay: an even block of 8..64 steps leaving the smallest
// remainder (0 for loops too short to be worth a graph).
static int graph_block(wp_ctx *c, int nt) {
  if (!c->use_graphs || nt < 16) return 0;
  int best = 0, best_rem = nt;
  for (int B = 64; B >= 8; B -= 2) {
    const int rem = nt % B;
    if (rem < best_rem) {
      best = B;
      best_rem = rem;
    }
  }
  return best;
}

static int alloc_field(Arena &ar, const Geom &G, Field3 *f, bool zero, cudaStream_t st) {
  TRY(ar.alloc(&f->p, G.nfield));
  if (zero) CU(cudaMemsetAsync(f->p, 0, G.field_bytes(), st));
  TRY(make_field_maps(f, G));
  return WP_OK;
}

// Time loop shared by forward and adjoint: for k = 0..nt-1 one update, inject
// data row (dir > 0 ? k : nt-1-k) at `inj`, sample `smp` into the same row of
// `out`.  u[k & 1] holds the current level before step k.  Full blocks of B
// steps run as replays of one CUDA graph (B even, so buffer parity repeats);
// the sparse kernels take their row from a device base the graph advances.
static int run_loop(Prop &P, Field3 u[2], int nt, const DevPoints &inj, const float *data, const DevPoints &smp,
                    float *out, int dir) {
  wp_ctx *c = P.c;
  PdlScope pdl_scope(c, P.G.R);
  int k0 = 0;
  const int B = graph_block(c, nt);
  auto one_step = [&](int k, long long row, const long long *rb) -> int {
    Field3 &cur = u[k & 1], &prv = u[(k + 1) & 1];
    TRY(prop_step(P, cur, prv, prv.p, kModeFwd, nullptr, nullptr));
    TRY(prop_inject(P, inj, data, row, prv.p, nullptr, nullptr, rb));
    if (out) TRY(prop_sample(P, smp, prv.p, out, row, rb));
    return WP_OK;
  };
  if (B > 0) {
    long long *rb = c->d_rows;
    CU(launch_set_row(c->stream, rb, dir > 0 ? 0 : nt - 1, pdl_next(c)));
    c->launches++;
    auto block = [&]() -> int {
      for (int j = 0; j < B; ++j) TRY(one_step(j, dir * j, rb));
      return prop_add_row(c, rb, static_cast<long long>(dir) * B);
    };
    TRY(graph_replay(c, block, nt / B));
    k0 = (nt / B) * B;
  }
  for (int k = k0; k < nt; ++k) TRY(one_step(k, dir > 0 ? k : nt - 1 - k, nullptr));
  return WP_OK;
}

// ---------------------------------------------------------------------------
// common call prologue
// ---------------------------------------------------------------------------
static int enter(wp_ctx *c, void *user_stream) {
  if (!c) return fail(WP_EINVAL, "context is NULL");
  if (c->broken) return fail(WP_ETIMEOUT, "context unusable after an earlier timeout");
  CU(cudaSetDevice(c->device));
  cudaStream_t us = static_cast<cudaStream_t>(user_stream);
  CU(cudaEventRecord(c->ev_in, us));
  CU(cudaStreamWaitEvent(c->stream, c->ev_in, 0));
  CU(cudaMemsetAsync(c->d_scalars, 0, 4 * sizeof(int), c->stream));
  return WP_OK;
}

static int leave(wp_ctx *c, void *user_stream, int rc) {
  if (rc == WP_OK) rc = check_device_error(c);
  if (rc == WP_OK && c->profiling) rc = prof_collect(c);
  if (rc != WP_OK && c) c->prof_used = 0;
  if (rc != WP_ETIMEOUT && c && !c->broken) {
    // order the caller's later work after ours (normally complete already)
    if (cudaEventRecord(c->ev_done, c->stream) == cudaSuccess)
      cudaStreamWaitEvent(static_cast<cudaStream_t>(user_stream), c->ev_done, 0);
    if (rc != WP_OK) cudaStreamSynchronize(c->stream);
  }
  return rc;
}

// Device-array arguments must be device (or managed) memory of `device`: a host
// pointer, or memory of another GPU, would be dereferenced by every kernel of
// the call.  NULL passes (the callers check which arrays are required).
struct DevArg {
  const void *p;
  const char *what;
};
static int check_dev_args(int device, std::initializer_list<DevArg> args) {
  for (const DevArg &a : args) {
    if (!a.p) continue;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, a.p);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(WP_EINVAL, "%s is not a CUDA device address (%s)", a.what, cudaGetErrorString(e));
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
      return fail(WP_EINVAL, "%s must be device memory (a host pointer was passed to a device-array call)", a.what);
    if (at.type == cudaMemoryTypeDevice && at.device != device)
      return fail(WP_EINVAL, "%s lives on device %d, the call runs on device %d", a.what, at.device, device);
  }
  return WP_OK;
}

// In an entry point after enter(): reject bad device-array arguments through leave().
#define DEV_ARGS(ctx, stream, ...)                                \
  do {                                                            \
    int rc_ = check_dev_args((ctx)->device, __VA_ARGS__);         \
    if (rc_ != WP_OK) return leave((ctx), (stream), rc_);         \
  } while (0)

static bool all_finite(const float *x, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(x[i])) return false;
  return true;
}

// ---------------------------------------------------------------------------
// forward / adjoint
// ---------------------------------------------------------------------------
// host_io: inputs/outputs are host pointers (copied in/out); otherwise device.
static int do_propagate(wp_ctx *c, const wp_grid *grid, const float *m, const float *eta, const float *inj_data,
                        int ninj, const double *inj_xyz, int nsmp, const double *smp_xyz, float *smp_out, int dir,
                        bool host_io) {
  NvtxRange range(dir > 0 ? "wp.forward" : "wp.adjoint");
  Geom G;
  TRY(make_geom(grid, &G));
  if (ninj < 0 || nsmp < 0) return fail(WP_EINVAL, "point counts must be >= 0");
  if (!m || !eta) return fail(WP_EINVAL, "m and eta must not be NULL");
  if (ninj > 0 && G.nt > 0 && !inj_data) return fail(WP_EINVAL, "injected data is NULL");
  if (nsmp > 0 && G.nt > 0 && !smp_out) return fail(WP_EINVAL, "output array is NULL");
  PointSet pin, psm;
  TRY(build_points(G, ninj, inj_xyz, &pin, dir > 0 ? "source" : "receiver"));
  TRY(build_points(G, nsmp, smp_xyz, &psm, dir > 0 ? "receiver" : "source"));
  const size_t n_in = size_t(G.nt) * ninj, n_out = size_t(G.nt) * nsmp;
  if (host_io && n_in && !all_finite(inj_data, n_in)) return fail(WP_ENONFINITE, "injected data holds NaN or Inf");

  Arena ar(c);
  Field3 u[2];
  TRY(alloc_field(ar, G, &u[0], false, c->stream));
  TRY(alloc_field(ar, G, &u[1], false, c->stream));
  const float *md = m, *ed = eta;
  if (host_io) {  // stage m, eta contiguously in the wavefield buffers
    CU(cudaMemcpyAsync(u[0].p, m, G.npoints * 4, cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemcpyAsync(u[1].p, eta, G.npoints * 4, cudaMemcpyHostToDevice, c->stream));
    md = u[0].p;
    ed = u[1].p;
  }
  Prop P;
  TRY(prop_setup(c, ar, G, md, ed, &P));
  CU(cudaMemsetAsync(u[0].p, 0, G.field_bytes(), c->stream));
  CU(cudaMemsetAsync(u[1].p, 0, G.field_bytes(), c->stream));
  DevPoints din, dsm;
  TRY(upload_points(c, ar, pin, false, true, &din));
  TRY(upload_points(c, ar, psm, true, false, &dsm));
  const float *data_d = inj_data;
  float *out_d = smp_out;
  if (host_io) {
    float *tmp_in = nullptr, *tmp_out = nullptr;
    if (n_in) {
      TRY(ar.alloc(&tmp_in, n_in));
      CU(cudaMemcpyAsync(tmp_in, inj_data, n_in * 4, cudaMemcpyHostToDevice, c->stream));
    }
    if (n_out) TRY(ar.alloc(&tmp_out, n_out));
    data_d = tmp_in;
    out_d = tmp_out;
  } else if (n_in) {
    int *bad = c->d_scalars + 1;
    CU(cudaMemsetAsync(bad, 0, sizeof(int), c->stream));
    CU(launch_check_finite(c->stream, inj_data, (long long)n_in, bad));
    c->launches++;
    CU(cudaMemcpyAsync(c->h_scalars + 1, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    TRY(ctx_wait(c));
    if (c->h_scalars[1]) return fail(WP_ENONFINITE, "injected data holds NaN or Inf");
  }
  TRY(run_loop(P, u, G.nt, din, data_d, dsm, n_out ? out_d : nullptr, dir));
  for (int i = 0; i < 2; ++i) CU(launch_check_padding(c->stream, u[i].p, G.fg(), c->d_scalars));
  if (host_io && n_out) CU(cudaMemcpyAsync(smp_out, out_d, n_out * 4, cudaMemcpyDeviceToHost, c->stream));
  return ctx_wait(c, dir > 0 ? "forward time loop" : "adjoint time loop");
}

// ---------------------------------------------------------------------------
// gradient: forward with snapshots, backward with recompute + fused gradient
// ---------------------------------------------------------------------------
struct wp_state {
  wp_ctx *c = nullptr;
  Geom G;
  Prop P;
  std::vector<void *> mem;     // device blocks owned by the state
  float *snaps = nullptr;      // [nseg][2][nfield]: (u^{sS-1}, u^{sS}); S = 1: [nt][nfield] = u^1..u^nt
  int S = 0, nseg = 0;
  std::vector<Field3> hist;    // S = 1: level j (1..nt) at hist[j-1], with its own descriptors
  std::vector<Field3> snapf;   // S > 1: the snapshot levels, [2 s] = u^{sS-1}, [2 s + 1] = u^{sS}
  PointSet psrc, prec;
  DevPoints dsrc, drec;
  float *wavelet = nullptr;    // [nt][nsrc] device copy
};

static void state_release(wp_state *st) {
  if (!st) return;
  for (void *p : st->mem) dev_free(st->c, p);
  st->mem.clear();
}

// host_in: m, eta and the wavelet are host arrays; host_rec: rec_out is a host array.
static int forward_save(wp_ctx *c, const wp_grid *grid, const float *m, const float *eta, const float *wavelet,
                        int nsrc, const double *src_xyz, int nrec, const double *rec_xyz, int snap_interval,
                        float *rec_out, bool host_in, bool host_rec, wp_state **out) {
  NvtxRange range("wp.forward_save");
  const bool host_io = host_in;
  *out = nullptr;
  wp_state *st = new wp_state();
  st->c = c;
  int rc = [&]() -> int {
    Geom &G = st->G;
    TRY(make_geom(grid, &G));
    if (nsrc < 0 || nrec < 0) return fail(WP_EINVAL, "point counts must be >= 0");
    if (!m || !eta) return fail(WP_EINVAL, "m and eta must not be NULL");
    if (nsrc > 0 && G.nt > 0 && !wavelet) return fail(WP_EINVAL, "wavelet is NULL");
    if (snap_interval < 0) return fail(WP_EINVAL, "snap_interval must be >= 0");
    if (snap_interval == 0) {
      // automatic: the whole history if it fits the budget left, else the smallest
      // snapshot interval that fits (fields: state + snapshots + recompute ring +
      // adjoint and gradient, with 5 % headroom)
      const double f = double(round_up(G.field_bytes(), 256));
      const double avail = 0.95 * (double(c->budget) - double(c->in_use)) - 8.0 * f;
      auto need = [&](int S) -> double {
        if (S == 1) return (double(G.nt) + 5.0) * f;
        const double nseg = std::ceil(double(G.nt) / S);
        return (2.0 * nseg + std::min(S, std::max(G.nt, 1)) + 5.0) * f;
      };
      int S = 1;
      while (S <= std::max(G.nt, 1) && need(S) > avail) S = S == 1 ? 2 : S + std::max(1, S / 4);
      if (S > std::max(G.nt, 1)) return fail(WP_ENOMEM, "no snapshot interval fits the device budget");
      snap_interval = S;
    }
    st->S = snap_interval;
    st->nseg = (G.nt + st->S - 1) / st->S;
    TRY(build_points(G, nsrc, src_xyz, &st->psrc, "source"));
    TRY(build_points(G, nrec, rec_xyz, &st->prec, "receiver"));
    const size_t n_in = size_t(G.nt) * nsrc, n_out = size_t(G.nt) * nrec;
    if (host_io && n_in && !all_finite(wavelet, n_in)) return fail(WP_ENONFINITE, "wavelet holds NaN or Inf");
    Arena keep(c);   // memory owned by the state
    Arena tmp(c);    // memory of this call only
    Field3 u[2];
    TRY(alloc_field(tmp, G, &u[0], false, c->stream));
    TRY(alloc_field(tmp, G, &u[1], false, c->stream));
    const float *md = m, *ed = eta;
    if (host_io) {
      CU(cudaMemcpyAsync(u[0].p, m, G.npoints * 4, cudaMemcpyHostToDevice, c->stream));
      CU(cudaMemcpyAsync(u[1].p, eta, G.npoints * 4, cudaMemcpyHostToDevice, c->stream));
      md = u[0].p;
      ed = u[1].p;
    }
    TRY(prop_setup(c, keep, G, md, ed, &st->P));
    CU(cudaMemsetAsync(u[0].p, 0, G.field_bytes(), c->stream));
    CU(cudaMemsetAsync(u[1].p, 0, G.field_bytes(), c->stream));
    TRY(upload_points(c, keep, st->psrc, false, true, &st->dsrc));
    TRY(upload_points(c, keep, st->prec, true, true, &st->drec));
    if (n_in) {
      TRY(keep.alloc(&st->wavelet, n_in));
      CU(cudaMemcpyAsync(st->wavelet, wavelet, n_in * 4, host_io ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                         c->stream));
      if (!host_io) {
        int *bad = c->d_scalars + 1;
        CU(cudaMemsetAsync(bad, 0, sizeof(int), c->stream));
        CU(launch_check_finite(c->stream, st->wavelet, (long long)n_in, bad));
        c->launches++;
        CU(cudaMemcpyAsync(c->h_scalars + 1, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        TRY(ctx_wait(c));
        if (c->h_scalars[1]) return fail(WP_ENONFINITE, "wavelet holds NaN or Inf");
      }
    }
    // S = 1 keeps the whole history once (each level written in place of a copy);
    // otherwise snapshot pairs every S steps
    if (st->S == 1 && G.nt > 0) {
      TRY(keep.alloc(&st->snaps, size_t(G.nt) * G.nfield));
      st->hist.resize(size_t(G.nt));
      for (int j = 0; j < G.nt; ++j) {
        st->hist[size_t(j)].p = st->snaps + size_t(j) * G.nfield;
        TRY(make_field_maps(&st->hist[size_t(j)], G));
      }
    } else if (st->nseg > 0) {
      // the step that produces a snapshot level writes it there, and the backward
      // pass reads it in place: no copies
      TRY(keep.alloc(&st->snaps, size_t(st->nseg) * 2 * G.nfield));
      st->snapf.resize(2 * size_t(st->nseg));
      for (size_t i = 0; i < st->snapf.size(); ++i) {
        st->snapf[i].p = st->snaps + i * G.nfield;
        TRY(make_field_maps(&st->snapf[i], G));
      }
      CU(cudaMemsetAsync(st->snapf[0].p, 0, G.field_bytes(), c->stream));  // u^{-1} = u^0 = 0
      CU(cudaMemsetAsync(st->snapf[1].p, 0, G.field_bytes(), c->stream));
    }
    float *rec_d = nullptr;
    if (rec_out && n_out) {
      if (host_rec) TRY(tmp.alloc(&rec_d, n_out));
      else rec_d = rec_out;
    }
    Prop &P = st->P;
    // level k of the full history: u^{-1}, u^0 in the zeroed work fields
    auto lev = [&](int k) -> Field3 & { return k == -1 ? u[0] : k == 0 ? u[1] : st->hist[size_t(k - 1)]; };
    // S > 1: level k is snapshot slot 2 s if k = sS - 1, 2 s + 1 if k = sS, else
    // the work field u[k & 1] (a level there is dead when k + 2 overwrites it)
    const int S = st->S;
    auto snap_slot = [&](int k) -> int {
      if ((k + 1) % S == 0 && (k + 1) / S < st->nseg) return 2 * ((k + 1) / S);
      if (k >= 0 && k % S == 0 && k / S < st->nseg) return 2 * (k / S) + 1;
      return -1;
    };
    auto slev = [&](int k) -> Field3 & {
      const int i = snap_slot(k);
      return i >= 0 ? st->snapf[size_t(i)] : u[k & 1];
    };
    auto step = [&](Field3 &cur, Field3 &prv, Field3 &nxt, int n) -> int {
      TRY(prop_step(P, cur, prv, nxt.p, kModeFwd, nullptr, nullptr));
      TRY(prop_inject(P, st->dsrc, st->wavelet, n, nxt.p, nullptr, nullptr));
      if (rec_d) TRY(prop_sample(P, st->drec, nxt.p, rec_d, n));
      return WP_OK;
    };
    {
      PdlScope pdl_scope(c, G.R);
      for (int n = 0; S == 1 && n < G.nt; ++n) TRY(step(lev(n), lev(n - 1), lev(n + 1), n));
      for (int n = 0; S > 1 && n < G.nt; ++n) TRY(step(slev(n), slev(n - 1), slev(n + 1), n));
    }
    if (host_rec && rec_d) CU(cudaMemcpyAsync(rec_out, rec_d, n_out * 4, cudaMemcpyDeviceToHost, c->stream));
    TRY(ctx_wait(c, "forward with snapshots"));
    keep.release_all_to(st->mem);
    return WP_OK;
  }();
  if (rc != WP_OK) {
    state_release(st);
    delete st;
    return rc;
  }
  *out = st;
  return WP_OK;
}

// host_res: the residual is a host array; host_grad: grad_out is a host array.
static int backward(wp_state *st, const float *residual, float *grad_out, bool host_res, bool host_grad) {
  NvtxRange range("wp.backward");
  const bool host_io = host_res;
  wp_ctx *c = st->c;
  const Geom &G = st->G;
  Prop &P = st->P;
  const int nrec = st->drec.npts;
  const size_t n_res = size_t(G.nt) * nrec;
  if (n_res && !residual) return fail(WP_EINVAL, "residual is NULL");
  if (!grad_out) return fail(WP_EINVAL, "grad_out is NULL");
  if (host_io && n_res && !all_finite(residual, n_res)) return fail(WP_ENONFINITE, "residual holds NaN or Inf");
  Arena tmp(c);
  const float *res_d = residual;
  if (n_res) {
    float *r = nullptr;
    if (host_io) {
      TRY(tmp.alloc(&r, n_res));
      CU(cudaMemcpyAsync(r, residual, n_res * 4, cudaMemcpyHostToDevice, c->stream));
      res_d = r;
    } else {
      int *bad = c->d_scalars + 1;
      CU(cudaMemsetAsync(bad, 0, sizeof(int), c->stream));
      CU(launch_check_finite(c->stream, residual, (long long)n_res, bad));
      c->launches++;
      CU(cudaMemcpyAsync(c->h_scalars + 1, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
      TRY(ctx_wait(c));
      if (c->h_scalars[1]) return fail(WP_ENONFINITE, "residual holds NaN or Inf");
    }
  }
  const int S = st->S;
  if (S == 1) {  // full history: no recomputation
    Field3 w[2], g;
    TRY(alloc_field(tmp, G, &w[0], true, c->stream));
    TRY(alloc_field(tmp, G, &w[1], true, c->stream));
    TRY(alloc_field(tmp, G, &g, true, c->stream));
    for (long long j = G.nt, kadj = 0; j >= 1; --j, ++kadj) {
      Field3 &w1 = w[kadj & 1], &w2 = w[(kadj + 1) & 1];
      const Field3 &uj = st->hist[size_t(j - 1)];
      TRY(prop_step(P, w1, w2, w2.p, kModeAdjGrad, &uj, &g));
      TRY(prop_inject(P, st->drec, res_d, int(j - 1), w2.p, g.p, uj.p));
    }
    CU(cudaMemcpy2DAsync(grad_out, size_t(G.nx) * 4, g.p, size_t(G.pitch) * 4, size_t(G.nx) * 4,
                         size_t(G.ny) * G.nz, host_grad ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                         c->stream));
    return ctx_wait(c, "backward (adjoint, gradient from the full history)");
  }
  // ring[2 ..] receive the recomputed levels; [0], [1] stand for the segment's
  // snapshot pair, read in place
  std::vector<Field3> ring(size_t(std::min(S, std::max(G.nt, 1))) + 2);
  for (size_t i = 2; i < ring.size(); ++i) TRY(alloc_field(tmp, G, &ring[i], false, c->stream));
  Field3 w[2], g;
  TRY(alloc_field(tmp, G, &w[0], true, c->stream));
  TRY(alloc_field(tmp, G, &w[1], true, c->stream));
  TRY(alloc_field(tmp, G, &g, true, c->stream));
  long long kadj = 0;  // adjoint steps done: w^{j+1} in w[kadj & 1]
  PdlScope pdl_scope(c, G.R);  // only step kernels are enqueued until the copy-out below
  for (int s = st->nseg - 1; s >= 0; --s) {
    const int s0 = s * S;
    const int len = std::min(S, G.nt - s0);
    ring[0] = st->snapf[2 * size_t(s)];
    ring[1] = st->snapf[2 * size_t(s) + 1];
    {
      NvtxRange rr("wp.recompute");
      for (int i = 0; i < len; ++i) {  // recompute u^{s0+1} .. u^{s0+len} into ring[2..]
        TRY(prop_step(P, ring[i + 1], ring[i], ring[i + 2].p, kModeFwd, nullptr, nullptr));
        TRY(prop_inject(P, st->dsrc, st->wavelet, s0 + i, ring[i + 2].p, nullptr, nullptr));
      }
    }
    NvtxRange ra("wp.adjoint_gradient");
    for (int j = s0 + len; j >= s0 + 1; --j, ++kadj) {
      Field3 &w1 = w[kadj & 1], &w2 = w[(kadj + 1) & 1];
      const Field3 &uj = ring[j - s0 + 1];
      TRY(prop_step(P, w1, w2, w2.p, kModeAdjGrad, &uj, &g));
      TRY(prop_inject(P, st->drec, res_d, j - 1, w2.p, g.p, uj.p));
    }
  }
  // pitched -> contiguous
  c->chain = false;
  CU(cudaMemcpy2DAsync(grad_out, size_t(G.nx) * 4, g.p, size_t(G.pitch) * 4, size_t(G.nx) * 4,
                       size_t(G.ny) * G.nz, host_grad ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->stream));
  return ctx_wait(c, "backward (recompute, adjoint, gradient)");
}

// ---------------------------------------------------------------------------
// Binomial checkpointing (optimal reversal with a fixed number of stored states)
// ---------------------------------------------------------------------------
// State k is the pair (u^{k-1}, u^k); the adjoint step j needs state j.  With the
// start state a stored and c free slots, n adjoint steps (j = a+n .. a+1) are
// reversed either directly (n = 1: advance one step; c = 0: for each j advance
// from a) or by advancing m steps, storing state a+m, reversing the upper n-m
// steps with c-1 slots and then the lower m steps from a again.  The cost (forward
// steps, one more for each store) obeys
//     T(n, c) = min_m  m + 1 + T(n-m, c-1) + T(m, c),   T(1, c) = 1,   T(n, 0) = n(n+1)/2,
// which is minimised by dynamic programming; the smallest optimal m is
// nondecreasing in n, so each row is found by a forward scan.
enum CkKind : int { kCkAdvance = 0, kCkStore = 1, kCkAdjoint = 2 };
struct CkOp {
  int kind, a, b, slot;  // advance: slot holding state a -> state b; store: state a -> slot; adjoint: j = a
};

struct CkTable {
  int nt = 0, c = 0;
  std::vector<long long> T;  // (nt+1) x (c+1)
  std::vector<int> opt;
  long long &t(int n, int k) { return T[size_t(n) * (c + 1) + k]; }
  int &o(int n, int k) { return opt[size_t(n) * (c + 1) + k]; }
};

static void ck_build(CkTable &tb, int nt, int c) {
  tb.nt = nt;
  tb.c = c;
  tb.T.assign(size_t(nt + 1) * (c + 1), 0);
  tb.opt.assign(size_t(nt + 1) * (c + 1), 0);
  for (int n = 0; n <= nt; ++n) tb.t(n, 0) = static_cast<long long>(n) * (n + 1) / 2;
  for (int k = 1; k <= c; ++k) {
    if (nt >= 1) tb.t(1, k) = 1;
    int lo = 1;
    for (int n = 2; n <= nt; ++n) {
      long long best = tb.t(n, k - 1);  // using fewer slots is always possible
      int bm = 0;
      int rises = 0;
      for (int m = lo; m < n; ++m) {
        const long long v = m + 1 + tb.t(n - m, k - 1) + tb.t(m, k);
        if (v < best || (bm == 0 && v == best)) {
          best = v;
          bm = m;
          rises = 0;
        } else if (bm && ++rises > 16) {
          break;
        }
      }
      tb.t(n, k) = best;
      tb.o(n, k) = bm;  // 0: do not split at this level
      if (bm) lo = bm;
    }
  }
}

// Op list reversing all nt steps from state 0 (slot 0) with `c` free slots 1..c.
static void ck_schedule(CkTable &tb, std::vector<CkOp> &ops) {
  std::vector<int> free_slots;
  for (int k = tb.c; k >= 1; --k) free_slots.push_back(k);
  // explicit recursion on the upper part (depth <= c); the lower part loops
  std::function<void(int, int, int)> rev = [&](int a, int n, int slot) {
    while (n > 0) {
      // best split with at most the free slots (0: none pays off)
      int m = 0;
      for (int k = std::min(static_cast<int>(free_slots.size()), tb.c); n >= 2 && k >= 1 && !m; --k) m = tb.o(n, k);
      if (n == 1 || m == 0) {
        for (int i = n; i >= 1; --i) {
          ops.push_back({kCkAdvance, a, a + i, slot});
          ops.push_back({kCkAdjoint, a + i, 0, 0});
        }
        return;
      }
      const int t = free_slots.back();
      free_slots.pop_back();
      ops.push_back({kCkAdvance, a, a + m, slot});
      ops.push_back({kCkStore, a + m, 0, t});
      rev(a + m, n - m, t);
      free_slots.push_back(t);
      n = m;
    }
  };
  rev(0, tb.nt, 0);
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char *wp_last_error(void) { return g_err.c_str(); }

int wp_create(wp_ctx **out, int device, size_t budget) {
  if (!out) return fail(WP_EINVAL, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  CU(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(WP_EINVAL, "device %d not present (%d devices)", device, ndev);
  CU(cudaSetDevice(device));
  wp_ctx *c = new wp_ctx();
  c->device = device;
  int rc = [&]() -> int {
    CU(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device));
    size_t fr = 0, tot = 0;
    CU(cudaMemGetInfo(&fr, &tot));
    c->budget = budget == WP_BUDGET_AUTO ? size_t(0.9 * double(fr)) : budget;
    CU(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    CU(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
    CU(cudaEventCreateWithFlags(&c->ev_done, cudaEventDisableTiming));
    CU(cudaMalloc(&c->d_scalars, 64));
    CU(cudaMalloc(&c->d_rows, 64));
    c->prof_ev = &c->prof_events;
    c->prof_n = &c->prof_used;
    const char *ng = getenv("WP_NO_GRAPHS");
    c->use_graphs = !(ng && atoi(ng) != 0);
    const char *np = getenv("WP_PDL");
    if (np) c->pdl_mode = atoi(np) == 0 ? 0 : atoi(np) == 1 ? 1 : 2;
    CU(cudaMallocHost(&c->h_scalars, 64));
    CU(cudaMemset(c->d_scalars, 0, 64));
    TRY(get_encode());
    for (int R = 1; R <= 8; ++R) {
      CU(prepare_stencil3d_fwd(R, &c->smem3d[0][R], &c->occ3d[0][R], &c->ty3d[0][R]));
      CU(prepare_stencil3d_adj(R, &c->smem3d[1][R], &c->occ3d[1][R], &c->ty3d[1][R]));
    }
    return WP_OK;
  }();
  if (rc != WP_OK) {
    wp_destroy(c);
    return rc;
  }
  *out = c;
  return WP_OK;
}

void wp_destroy(wp_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream && !c->broken) cudaStreamSynchronize(c->stream);
  for (wp_state *st : c->states) {
    state_release(st);
    st->c = nullptr;
  }
  c->states.clear();
  for (auto &kv : c->live) cudaFreeAsync(kv.first, c->stream);
  for (auto &kv : c->cache) cudaFreeAsync(kv.second, c->stream);
  if (c->stream && !c->broken) cudaStreamSynchronize(c->stream);
  if (c->d_scalars) cudaFree(c->d_scalars);
  if (c->h_scalars) cudaFreeHost(c->h_scalars);
  for (cudaEvent_t e : c->prof_events) cudaEventDestroy(e);
  for (GraphEntry *g : c->graphs) graph_destroy(g);
  if (c->d_rows) cudaFree(c->d_rows);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_done) cudaEventDestroy(c->ev_done);
  if (c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

int wp_set_timeout(wp_ctx *c, double seconds) {
  if (!c || !(seconds > 0)) return fail(WP_EINVAL, "bad context or timeout");
  c->timeout_s = seconds;
  return WP_OK;
}

// ---------------------------------------------------------------------------
// CFD examples of Sec. 5 (2D, FP32): convection, Burgers' equation, Poisson
// ---------------------------------------------------------------------------
static int cfd_args(int nx, int ny, double dx, double dy, int steps) {
  if (nx < 3 || ny < 3 || nx > (1 << 24) || ny > (1 << 24)) return fail(WP_EINVAL, "nx and ny must be in [3, 2^24]");
  if (!(dx > 0) || !(dy > 0) || !std::isfinite(dx) || !std::isfinite(dy))
    return fail(WP_EINVAL, "dx and dy must be positive and finite");
  if (steps < 0) return fail(WP_EINVAL, "the number of steps must be >= 0");
  return WP_OK;
}

// stage n floats from the caller into dst, checking them for NaN/Inf
static int cfd_stage(wp_ctx *c, float *dst, const float *src, size_t n, bool host_io, const char *what) {
  if (!src) return fail(WP_EINVAL, "%s is NULL", what);
  if (host_io) {
    if (!all_finite(src, n)) return fail(WP_ENONFINITE, "%s holds NaN or Inf", what);
    CU(cudaMemcpyAsync(dst, src, n * 4, cudaMemcpyHostToDevice, c->stream));
    return WP_OK;
  }
  CU(cudaMemcpyAsync(dst, src, n * 4, cudaMemcpyDeviceToDevice, c->stream));
  int *bad = c->d_scalars + 1;
  CU(cudaMemsetAsync(bad, 0, sizeof(int), c->stream));
  CU(launch_check_finite(c->stream, dst, static_cast<long long>(n), bad));
  c->launches++;
  CU(cudaMemcpyAsync(c->h_scalars + 1, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  TRY(ctx_wait(c, "input check"));
  if (c->h_scalars[1]) return fail(WP_ENONFINITE, "%s holds NaN or Inf", what);
  return WP_OK;
}

static int convection_impl(wp_ctx *c, int nx, int ny, double dx, double dy, double dt, double cs, int nt,
                           const float *u0, float *u_out, bool host_io) {
  TRY(cfd_args(nx, ny, dx, dy, nt));
  if (!u_out) return fail(WP_EINVAL, "u_out is NULL");
  if (!(dt >= 0) || !std::isfinite(dt) || !std::isfinite(cs)) return fail(WP_EINVAL, "dt and c must be finite, dt >= 0");
  const double sx = cs * dt / dx, sy = cs * dt / dy;
  if (cs < 0 || sx + sy > 1.0 + 1e-12)
    return fail(WP_ECFL, "upwind convection needs c >= 0 and c dt/dx + c dt/dy <= 1 (got %.6g)", sx + sy);
  const size_t n = size_t(nx) * ny;
  Arena ar(c);
  float *f[2];
  TRY(ar.alloc(&f[0], n));
  TRY(ar.alloc(&f[1], n));
  TRY(cfd_stage(c, f[0], u0, n, host_io, "u0"));
  for (int k = 0; k < nt; ++k) {
    CU(launch_convection(c->stream, f[k & 1], f[(k + 1) & 1], nx, ny, float(sx), float(sy)));
    c->launches++;
  }
  CU(cudaMemcpyAsync(u_out, f[nt & 1], n * 4, host_io ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                     c->stream));
  return ctx_wait(c, "convection");
}

static int burgers_impl(wp_ctx *c, int nx, int ny, double dx, double dy, double dt, double nu, int nt,
                        const float *u0, const float *v0, float *u_out, float *v_out, bool host_io) {
  TRY(cfd_args(nx, ny, dx, dy, nt));
  if (!u_out || !v_out) return fail(WP_EINVAL, "u_out and v_out must not be NULL");
  if (!(dt >= 0) || !std::isfinite(dt) || !(nu >= 0) || !std::isfinite(nu))
    return fail(WP_EINVAL, "dt and nu must be finite and >= 0");
  const size_t n = size_t(nx) * ny;
  Arena ar(c);
  float *uf[2], *vf[2];
  for (int k = 0; k < 2; ++k) {
    TRY(ar.alloc(&uf[k], n));
    TRY(ar.alloc(&vf[k], n));
  }
  TRY(cfd_stage(c, uf[0], u0, n, host_io, "u0"));
  TRY(cfd_stage(c, vf[0], v0, n, host_io, "v0"));
  for (int k = 0; k < nt; ++k) {
    CU(launch_burgers(c->stream, uf[k & 1], vf[k & 1], uf[(k + 1) & 1], vf[(k + 1) & 1], nx, ny, float(1.0 / dx),
                      float(1.0 / dy), float(dt), float(nu / (dx * dx)), float(nu / (dy * dy))));
    c->launches++;
  }
  const cudaMemcpyKind kind = host_io ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  CU(cudaMemcpyAsync(u_out, uf[nt & 1], n * 4, kind, c->stream));
  CU(cudaMemcpyAsync(v_out, vf[nt & 1], n * 4, kind, c->stream));
  return ctx_wait(c, "burgers");
}

static int poisson_impl(wp_ctx *c, int nx, int ny, double dx, double dy, int nit, const float *p0, const float *b,
                        float *p_out, bool host_io) {
  TRY(cfd_args(nx, ny, dx, dy, nit));
  if (!p_out) return fail(WP_EINVAL, "p_out is NULL");
  const size_t n = size_t(nx) * ny;
  Arena ar(c);
  float *f[2], *bd;
  TRY(ar.alloc(&f[0], n));
  TRY(ar.alloc(&f[1], n));
  TRY(ar.alloc(&bd, n));
  TRY(cfd_stage(c, f[0], p0, n, host_io, "p0"));
  TRY(cfd_stage(c, bd, b, n, host_io, "b"));
  const double dx2 = dx * dx, dy2 = dy * dy;
  for (int k = 0; k < nit; ++k) {
    CU(launch_poisson(c->stream, f[k & 1], bd, f[(k + 1) & 1], nx, ny, float(dx2), float(dy2),
                      float(1.0 / (2.0 * (dx2 + dy2)))));
    c->launches++;
  }
  CU(cudaMemcpyAsync(p_out, f[nit & 1], n * 4, host_io ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                     c->stream));
  return ctx_wait(c, "poisson");
}

int wp_convection_2d(wp_ctx *c, int nx, int ny, double dx, double dy, double dt, double cs, int nt, const float *u0,
                     float *u_out) {
  TRY(enter(c, nullptr));
  return leave(c, nullptr, convection_impl(c, nx, ny, dx, dy, dt, cs, nt, u0, u_out, true));
}

int wp_convection_2d_dev(wp_ctx *c, int nx, int ny, double dx, double dy, double dt, double cs, int nt,
                         const float *u0, float *u_out, void *stream) {
  TRY(enter(c, stream));
  DEV_ARGS(c, stream, {{u0, "u0"}, {u_out, "u_out"}});
  return leave(c, stream, convection_impl(c, nx, ny, dx, dy, dt, cs, nt, u0, u_out, false));
}

int wp_burgers_2d(wp_ctx *c, int nx, int ny, double dx, double dy, double dt, double nu, int nt, const float *u0,
                  const float *v0, float *u_out, float *v_out) {
  TRY(enter(c, nullptr));
  return leave(c, nullptr, burgers_impl(c, nx, ny, dx, dy, dt, nu, nt, u0, v0, u_out, v_out, true));
}

int wp_burgers_2d_dev(wp_ctx *c, int nx, int ny, double dx, double dy, double dt, double nu, int nt, const float *u0,
                      const float *v0, float *u_out, float *v_out, void *stream) {
  TRY(enter(c, stream));
  DEV_ARGS(c, stream, {{u0, "u0"}, {v0, "v0"}, {u_out, "u_out"}, {v_out, "v_out"}});
  return leave(c, stream, burgers_impl(c, nx, ny, dx, dy, dt, nu, nt, u0, v0, u_out, v_out, false));
}

int wp_poisson_2d(wp_ctx *c, int nx, int ny, double dx, double dy, int nit, const float *p0, const float *b,
                  float *p_out) {
  TRY(enter(c, nullptr));
  return leave(c, nullptr, poisson_impl(c, nx, ny, dx, dy, nit, p0, b, p_out, true));
}

int wp_poisson_2d_dev(wp_ctx *c, int nx, int ny, double dx, double dy, int nit, const float *p0, const float *b,
                      float *p_out, void *stream) {
  TRY(enter(c, stream));
  DEV_ARGS(c, stream, {{p0, "p0"}, {b, "b"}, {p_out, "p_out"}});
  return leave(c, stream, poisson_impl(c, nx, ny, dx, dy, nit, p0, b, p_out, false));
}

int wp_set_wait_limit(wp_ctx *c, double seconds) {
  if (!c) return fail(WP_EINVAL, "context is NULL");
  if (!(seconds >= 0.0) || seconds > 60.0) return fail(WP_EINVAL, "wait limit must be in [0, 60] s");
  c->wait_ns = static_cast<uint64_t>(seconds * 1e9);
  return WP_OK;
}

size_t wp_bytes_in_use(const wp_ctx *c) { return c ? c->in_use : 0; }

int wp_set_profiling(wp_ctx *c, int every) {
  if (!c) return fail(WP_EINVAL, "context is NULL");
  if (every < 0) return fail(WP_EINVAL, "every must be >= 0");
  c->profiling = every > 0;
  c->prof_every = every > 0 ? every : 1;
  c->prof_seq = 0;
  c->prof_used = 0;
  return WP_OK;
}

int wp_profile_read(wp_ctx *c, double *stencil_ms, uint64_t *stencil_launches, int reset) {
  if (!c) return fail(WP_EINVAL, "context is NULL");
  if (stencil_ms) *stencil_ms = c->prof_ms;
  if (stencil_launches) *stencil_launches = c->prof_count;
  if (reset) {
    c->prof_ms = 0.0;
    c->prof_count = 0;
  }
  return WP_OK;
}
uint64_t wp_kernel_launches(const wp_ctx *c) { return c ? c->launches : 0; }

int wp_fd_weights(int k, double *alpha) {
  if (!alpha) return fail(WP_EINVAL, "alpha is NULL");
  if (!weights(k, alpha)) return fail(WP_EINVAL, "space_order must be even in [2, 16] (got %d)", k);
  return WP_OK;
}

int wp_cfl_dt(const wp_grid *grid, double vmax, double *dt_max) {
  Geom G;
  TRY(make_geom(grid, &G, false));
  if (!dt_max) return fail(WP_EINVAL, "dt_max is NULL");
  if (!(vmax > 0) || !std::isfinite(vmax)) return fail(WP_EINVAL, "vmax must be positive");
  *dt_max = cfl_limit(G, vmax);
  return WP_OK;
}

int wp_estimate_bytes(const wp_grid *grid, int nsrc, int nrec, int mode, int snap_interval, size_t *bytes) {
  Geom G;
  TRY(make_geom(grid, &G, false));
  if (!bytes) return fail(WP_EINVAL, "bytes is NULL");
  const size_t f = round_up(G.field_bytes(), 256);
  const size_t pts = size_t(nsrc + nrec) * 8 * 24 + size_t(G.nt) * (nsrc + nrec) * 4 * 2;
  const size_t flags = size_t(G.nz) * G.tiles_x * G.tiles_y;
  size_t b = 4 * f + pts + flags + (1 << 20);
  if (mode == 1 && snap_interval <= 1) {
    b += size_t(G.nt) * f + 3 * f;  // full history + adjoint + gradient
  } else if (mode == 1) {
    const int S = std::max(snap_interval, 1);
    const size_t nseg = (size_t(G.nt) + S - 1) / S;
    b += 2 * nseg * f + size_t(std::min(S, std::max(G.nt, 1)) + 2 + 3) * f;
  } else if (mode == 2) {
    b += (2 * size_t(std::max(snap_interval, 0)) + 2 + 3) * f;  // stored states + state 0 + adjoint + gradient
  } else if (mode == 3) {
    // two forward, two adjoint fields, the gradient, and the stored rings: a ring of
    // width R around any box inside the grid has at most 2R x (the grid's surface) points
    const size_t surf = G.ndim == 3 ? size_t(G.nx) * G.ny + size_t(G.ny) * G.nz + size_t(G.nz) * G.nx
                                    : size_t(G.nx) + size_t(G.nz);
    b += 5 * f + size_t(std::max(G.nt - 2, 0)) * 2 * G.R * surf * 4;
  }
  *bytes = b;
  return WP_OK;
}

int wp_forward_dev(wp_ctx *c, const wp_grid *grid, const float *m, const float *eta, const float *wavelet, int nsrc,
                   const double *src, int nrec, const double *rec, float *rec_out, void *stream) {
  TRY(enter(c, stream));
  DEV_ARGS(c, stream, {{m, "m"}, {eta, "eta"}, {wavelet, "wavelet"}, {rec_out, "rec_out"}});
  return leave(c, stream, do_propagate(c, grid, m, eta, wavelet, nsrc, src, nrec, rec, rec_out, +1, false));
}

int wp_forward(wp_ctx *c, const wp_grid *grid, const float *m, const float *eta, const float *wavelet, int nsrc,
               const double *src, int nrec, const double *rec, float *rec_out) {
  TRY(enter(c, nullptr));
  return leave(c, nullptr, do_propagate(c, grid, m, eta, wavelet, nsrc, src, nrec, rec, rec_out, +1, true));
}

int wp_adjoint_dev(wp_ctx *c, const wp_grid *grid, const float *m, const float *eta, const float *rec_data, int nrec,
                   const double *rec, int nsrc, const double *src, float *src_out, void *stream) {
  TRY(enter(c, stream));
  DEV_ARGS(c, stream, {{m, "m"}, {eta, "eta"}, {rec_data, "rec_data"}, {src_out, "src_out"}});
  return leave(c, stream, do_propagate(c, grid, m, eta, rec_data, nrec, rec, nsrc, src, src_out, -1, false));
}

int wp_adjoint(wp_ctx *c, const wp_grid *grid, const float *m, const float *eta, const float *rec_data, int nrec,
               const double *rec, int nsrc, const double *src, float *src_out) {
  TRY(enter(c, nullptr));
  return leave(c, nullptr, do_propagate(c, grid, m, eta, rec_data, nrec, rec, nsrc, src, src_out, -1, true));
}

static int gradient_impl(wp_ctx *c, const wp_grid *grid, const float *m, const float *eta, const float *wavelet,
                         int nsrc, const double *src, const float *residual, int nrec, const double *rec, int S,
                         float *grad_out, bool host_io) {
  wp_state *st = nullptr;
  TRY(forward_save(c, grid, m, eta, wavelet, nsrc, src, nrec, rec, S, nullptr, host_io, host_io, &st));
  int rc = backward(st, residual, grad_out, host_io, host_io);
  state_release(st);
  delete st;
  return rc;
}

int wp_gradient(wp_ctx *c, const wp_grid *grid, const float *m, const float *eta, const float *wavelet, int nsrc,
                const double *src, const float *residual, int nrec, const double *rec, int S, float *grad_out) {
  TRY(enter(c, nullptr));
  return leave(c, nullptr, gradient_impl(c, grid, m, eta, wavelet, nsrc, src, residual, nrec, rec, S, grad_out, true));
}

int wp_gradient_dev(wp_ctx *c, const wp_grid *grid, const float *m, const float *eta, const float *wavelet, int nsrc,
                    const double *src, const float *residual, int nrec, const double *rec, int S, float *grad_out,
                    void *stream) {
  TRY(enter(c, stream));
  DEV_ARGS(c, stream, {{m, "m"}, {eta, "eta"}, {wavelet, "wavelet"},
                                                  {residual, "residual"}, {grad_out, "grad_out"}});
  return leave(c, stream,
               gradient_impl(c, grid, m, eta, wavelet, nsrc, src, residual, nrec, rec, S, grad_out, false));
}

// FWI objective and gradient of one shot: forward with snapshots, r = d - d_obs
// and J = 1/2 ||r||^2, backward with r.
static int fwi_gradient_impl(wp_ctx *c, const wp_grid *grid, const float *m, const float *eta,
                             const float *wavelet, int nsrc, const double *src, const float *d_obs, int nrec,
                             const double *rec, int S, float *grad_out, double *misfit, bool host_io) {
  Geom G;
  TRY(make_geom(grid, &G));
  if (nrec < 0) return fail(WP_EINVAL, "point counts must be >= 0");
  const size_t n = size_t(G.nt) * size_t(nrec);
  if (n && !d_obs) return fail(WP_EINVAL, "d_obs is NULL");
  if (host_io && n && !all_finite(d_obs, n)) return fail(WP_ENONFINITE, "d_obs holds NaN or Inf");
  Arena tmp(c);
  float *d = nullptr, *r = nullptr, *dobs_d = nullptr;
  double *partial = nullptr;
  const int max_blocks = 1024;
  if (n) {
    TRY(tmp.alloc(&d, n));
    TRY(tmp.alloc(&r, n));
    TRY(tmp.alloc(&partial, size_t(max_blocks)));
    if (host_io) {
      TRY(tmp.alloc(&dobs_d, n));
      CU(cudaMemcpyAsync(dobs_d, d_obs, n * 4, cudaMemcpyHostToDevice, c->stream));
    } else {
      dobs_d = const_cast<float *>(d_obs);
    }
  }
  wp_state *st = nullptr;
  TRY(forward_save(c, grid, m, eta, wavelet, nsrc, src, nrec, rec, S, d, host_io, false, &st));
  int rc = [&]() -> int {
    double J = 0.0;
    if (n) {
      int used = 0;
      CU(launch_residual(c->stream, d, dobs_d, r, (long long)n, partial, max_blocks, &used));
      c->launches++;
      std::vector<double> h(static_cast<size_t>(used));
      CU(cudaMemcpyAsync(h.data(), partial, size_t(used) * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      TRY(ctx_wait(c, "residual"));
      for (double v : h) J += v;
      J *= 0.5;
    }
    if (misfit) *misfit = J;
    if (!std::isfinite(J)) return fail(WP_ENONFINITE, "d_obs or the modelled data holds NaN or Inf");
    return backward(st, r, grad_out, false, host_io);
  }();
  state_release(st);
  delete st;
  return rc;
}

// Inputs of a one-shot gradient staged on the device: coefficients, point tables,
// wavelet and residual (validated), two work fields W (which hold m and eta
// while the coefficients are built from host arrays).
struct GradSetup {
  explicit GradSetup(wp_ctx *c) : ar(c) {}
  Geom G;
  Arena ar;
  Field3 W[2];
  Prop P;
  DevPoints dsrc, drec;
  const float *q_d = nullptr, *r_d = nullptr, *eta_d = nullptr;
};

static int grad_setup(wp_ctx *c, const wp_grid *grid, const float *m, const float *eta, const float *wavelet,
                      int nsrc, const double *src, const float *residual, int nrec, const double *rec,
                      const float *grad_out, bool host_io, GradSetup &S) {
  Geom &G = S.G;
  TRY(make_geom(grid, &G));
  if (nsrc < 0 || nrec < 0) return fail(WP_EINVAL, "point counts must be >= 0");
  if (!m || !eta || !grad_out) return fail(WP_EINVAL, "m, eta and grad_out must not be NULL");
  const size_t n_in = size_t(G.nt) * nsrc, n_res = size_t(G.nt) * nrec;
  if (n_in && !wavelet) return fail(WP_EINVAL, "wavelet is NULL");
  if (n_res && !residual) return fail(WP_EINVAL, "residual is NULL");
  if (host_io && n_in && !all_finite(wavelet, n_in)) return fail(WP_ENONFINITE, "wavelet holds NaN or Inf");
  if (host_io && n_res && !all_finite(residual, n_res)) return fail(WP_ENONFINITE, "residual holds NaN or Inf");
  PointSet psrc, prec;
  TRY(build_points(G, nsrc, src, &psrc, "source"));
  TRY(build_points(G, nrec, rec, &prec, "receiver"));
  TRY(alloc_field(S.ar, G, &S.W[0], false, c->stream));
  TRY(alloc_field(S.ar, G, &S.W[1], false, c->stream));
  const float *md = m, *ed = eta;
  if (host_io) {
    CU(cudaMemcpyAsync(S.W[0].p, m, G.npoints * 4, cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemcpyAsync(S.W[1].p, eta, G.npoints * 4, cudaMemcpyHostToDevice, c->stream));
    md = S.W[0].p;
    ed = S.W[1].p;
  }
  S.eta_d = ed;
  TRY(prop_setup(c, S.ar, G, md, ed, &S.P));
  TRY(upload_points(c, S.ar, psrc, false, true, &S.dsrc));
  TRY(upload_points(c, S.ar, prec, false, true, &S.drec));
  S.q_d = wavelet;
  S.r_d = residual;
  if (host_io && (n_in || n_res)) {
    float *tmp = nullptr;
    TRY(S.ar.alloc(&tmp, n_in + n_res));
    if (n_in) CU(cudaMemcpyAsync(tmp, wavelet, n_in * 4, cudaMemcpyHostToDevice, c->stream));
    if (n_res) CU(cudaMemcpyAsync(tmp + n_in, residual, n_res * 4, cudaMemcpyHostToDevice, c->stream));
    S.q_d = tmp;
    S.r_d = tmp + n_in;
  } else if (!host_io && (n_in || n_res)) {
    int *bad = c->d_scalars + 1;
    CU(cudaMemsetAsync(bad, 0, sizeof(int), c->stream));
    if (n_in) CU(launch_check_finite(c->stream, wavelet, (long long)n_in, bad));
    if (n_res) CU(launch_check_finite(c->stream, residual, (long long)n_res, bad));
    c->launches += (n_in ? 1 : 0) + (n_res ? 1 : 0);
    CU(cudaMemcpyAsync(c->h_scalars + 1, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    TRY(ctx_wait(c, "input checks"));
    if (c->h_scalars[1]) return fail(WP_ENONFINITE, "wavelet or residual holds NaN or Inf");
  }
  return WP_OK;
}

// pitched gradient -> the caller's contiguous array
static int grad_copy_out(wp_ctx *c, const Geom &G, const Field3 &g, float *grad_out, bool host_io) {
  CU(cudaMemcpy2DAsync(grad_out, size_t(G.nx) * 4, g.p, size_t(G.pitch) * 4, size_t(G.nx) * 4,
                       size_t(G.ny) * G.nz, host_io ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->stream));
  return WP_OK;
}

// Gradient (as wp_gradient) with binomial checkpointing: `nslots` stored states
// replace the periodic snapshots; the forward field is recomputed from state 0
// and the stored states by the schedule of ck_schedule.
static int gradient_ckpt_impl(wp_ctx *c, const wp_grid *grid, const float *m, const float *eta,
                              const float *wavelet, int nsrc, const double *src, const float *residual, int nrec,
                              const double *rec, int nslots, float *grad_out, bool host_io) {
  NvtxRange range("wp.gradient_checkpointed");
  if (nslots < 0 || nslots > 4096) return fail(WP_EINVAL, "checkpoints must be in [0, 4096]");
  GradSetup S(c);
  TRY(grad_setup(c, grid, m, eta, wavelet, nsrc, src, residual, nrec, rec, grad_out, host_io, S));
  const Geom &G = S.G;
  Arena &ar = S.ar;
  Field3 *W = S.W;
  // state 0 = (0, 0) in slot 0; slots 1..nslots for stored states
  std::vector<Field3> sp(size_t(nslots) + 1), sc(size_t(nslots) + 1);
  for (int k = 0; k <= nslots; ++k) {
    TRY(alloc_field(ar, G, &sp[size_t(k)], k == 0, c->stream));
    TRY(alloc_field(ar, G, &sc[size_t(k)], k == 0, c->stream));
  }
  Field3 A[2], g;
  TRY(alloc_field(ar, G, &A[0], true, c->stream));
  TRY(alloc_field(ar, G, &A[1], true, c->stream));
  TRY(alloc_field(ar, G, &g, true, c->stream));
  CkTable tb;
  ck_build(tb, G.nt, nslots);
  std::vector<CkOp> ops;
  ck_schedule(tb, ops);
  const Field3 *cp = nullptr, *cc = nullptr;  // current state (u^{k-1}, u^k)
  int state = -1;
  long long kadj = 0;
  auto is_work = [&](const Field3 *f) { return f == &W[0] || f == &W[1]; };
  for (const CkOp &op : ops) {
    if (op.kind == kCkAdvance) {
      cp = &sp[size_t(op.slot)];
      cc = &sc[size_t(op.slot)];
      for (int k = op.a; k < op.b; ++k) {
        Field3 *out = is_work(cp) ? const_cast<Field3 *>(cp) : (cc == &W[0] ? &W[1] : &W[0]);
        TRY(prop_step(S.P, *cc, *cp, out->p, kModeFwd, nullptr, nullptr));
        TRY(prop_inject(S.P, S.dsrc, S.q_d, k, out->p, nullptr, nullptr));
        cp = cc;
        cc = out;
      }
      state = op.b;
    } else if (op.kind == kCkStore) {
      if (state != op.a) return fail(WP_ECUDA, "internal error: checkpoint schedule out of order");
      CU(cudaMemcpyAsync(sp[size_t(op.slot)].p, cp->p, G.field_bytes(), cudaMemcpyDeviceToDevice, c->stream));
      CU(cudaMemcpyAsync(sc[size_t(op.slot)].p, cc->p, G.field_bytes(), cudaMemcpyDeviceToDevice, c->stream));
    } else {
      if (state != op.a) return fail(WP_ECUDA, "internal error: checkpoint schedule out of order");
      Field3 &w1 = A[kadj & 1], &w2 = A[(kadj + 1) & 1];
      TRY(prop_step(S.P, w1, w2, w2.p, kModeAdjGrad, cc, &g));
      TRY(prop_inject(S.P, S.drec, S.r_d, op.a - 1, w2.p, g.p, cc->p));
      ++kadj;
    }
  }
  TRY(grad_copy_out(c, G, g, grad_out, host_io));
  return ctx_wait(c, "checkpointed gradient");
}

// ---------------------------------------------------------------------------
// Boundary-wavefield reconstruction
// ---------------------------------------------------------------------------
// Where eta = 0 the update is symmetric in time: the forward step
//     u^{n+1} = u^n + (u^n - u^{n-1}) + b L u^n + b P_s^T q^n
// solved for u^{n-1} is the same expression with u^{n+1} and u^{n-1} swapped, so
// the K1/K2 kernels run backward reproduce u^{n-1} on the box Z where eta = 0,
// given u^n on Z and on the ring of width R around it (the Laplacian's reach).
// The forward pass stores that ring for every level the backward pass rebuilds;
// its end state (u^{nt-1}, u^nt) starts the reversal.  Values outside Z come out
// wrong (the layer's damping is not reversible), so the gradient is returned on
// Z and zero in the damping layer.

// The box Z = {eta == 0}: bounding box of the zero points, verified to hold no
// nonzero point.
static int undamped_box(wp_ctx *c, const Geom &G, const float *eta_d, Box *Z) {
  int *d = c->d_scalars + 8;  // 7 ints: bbox (6) + count
  const int init[7] = {INT_MAX, -1, INT_MAX, -1, INT_MAX, -1, 0};
  int *h = c->h_scalars + 8;
  for (int i = 0; i < 7; ++i) h[i] = init[i];
  CU(cudaMemcpyAsync(d, h, sizeof(init), cudaMemcpyHostToDevice, c->stream));
  CU(launch_zero_bbox(c->stream, eta_d, G.fg(), d));
  CU(cudaMemcpyAsync(h, d, 6 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  c->launches++;
  TRY(ctx_wait(c, "undamped box"));
  if (h[1] < 0) return fail(WP_EINVAL, "eta is nonzero everywhere: no undamped region to reconstruct");
  *Z = Box{h[0], h[1] + 1, h[2], h[3] + 1, h[4], h[5] + 1};
  CU(launch_count_nonzero(c->stream, eta_d, G.fg(), *Z, d + 6));
  CU(cudaMemcpyAsync(h + 6, d + 6, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  c->launches++;
  TRY(ctx_wait(c, "undamped box check"));
  if (h[6]) return fail(WP_EINVAL, "the region where eta = 0 is not a box (%d nonzero points inside its bounds)", h[6]);
  return WP_OK;
}

// The ring (Z grown by R along every axis longer than one point, clipped to the
// grid) minus Z, as up to six boxes.
static RingBoxes ring_boxes(const Geom &G, const Box &Z) {
  const int rz = G.R, ry = G.ny > 1 ? G.R : 0, rx = G.R;
  const Box E{std::max(Z.z0 - rz, 0), std::min(Z.z1 + rz, G.nz), std::max(Z.y0 - ry, 0), std::min(Z.y1 + ry, G.ny),
              std::max(Z.x0 - rx, 0), std::min(Z.x1 + rx, G.nx)};
  const Box cand[6] = {
      {E.z0, Z.z0, E.y0, E.y1, E.x0, E.x1}, {Z.z1, E.z1, E.y0, E.y1, E.x0, E.x1},
      {Z.z0, Z.z1, E.y0, Z.y0, E.x0, E.x1}, {Z.z0, Z.z1, Z.y1, E.y1, E.x0, E.x1},
      {Z.z0, Z.z1, Z.y0, Z.y1, E.x0, Z.x0}, {Z.z0, Z.z1, Z.y0, Z.y1, Z.x1, E.x1},
  };
  RingBoxes rb;
  std::memset(&rb, 0, sizeof(rb));
  for (const Box &b : cand) {
    const long long n = static_cast<long long>(b.z1 - b.z0) * (b.y1 - b.y0) * (b.x1 - b.x0);
    if (b.z1 <= b.z0 || b.y1 <= b.y0 || b.x1 <= b.x0) continue;
    rb.b[rb.n] = b;
    rb.start[rb.n + 1] = rb.start[rb.n] + n;
    ++rb.n;
  }
  return rb;
}

static int gradient_recon_impl(wp_ctx *c, const wp_grid *grid, const float *m, const float *eta,
                               const float *wavelet, int nsrc, const double *src, const float *residual, int nrec,
                               const double *rec, float *grad_out, bool host_io) {
  NvtxRange range("wp.gradient_reconstruct");
  GradSetup S(c);
  TRY(grad_setup(c, grid, m, eta, wavelet, nsrc, src, residual, nrec, rec, grad_out, host_io, S));
  const Geom &G = S.G;
  Arena &ar = S.ar;
  Box Z;
  TRY(undamped_box(c, G, S.eta_d, &Z));
  const RingBoxes rb = ring_boxes(G, Z);
  if (G.ndim == 3) {  // the backward update runs on Z only (x start rounded down for TMA)
    S.P.sub = true;
    S.P.box = Z;
    S.P.box.x0 = Z.x0 & ~3;
    const Box &bx = S.P.box;
    S.P.plan_sub[0] = plan_items(bx.x1 - bx.x0, bx.y1 - bx.y0, bx.z1 - bx.z0, G.R, stencil3d_tile_x(G.R, 0),
                                 stencil3d_tile_y(G.R, 0), G.R, c->num_sms, c->occ3d[0][G.R]);
  }
  const long long nring = rb.start[rb.n];
  const int nstore = std::max(G.nt - 2, 0);  // levels 1 .. nt-2
  float *store = nullptr;
  if (nring && nstore) TRY(ar.alloc(&store, size_t(nring) * nstore));
  Field3 U[2], A[2], g;
  TRY(alloc_field(ar, G, &U[0], true, c->stream));
  TRY(alloc_field(ar, G, &U[1], true, c->stream));
  TRY(alloc_field(ar, G, &A[0], true, c->stream));
  TRY(alloc_field(ar, G, &A[1], true, c->stream));
  TRY(alloc_field(ar, G, &g, true, c->stream));
  // forward: (U[p], U[1-p]) = (u^{n-1}, u^n)
  int p = 0;
  for (int n = 0; n < G.nt; ++n) {
    Field3 &prv = U[p], &cur = U[1 - p];
    TRY(prop_step(S.P, cur, prv, prv.p, kModeFwd, nullptr, nullptr));
    TRY(prop_inject(S.P, S.dsrc, S.q_d, n, prv.p, nullptr, nullptr));
    p = 1 - p;  // prv now holds u^{n+1}
    if (n + 1 <= nstore && nring) {
      CU(launch_ring_copy(c->stream, prv.p, G.fg(), store + size_t(n) * nring, rb, true));
      c->launches++;
    }
  }
  // backward: lo = u^{j-1}, hi = u^j
  Field3 *lo = &U[p], *hi = &U[1 - p];
  long long kadj = 0;
  for (int j = G.nt; j >= 1; --j, ++kadj) {
    Field3 &w1 = A[kadj & 1], &w2 = A[(kadj + 1) & 1];
    TRY(prop_step(S.P, w1, w2, w2.p, kModeAdjGrad, hi, &g));
    TRY(prop_inject(S.P, S.drec, S.r_d, j - 1, w2.p, g.p, hi->p));
    if (j >= 3) {
      // u^{j-2} = u^{j-1} + (u^{j-1} - u^j) + b L u^{j-1} + b P_s^T q^{j-1} on Z, into hi
      TRY(prop_step(S.P, *lo, *hi, hi->p, kModeFwd, nullptr, nullptr, true));
      TRY(prop_inject(S.P, S.dsrc, S.q_d, j - 1, hi->p, nullptr, nullptr));
      if (nring) {
        CU(launch_ring_copy(c->stream, hi->p, G.fg(), store + size_t(j - 3) * nring, rb, false));
        c->launches++;
      }
      std::swap(lo, hi);
    } else {
      hi = lo;
    }
  }
  CU(launch_zero_outside(c->stream, g.p, G.fg(), Z));
  c->launches++;
  TRY(grad_copy_out(c, G, g, grad_out, host_io));
  return ctx_wait(c, "gradient by boundary reconstruction");
}

int wp_forward_save(wp_ctx *c, const wp_grid *grid, const float *m, const float *eta, const float *wavelet, int nsrc,
                    const double *src, int nrec, const double *rec, int S, float *rec_out, void *stream,
                    wp_state **state) {
  if (!state) return fail(WP_EINVAL, "state is NULL");
  *state = nullptr;
  TRY(enter(c, stream));
  DEV_ARGS(c, stream, {{m, "m"}, {eta, "eta"}, {wavelet, "wavelet"}, {rec_out, "rec_out"}});
  const int rc = leave(c, stream,
                       forward_save(c, grid, m, eta, wavelet, nsrc, src, nrec, rec, S, rec_out, false, false, state));
  if (rc == WP_OK && *state) {
    c->states.insert(*state);
  } else if (*state) {
    state_release(*state);
    delete *state;
    *state = nullptr;
  }
  return rc;
}

int wp_backward(wp_state *st, const float *residual, float *grad_out, void *stream) {
  if (!st) return fail(WP_EINVAL, "state is NULL");
  if (!st->c) return fail(WP_EINVAL, "the state's context has been destroyed");
  TRY(enter(st->c, stream));
  DEV_ARGS(st->c, stream, {{residual, "residual"}, {grad_out, "grad_out"}});
  return leave(st->c, stream, backward(st, residual, grad_out, false, false));
}

int wp_fwi_gradient(wp_ctx *c, const wp_grid *grid, const float *m, const float *eta, const float *wavelet, int nsrc,
                    const double *src, const float *d_obs, int nrec, const double *rec, int S, float *grad_out,
                    double *misfit) {
  TRY(enter(c, nullptr));
  return leave(c, nullptr,
               fwi_gradient_impl(c, grid, m, eta, wavelet, nsrc, src, d_obs, nrec, rec, S, grad_out, misfit, true));
}

int wp_fwi_gradient_dev(wp_ctx *c, const wp_grid *grid, const float *m, const float *eta, const float *wavelet,
                        int nsrc, const double *src, const float *d_obs, int nrec, const double *rec, int S,
                        float *grad_out, double *misfit, void *stream) {
  TRY(enter(c, stream));
  DEV_ARGS(c, stream, {{m, "m"}, {eta, "eta"}, {wavelet, "wavelet"}, {d_obs, "d_obs"},
                                                  {grad_out, "grad_out"}});
  return leave(c, stream,
               fwi_gradient_impl(c, grid, m, eta, wavelet, nsrc, src, d_obs, nrec, rec, S, grad_out, misfit, false));
}

int wp_gradient_checkpointed(wp_ctx *c, const wp_grid *grid, const float *m, const float *eta, const float *wavelet,
                             int nsrc, const double *src, const float *residual, int nrec, const double *rec,
                             int checkpoints, float *grad_out) {
  TRY(enter(c, nullptr));
  return leave(c, nullptr, gradient_ckpt_impl(c, grid, m, eta, wavelet, nsrc, src, residual, nrec, rec, checkpoints,
                                              grad_out, true));
}

int wp_gradient_checkpointed_dev(wp_ctx *c, const wp_grid *grid, const float *m, const float *eta,
                                 const float *wavelet, int nsrc, const double *src, const float *residual, int nrec,
                                 const double *rec, int checkpoints, float *grad_out, void *stream) {
  TRY(enter(c, stream));
  DEV_ARGS(c, stream, {{m, "m"}, {eta, "eta"}, {wavelet, "wavelet"},
                                                  {residual, "residual"}, {grad_out, "grad_out"}});
  return leave(c, stream, gradient_ckpt_impl(c, grid, m, eta, wavelet, nsrc, src, residual, nrec, rec, checkpoints,
                                             grad_out, false));
}

int wp_gradient_reconstruct(wp_ctx *c, const wp_grid *grid, const float *m, const float *eta, const float *wavelet,
                            int nsrc, const double *src, const float *residual, int nrec, const double *rec,
                            float *grad_out) {
  TRY(enter(c, nullptr));
  return leave(c, nullptr,
               gradient_recon_impl(c, grid, m, eta, wavelet, nsrc, src, residual, nrec, rec, grad_out, true));
}

int wp_gradient_reconstruct_dev(wp_ctx *c, const wp_grid *grid, const float *m, const float *eta,
                                const float *wavelet, int nsrc, const double *src, const float *residual, int nrec,
                                const double *rec, float *grad_out, void *stream) {
  TRY(enter(c, stream));
  DEV_ARGS(c, stream, {{m, "m"}, {eta, "eta"}, {wavelet, "wavelet"},
                                                  {residual, "residual"}, {grad_out, "grad_out"}});
  return leave(c, stream,
               gradient_recon_impl(c, grid, m, eta, wavelet, nsrc, src, residual, nrec, rec, grad_out, false));
}

int wp_checkpoint_schedule(int nt, int checkpoints, int *ops, int max_ops, int *nops, long long *forward_steps) {
  if (nt < 0 || checkpoints < 0 || checkpoints > 4096 || !nops) return fail(WP_EINVAL, "bad schedule arguments");
  CkTable tb;
  ck_build(tb, nt, checkpoints);
  std::vector<CkOp> v;
  ck_schedule(tb, v);
  *nops = static_cast<int>(v.size());
  long long fw = 0;
  for (const CkOp &op : v)
    if (op.kind == kCkAdvance) fw += op.b - op.a;
  if (forward_steps) *forward_steps = fw;
  if (ops) {
    if (max_ops < static_cast<int>(v.size())) return fail(WP_EINVAL, "ops holds %d entries, %zu needed", max_ops, v.size());
    for (size_t i = 0; i < v.size(); ++i) {
      ops[4 * i] = v[i].kind;
      ops[4 * i + 1] = v[i].a;
      ops[4 * i + 2] = v[i].b;
      ops[4 * i + 3] = v[i].slot;
    }
  }
  return WP_OK;
}

int wp_axpy_dev(wp_ctx *c, long long n, float alpha, const float *x, float *y, void *stream) {
  if (n < 0 || (n > 0 && (!x || !y))) return fail(WP_EINVAL, "bad axpy arguments");
  TRY(enter(c, stream));
  DEV_ARGS(c, stream, {{x, "x"}, {y, "y"}});
  int rc = [&]() -> int {
    CU(launch_axpy(c->stream, n, alpha, x, y));
    c->launches++;
    return ctx_wait(c, "axpy");
  }();
  return leave(c, stream, rc);
}

int wp_misfit_dev(wp_ctx *c, long long n, const float *d, const float *d_obs, float *r_out, double *misfit,
                  void *stream) {
  if (n < 0 || (n > 0 && (!d || !d_obs || !r_out)) || !misfit) return fail(WP_EINVAL, "bad misfit arguments");
  TRY(enter(c, stream));
  DEV_ARGS(c, stream, {{d, "d"}, {d_obs, "d_obs"}, {r_out, "r_out"}});
  int rc = [&]() -> int {
    double J = 0.0;
    if (n) {
      Arena tmp(c);
      double *partial = nullptr;
      const int max_blocks = 1024;
      TRY(tmp.alloc(&partial, size_t(max_blocks)));
      int used = 0;
      CU(launch_residual(c->stream, d, d_obs, r_out, n, partial, max_blocks, &used));
      c->launches++;
      std::vector<double> h(static_cast<size_t>(used));
      CU(cudaMemcpyAsync(h.data(), partial, size_t(used) * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      TRY(ctx_wait(c, "misfit"));
      for (double v : h) J += v;
      J *= 0.5;
    }
    *misfit = J;
    if (!std::isfinite(J)) return fail(WP_ENONFINITE, "d or d_obs holds NaN or Inf");
    return WP_OK;
  }();
  return leave(c, stream, rc);
}

int wp_update_model_dev(wp_ctx *c, long long n, float step, const float *grad, float *m, float m_min, float m_max,
                        void *stream) {
  if (n < 0 || (n > 0 && (!grad || !m)) || !(m_min > 0.f) || !(m_max >= m_min))
    return fail(WP_EINVAL, "bad model-update arguments");
  TRY(enter(c, stream));
  DEV_ARGS(c, stream, {{grad, "grad"}, {m, "m"}});
  int rc = [&]() -> int {
    CU(launch_update_model(c->stream, n, step, grad, m, m_min, m_max));
    c->launches++;
    return ctx_wait(c, "model update");
  }();
  return leave(c, stream, rc);
}

int wp_set_budget(wp_ctx *c, size_t bytes) {
  if (!c) return fail(WP_EINVAL, "context is NULL");
  c->budget = bytes;
  return WP_OK;
}

int wp_trim(wp_ctx *c, size_t keep_bytes) {
  if (!c) return fail(WP_EINVAL, "context is NULL");
  CU(cudaSetDevice(c->device));
  CU(cudaStreamSynchronize(c->stream));
  while (!c->cache.empty() && c->in_use > keep_bytes) {
    auto it = std::prev(c->cache.end());
    cudaFreeAsync(it->second, c->stream);
    c->in_use -= it->first;
    c->cache.erase(it);
  }
  CU(cudaStreamSynchronize(c->stream));  // lets the stream-ordered pool hand the memory back
  return WP_OK;
}

void wp_state_free(wp_state *st) {
  if (!st) return;
  if (st->c) {  // still attached: give its blocks back to the context
    st->c->states.erase(st);
    state_release(st);
  }
  delete st;
}

int wp_propagate_dev(wp_ctx *c, const wp_grid *grid, const float *m, const float *eta, float *u_prev, float *u,
                     int nsteps, void *stream) {
  TRY(enter(c, stream));
  DEV_ARGS(c, stream, {{m, "m"}, {eta, "eta"}, {u_prev, "u_prev"}, {u, "u"}});
  int rc = [&]() -> int {
    Geom G;
    TRY(make_geom(grid, &G));
    if (!m || !eta || !u_prev || !u) return fail(WP_EINVAL, "NULL field");
    if (nsteps < 0) return fail(WP_EINVAL, "nsteps must be >= 0");
    Arena ar(c);
    Field3 f[2];
    TRY(alloc_field(ar, G, &f[0], true, c->stream));
    TRY(alloc_field(ar, G, &f[1], true, c->stream));
    Prop P;
    TRY(prop_setup(c, ar, G, m, eta, &P));
    const size_t w = size_t(G.nx) * 4, hp = size_t(G.pitch) * 4, rows = size_t(G.ny) * G.nz;
    CU(cudaMemcpy2DAsync(f[0].p, hp, u, w, w, rows, cudaMemcpyDeviceToDevice, c->stream));
    CU(cudaMemcpy2DAsync(f[1].p, hp, u_prev, w, w, rows, cudaMemcpyDeviceToDevice, c->stream));
    DevPoints none;
    TRY(run_loop(P, f, nsteps, none, nullptr, none, nullptr, +1));
    CU(cudaMemcpy2DAsync(u, w, f[nsteps & 1].p, hp, w, rows, cudaMemcpyDeviceToDevice, c->stream));
    CU(cudaMemcpy2DAsync(u_prev, w, f[(nsteps + 1) & 1].p, hp, w, rows, cudaMemcpyDeviceToDevice, c->stream));
    return ctx_wait(c, "propagation");
  }();
  return leave(c, stream, rc);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Forward without device allocation (wp_forward_noalloc).  The work space lives
// in one statically declared device array; host code must use the address that
// cudaGetSymbolAddress returns for the current device (the array's name in host
// code is only a host-side stand-in).
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[WP_NOALLOC_MAX_BYTES];

static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[256];  // per device, filled on the first call there

static int noalloc_scratch(void **out) {
  int dev = 0;
  CU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return fail(WP_EINVAL, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(WP_ECUDA, "cudaGetSymbolAddress of the no-allocation work space failed: %s",
                  cudaGetErrorString(e));
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return WP_OK;
}

// Carves 256-byte aligned pieces out of the fixed work space.
struct Carve {
  unsigned char *base;
  size_t used = 0, cap;
  bool over = false;
  template <class T>
  T *take(size_t count) {
    const size_t off = round_up(used, 256);
    const size_t bytes = std::max<size_t>(count * sizeof(T), 1);
    if (off + bytes > cap) {
      over = true;
      used = off + bytes;
      return nullptr;
    }
    used = off + bytes;
    return base ? reinterpret_cast<T *>(base + off) : nullptr;
  }
};

// Injection table in the same (target, point, corner) order as the context path.
static void csr_of(const PointSet &ps, std::vector<long long> &target, std::vector<int> &rowptr,
                   std::vector<int> &pid, std::vector<float> &cw) {
  const size_t ne = size_t(ps.npts) * ps.nc;
  std::vector<size_t> order(ne);
  for (size_t e = 0; e < ne; ++e) order[e] = e;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return ps.idx[a] < ps.idx[b]; });
  for (size_t k = 0; k < ne; ++k) {
    const size_t e = order[k];
    if (target.empty() || target.back() != ps.idx[e]) {
      target.push_back(ps.idx[e]);
      rowptr.push_back(int(k));
    }
    pid.push_back(int(e / ps.nc));
    cw.push_back(ps.w[e]);
  }
  rowptr.push_back(int(ne));
}

// `touched` is set once the call has queued work on `st`.
static int forward_noalloc_body(const wp_grid *grid, const float *m, const float *eta, const float *wavelet,
                                int nsrc, const double *src, int nrec, const double *rec, float *rec_out,
                                cudaStream_t st, bool *touched) {
  NvtxRange range("wp.forward_noalloc");
  Geom G;
  TRY(make_geom(grid, &G));
  if (nsrc < 0 || nrec < 0) return fail(WP_EINVAL, "point counts must be >= 0");
  if (!m || !eta) return fail(WP_EINVAL, "m and eta must not be NULL");
  if (nsrc > 0 && G.nt > 0 && !wavelet) return fail(WP_EINVAL, "wavelet is NULL");
  if (nrec > 0 && G.nt > 0 && !rec_out) return fail(WP_EINVAL, "rec_out is NULL");
  // everything runs on the current device: the arrays and the stream must belong to it
  int dev = 0, sdev = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaStreamGetDevice(st, &sdev));
  if (sdev != dev) return fail(WP_EINVAL, "the stream belongs to device %d, the current device is %d", sdev, dev);
  TRY(check_dev_args(dev, {{m, "m"}, {eta, "eta"}, {wavelet, "wavelet"}, {rec_out, "rec_out"}}));
  PointSet ps, pr;
  TRY(build_points(G, nsrc, src, &ps, "source"));
  TRY(build_points(G, nrec, rec, &pr, "receiver"));
  std::vector<long long> target;
  std::vector<int> rowptr, pid;
  std::vector<float> cw;
  csr_of(ps, target, rowptr, pid, cw);

  // size the work space before touching the device
  Carve cv{nullptr, 0, WP_NOALLOC_MAX_BYTES};
  auto plan = [&](Carve &c, int **scal, float **b, float **s, float **u0, float **u1, unsigned **tbits,
                  unsigned char **tflag,
                  long long **d_target, int **d_rowptr, int **d_pid, float **d_cw, long long **d_ridx,
                  float **d_rw) {
    *scal = c.take<int>(16);
    *b = c.take<float>(G.nfield);
    *s = c.take<float>(G.nfield);
    *u0 = c.take<float>(G.nfield);
    *u1 = c.take<float>(G.nfield);
    *tbits = G.ndim == 3 ? c.take<unsigned>(size_t(G.tiles_y) * G.tiles_x * G.nzw) : nullptr;
    *tflag = G.ndim == 3 ? c.take<unsigned char>(size_t(G.nz) * G.tiles_y * G.tiles_x) : nullptr;
    *d_target = c.take<long long>(target.size());
    *d_rowptr = c.take<int>(rowptr.size());
    *d_pid = c.take<int>(pid.size());
    *d_cw = c.take<float>(cw.size());
    *d_ridx = c.take<long long>(pr.idx.size());
    *d_rw = c.take<float>(pr.w.size());
  };
  int *scal;
  float *b, *s, *u0, *u1, *d_cw, *d_rw;
  unsigned *tbits;
  unsigned char *tflag;
  long long *d_target, *d_ridx;
  int *d_rowptr, *d_pid;
  plan(cv, &scal, &b, &s, &u0, &u1, &tbits, &tflag, &d_target, &d_rowptr, &d_pid, &d_cw, &d_ridx, &d_rw);
  if (cv.over)
    return fail(WP_ENOMEM, "this problem needs %zu bytes of work space; wp_forward_noalloc is limited to %zu",
                cv.used, size_t(WP_NOALLOC_MAX_BYTES));
  void *base = nullptr;
  TRY(noalloc_scratch(&base));
  Carve c{static_cast<unsigned char *>(base), 0, WP_NOALLOC_MAX_BYTES};
  plan(c, &scal, &b, &s, &u0, &u1, &tbits, &tflag, &d_target, &d_rowptr, &d_pid, &d_cw, &d_ridx, &d_rw);

  // the array keeps the last call's contents: clear what must start at zero
  *touched = true;
  CU(cudaMemsetAsync(scal, 0, 16 * sizeof(int), st));
  if (tflag) CU(cudaMemsetAsync(tflag, 0, size_t(G.nz) * G.tiles_y * G.tiles_x, st));
  if (!target.empty()) {
    CU(cudaMemcpyAsync(d_target, target.data(), target.size() * sizeof(long long), cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(d_rowptr, rowptr.data(), rowptr.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(d_pid, pid.data(), pid.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(d_cw, cw.data(), cw.size() * sizeof(float), cudaMemcpyHostToDevice, st));
  }
  if (!pr.idx.empty()) {
    CU(cudaMemcpyAsync(d_ridx, pr.idx.data(), pr.idx.size() * sizeof(long long), cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(d_rw, pr.w.data(), pr.w.size() * sizeof(float), cudaMemcpyHostToDevice, st));
  }
  CoefArgs ca;
  memset(&ca, 0, sizeof ca);
  ca.m = m;
  ca.eta = eta;
  ca.g = G.fg();
  coef_set_dt(&ca, G.dt);
  ca.b = b;
  ca.s = s;
  ca.tflag = tflag;
  ca.tbits = tbits;
  ca.nzw = G.nzw;
  ca.tiles_x = G.tiles_x;
  ca.tiles_y = G.tiles_y;
  ca.tile_w = kFlagTX;
  ca.tile_h = kTileFlagTY;
  ca.max_inv_m_bits = reinterpret_cast<unsigned int *>(scal + 2);
  ca.bad = scal + 1;
  CU(launch_coef(st, ca));
  if (size_t(G.nt) * nsrc > 0) CU(launch_check_finite(st, wavelet, (long long)G.nt * nsrc, scal + 3));
  int h[16];
  CU(cudaMemcpyAsync(h, scal, sizeof h, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  if ((h[1] & 1) || h[3]) return fail(WP_ENONFINITE, "m, eta or the wavelet holds NaN or Inf");
  if (h[1] & 2) return fail(WP_EINVAL, "m must be > 0 and eta >= 0 everywhere");
  float max_inv_m;
  memcpy(&max_inv_m, &h[2], 4);
  const double vmax = std::sqrt(double(max_inv_m));
  const double lim = cfl_limit(G, vmax);
  if (G.dt > lim * (1.0 + 1e-5))
    return fail(WP_ECFL, "dt = %.6g exceeds the stability limit %.6g for vmax = %.6g", G.dt, lim, vmax);
  CU(cudaMemsetAsync(u0, 0, G.field_bytes(), st));
  CU(cudaMemsetAsync(u1, 0, G.field_bytes(), st));

  const LapCoef lc = lap_coef(G);
  const float neg_inv_dt2 = static_cast<float>(-1.0 / (G.dt * G.dt));
  float *u[2] = {u0, u1};
  CUtensorMap halo[2], tile[2], tb, ts;
  Plan3d pl;
  if (G.ndim == 3) {
    const int tx = stencil3d_tile_x(G.R, kModeFwd), ty = stencil3d_tile_y(G.R, kModeFwd);
    for (int i = 0; i < 2; ++i) {
      TRY(make_map(&halo[i], u[i], G, halo_box_w(G.R, kModeFwd), ty + 2 * G.R));
      TRY(make_map(&tile[i], u[i], G, tx, ty));
    }
    TRY(make_map(&tb, b, G, tx, ty));
    TRY(make_map(&ts, s, G, tx, ty));
    int smem = 0, occ = 0, ty_k = 0, nsm = 0;
    CU(prepare_stencil3d_fwd(G.R, &smem, &occ, &ty_k));
    CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    pl = plan3d(G, kModeFwd, nsm, occ);
  }
  for (int k = 0; k < G.nt; ++k) {
    float *cur = u[k & 1], *prv = u[(k + 1) & 1];
    if (G.ndim == 3) {
      Stencil3dArgs a;
      memset(&a, 0, sizeof a);
      a.g = G.fg();
      a.c = lc;
      a.u = cur;
      a.out = prv;
      a.grad = nullptr;
      a.neg_inv_dt2 = neg_inv_dt2;
      a.tbits = tbits;
      a.nzw = G.nzw;
      a.tiles_x = pl.tiles_x;
      a.tiles_y = pl.tiles_y;
      a.flag_tiles_x = G.tiles_x;
      a.flag_tiles_y = G.tiles_y;
      a.zchunk = pl.zchunk;
      a.nzc = pl.nzc;
      a.nitems = pl.nitems;
      a.err = scal;
      a.bx1 = G.nx;  // the whole grid
      a.by1 = G.ny;
      a.bz1 = G.nz;
      a.wait_ns = kWaitLimitNs;
      const CUtensorMap maps[7] = {halo[k & 1], tile[(k + 1) & 1], tb, ts, tb, tb, tile[k & 1]};
      CU(launch_stencil3d_fwd(G.R, pl.grid, st, maps, a));
    } else {
      Stencil2dArgs a;
      memset(&a, 0, sizeof a);
      a.g = G.fg();
      a.c = lc;
      a.u = cur;
      a.um = prv;
      a.b = b;
      a.s = s;
      a.out = prv;
      a.grad = nullptr;
      a.uj = nullptr;
      a.neg_inv_dt2 = neg_inv_dt2;
      CU(launch_stencil2d(G.R, kModeFwd, st, a));
    }
    if (!target.empty()) {
      InjectArgs ia;
      memset(&ia, 0, sizeof ia);
      ia.row_base = nullptr;
      ia.ntarget = int(target.size());
      ia.target = d_target;
      ia.rowptr = d_rowptr;
      ia.pid = d_pid;
      ia.w = d_cw;
      ia.data = wavelet;
      ia.npts = nsrc;
      ia.row = k;
      ia.u = prv;
      ia.b = b;
      ia.grad = nullptr;
      ia.uj = nullptr;
      ia.neg_inv_dt2 = neg_inv_dt2;
      ia.nfield = G.nfield;
      ia.err = scal;
      CU(launch_inject(st, ia));
    }
    if (nrec > 0) {
      InterpArgs pa;
      memset(&pa, 0, sizeof pa);
      pa.row_base = nullptr;
      pa.npts = nrec;
      pa.ncorner = pr.nc;
      pa.idx = d_ridx;
      pa.w = d_rw;
      pa.u = prv;
      pa.out = rec_out;
      pa.row = k;
      pa.nfield = G.nfield;
      pa.err = scal;
      CU(launch_interp(st, pa));
    }
  }
  CU(cudaMemcpyAsync(h, scal, sizeof h, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  if (h[0] != 0) return fail(WP_EDEVICE, "a kernel reported device error %d: %s", h[0], device_error_text(h[0]));
  return WP_OK;
}

extern "C" int wp_forward_noalloc(const wp_grid *grid, const float *m, const float *eta, const float *wavelet,
                                  int nsrc, const double *src_coords, int nrec, const double *rec_coords,
                                  float *rec_out, void *stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  bool touched = false;
  const int rc = forward_noalloc_body(grid, m, eta, wavelet, nsrc, src_coords, nrec, rec_coords, rec_out, st, &touched);
  // after an error, let whatever was queued finish before the caller may reuse the
  // work space (a failed launch leaves earlier kernels running on it)
  if (rc != WP_OK && touched) cudaStreamSynchronize(st);
  return rc;
}
