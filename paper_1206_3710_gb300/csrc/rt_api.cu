// rt_api.cu -- the C ABI of librt.so (declared in include/rt.h): contexts,
// grid flattening, argument validation, job tables, launches, bounded waits.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "rt_internal.cuh"

using namespace rtk;

// ------------------------------------------------------------------------
// errors
// ------------------------------------------------------------------------
static thread_local std::string g_err;

static int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CK(expr)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(e_ == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA, "%s: %s (%s:%d)", \
                  #expr, cudaGetErrorString(e_), __FILE__, __LINE__);                     \
  } while (0)

extern "C" const char* rt_last_error(void) { return g_err.c_str(); }

// lets other translation units of the library report through rt_last_error
namespace rtk {
int set_error(int code, const char* msg) { return fail(code, "%s", msg); }
}  // namespace rtk
extern "C" const char* rt_version(void) { return "librt 0.1 (sm_103a)"; }

// ------------------------------------------------------------------------
// context
// ------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t n = 0;
  int ensure(size_t bytes) {
    if (bytes <= n) return RT_OK;
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
    size_t want = std::max(bytes, (size_t)4096);
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
      p = nullptr;
      return fail(RT_ERR_OOM, "cudaMalloc(%zu) failed: %s", want, cudaGetErrorString(e));
    }
    n = want;
    return RT_OK;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
};

struct rt_ctx {
  int device = 0;
  int sm_count = 0;
  std::mutex mu;
  DevBuf table;        // job tables
  DevBuf small;        // ledgers + counter
  DevBuf scan_tmp;
  DevBuf dust_arrays;  // lambda, kappa_abs, dnu, temperature table
  DevBuf lam;          // Lambda iteration: stored fields, previous T, hits
  std::vector<DevBuf> cdf;  // per dust source
  void* pinned = nullptr;
  size_t pinned_n = 0;
  cudaEvent_t ev_a = nullptr, ev_b = nullptr, ev_c = nullptr, ev_m = nullptr;
  DevBuf peel_q;                          // deferred peel-off records
  DevBuf peel_q2;                         // the same sorted by block of root cells
  long long peel_q_max = 1ll << 27;       // records; 0: peel-off inline
  int tile_edge = -1;                     // tiled tracing: -1 auto, 0 off, > 0 tile edge in root cells
  long long tile_rec_max = 0;             // tiled tracing: record buffer capacity (0: default)
  DevBuf tile_a, tile_b, tile_key, tile_hist;
  unsigned long long* pin_count = nullptr;  // pinned: record count read back per round
  // the event of a wait that ran out of time: that call's kernels and its
  // copies into the pinned buffers may still be running, so the context
  // takes no new work until the event has completed (RT_ERR_BUSY)
  cudaEvent_t busy = nullptr;
  // pinned landing area of the results read back at the end of a call
  // (ledgers, tile status, scalars); only grown while the context is idle
  void* pin_rb = nullptr;
  size_t pin_rb_n = 0;
  // launch defaults chosen by rt_autotune, per [FP64][peel-off]
  struct Tuned {
    bool set = false;
    int block = 256, refill = 8, blocks_per_sm = 0;
  } tuned[2][2];
  int cc_major = 0, cc_minor = 0;
};

struct rt_grid {
  rt_ctx* ctx = nullptr;
  int device = 0;
  int root[3] = {0, 0, 0};
  double box[3] = {0, 0, 0};
  double h0 = 0;
  int n_levels = 0;
  int64_t n_cells = 0, n_leaves = 0, n0 = 0;
  std::vector<long long> level_off;
  float* density = nullptr;
  uint32_t* child = nullptr;
  uint8_t* level = nullptr;
  uint32_t* node = nullptr;
  double* rho64 = nullptr;
  uint64_t* coord = nullptr;
  double* scratch = nullptr;  // [0] densest leaf, [1] invalid-density flag (rt_grid_set_density)
  double rho_scale = 1.0;
  size_t bytes = 0;
};

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int d) {
    cudaGetDevice(&prev);
    if (prev != d) cudaSetDevice(d);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

static int ensure_pinned(rt_ctx* c, size_t bytes) {
  if (bytes <= c->pinned_n) return RT_OK;
  if (c->pinned) cudaFreeHost(c->pinned);
  c->pinned = nullptr;
  c->pinned_n = 0;
  size_t want = std::max(bytes, (size_t)65536);
  cudaError_t e = cudaMallocHost(&c->pinned, want);
  if (e != cudaSuccess) return fail(RT_ERR_OOM, "cudaMallocHost(%zu): %s", want, cudaGetErrorString(e));
  c->pinned_n = want;
  return RT_OK;
}

static int ensure_pin_rb(rt_ctx* c, size_t bytes) {
  if (bytes <= c->pin_rb_n) return RT_OK;
  if (c->pin_rb) cudaFreeHost(c->pin_rb);
  c->pin_rb = nullptr;
  c->pin_rb_n = 0;
  size_t want = std::max(bytes, (size_t)4096);
  cudaError_t e = cudaMallocHost(&c->pin_rb, want);
  if (e != cudaSuccess) return fail(RT_ERR_OOM, "cudaMallocHost(%zu): %s", want, cudaGetErrorString(e));
  c->pin_rb_n = want;
  return RT_OK;
}

extern "C" int rt_ctx_create(int device, rt_ctx** out) {
  if (!out) return fail(RT_ERR_INVALID, "rt_ctx_create: out is NULL");
  *out = nullptr;
  int n = 0;
  CK(cudaGetDeviceCount(&n));
  if (device < 0 || device >= n) return fail(RT_ERR_INVALID, "rt_ctx_create: device %d of %d", device, n);
  DeviceGuard g(device);
  rt_ctx* c = new rt_ctx();
  c->device = device;
  cudaError_t e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->cc_major, cudaDevAttrComputeCapabilityMajor, device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->cc_minor, cudaDevAttrComputeCapabilityMinor, device);
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev_a);
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev_b);
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev_c);
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev_m);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->pin_count, 64);
  if (e != cudaSuccess) {
    delete c;
    return fail(RT_ERR_CUDA, "rt_ctx_create: %s", cudaGetErrorString(e));
  }
  *out = c;
  return RT_OK;
}

extern "C" void rt_ctx_destroy(rt_ctx* c) {
  if (!c) return;
  DeviceGuard g(c->device);
  c->table.release();
  c->small.release();
  c->scan_tmp.release();
  c->dust_arrays.release();
  c->lam.release();
  for (auto& b : c->cdf) b.release();
  if (c->pinned) cudaFreeHost(c->pinned);
  if (c->pin_rb) cudaFreeHost(c->pin_rb);
  if (c->ev_a) cudaEventDestroy(c->ev_a);
  if (c->ev_b) cudaEventDestroy(c->ev_b);
  if (c->ev_c) cudaEventDestroy(c->ev_c);
  if (c->ev_m) cudaEventDestroy(c->ev_m);
  if (c->pin_count) cudaFreeHost(c->pin_count);
  c->peel_q.release();
  c->peel_q2.release();
  c->tile_a.release();
  c->tile_b.release();
  c->tile_key.release();
  c->tile_hist.release();
  delete c;
}

extern "C" int rt_ctx_set_tiles(rt_ctx* c, int tile_edge) {
  if (!c) return fail(RT_ERR_INVALID, "rt_ctx_set_tiles: NULL context");
  if (tile_edge > 0 && (tile_edge & (tile_edge - 1)))
    return fail(RT_ERR_INVALID, "rt_ctx_set_tiles: tile edge must be a power of two");
  std::lock_guard<std::mutex> lk(c->mu);
  c->tile_edge = tile_edge < 0 ? -1 : tile_edge;
  return RT_OK;
}

extern "C" int rt_ctx_set_tile_records(rt_ctx* c, int64_t max_records) {
  if (!c) return fail(RT_ERR_INVALID, "rt_ctx_set_tile_records: NULL context");
  std::lock_guard<std::mutex> lk(c->mu);
  c->tile_rec_max = max_records > 0 ? (long long)max_records : 0;
  return RT_OK;
}

extern "C" int rt_ctx_set_peel_queue(rt_ctx* c, int64_t max_records) {
  if (!c) return fail(RT_ERR_INVALID, "rt_ctx_set_peel_queue: NULL context");
  std::lock_guard<std::mutex> lk(c->mu);
  c->peel_q_max = max_records < 0 ? (1ll << 27) : (long long)max_records;
  return RT_OK;
}

// Queue for the deferred peel-off of one launch: min(max_records, 2 x total)
// records, at least 2^20.  When the device has no room for it the launch
// peels off inline (same results), so an allocation failure is not an error.
static PeelQueue make_queue(DevBuf& buf, long long max_records, bool peel, int n_jobs, long long total,
                            int precision, unsigned long long* count_dev) {
  PeelQueue q;
  q.rec = nullptr;
  q.count = count_dev;
  q.cap = 0;
  if (!peel || max_records <= 0 || n_jobs > RT_PEEL_MAX_JOBS) return q;
  const long long cap = std::min<long long>(max_records, std::max<long long>(2 * total, 1ll << 20));
  if (buf.ensure(peel_record_bytes(precision) * (size_t)cap) != RT_OK) {
    cudaGetLastError();  // allocation failures are not sticky
    return q;
  }
  q.rec = buf.p;
  q.cap = cap;
  return q;
}


// wait for an event with a deadline; the device keeps running on timeout
static int wait_event(cudaEvent_t ev, double timeout_s) {
  const auto t0 = std::chrono::steady_clock::now();
  int spins = 0;
  for (;;) {
    cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return RT_OK;
    if (e != cudaErrorNotReady) return fail(RT_ERR_CUDA, "device error while waiting: %s", cudaGetErrorString(e));
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (el > timeout_s) return fail(RT_ERR_TIMEOUT, "device work did not finish within %.3f s", timeout_s);
    if (++spins > 64) std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

// wait_event for work of the context: on a timeout the context remembers
// the event, because the device may still write into the context's pinned
// buffers and device scratch until that event has completed
static int ctx_wait(rt_ctx* c, cudaEvent_t ev, double timeout_s) {
  const int rc = wait_event(ev, timeout_s);
  if (rc == RT_ERR_TIMEOUT) c->busy = ev;
  return rc;
}

// RT_ERR_BUSY while the work of an earlier call that timed out is still
// running (its kernels use the context's scratch and its copies land in the
// context's pinned buffers)
static int ctx_idle(rt_ctx* c) {
  if (!c->busy) return RT_OK;
  const cudaError_t e = cudaEventQuery(c->busy);
  if (e == cudaErrorNotReady)
    return fail(RT_ERR_BUSY, "the device work of an earlier call that timed out is still running");
  c->busy = nullptr;
  if (e != cudaSuccess) return fail(RT_ERR_CUDA, "device error in the work of an earlier call: %s", cudaGetErrorString(e));
  return RT_OK;
}

// lock the context for one call and check that it is idle
#define CTX_ENTER(c)                       \
  std::lock_guard<std::mutex> lk((c)->mu); \
  do {                                     \
    const int rc_idle_ = ctx_idle(c);      \
    if (rc_idle_) return rc_idle_;         \
  } while (0)

namespace rtk {
int ctx_device(const rt_ctx* c) { return c->device; }
}  // namespace rtk

// ------------------------------------------------------------------------
// grid
// ------------------------------------------------------------------------
extern "C" int rt_build_grid(rt_ctx* ctx, const rt_tree_desc* d, rt_grid** out) {
  if (!ctx || !d || !out) return fail(RT_ERR_INVALID, "rt_build_grid: NULL argument");
  *out = nullptr;
  if (d->root[0] <= 0 || d->root[1] <= 0 || d->root[2] <= 0)
    return fail(RT_ERR_INVALID, "rt_build_grid: root dims must be positive");
  if (d->n_levels <= 0 || d->n_levels > 24 || !d->n_refined || !d->refine_flags || !d->density)
    return fail(RT_ERR_INVALID, "rt_build_grid: bad level count or NULL arrays");
  for (int a = 0; a < 3; ++a)
    if (!(d->box[a] > 0.0) || !std::isfinite(d->box[a])) return fail(RT_ERR_INVALID, "rt_build_grid: bad box size");
  const double h0 = d->box[0] / d->root[0];
  for (int a = 1; a < 3; ++a)
    if (std::fabs(d->box[a] / d->root[a] - h0) > 1e-12 * h0)
      return fail(RT_ERR_INVALID, "rt_build_grid: root cells are not cubic");
  // level sizes
  std::vector<long long> off(d->n_levels + 1, 0);
  long long lvl_n = (long long)d->root[0] * d->root[1] * d->root[2];
  off[1] = lvl_n;
  for (int l = 0; l < d->n_levels; ++l) {
    if (d->n_refined[l] < 0 || d->n_refined[l] > lvl_n)
      return fail(RT_ERR_INVALID, "rt_build_grid: n_refined[%d]=%lld out of range", l, (long long)d->n_refined[l]);
    if (l == d->n_levels - 1 && d->n_refined[l] != 0)
      return fail(RT_ERR_INVALID, "rt_build_grid: deepest level has refined cells");
    if (l + 1 < d->n_levels) {
      lvl_n = 8ll * d->n_refined[l];
      off[l + 2] = off[l + 1] + lvl_n;
    }
  }
  const long long n = off[d->n_levels];
  if (n >= (1ll << 31)) return fail(RT_ERR_INVALID, "rt_build_grid: %lld cells exceed 2^31", n);
  const int depth = d->n_levels - 1;
  for (int a = 0; a < 3; ++a)
    if (((long long)d->root[a] << depth) > (1ll << RT_COORD_BITS))
      return fail(RT_ERR_INVALID, "rt_build_grid: finest lattice exceeds 2^%d cells per axis", RT_COORD_BITS);
  // flags are 0/1 and their per-level counts match
  for (int l = 0; l < d->n_levels; ++l) {
    long long cnt = 0;
    for (long long i = off[l]; i < off[l + 1]; ++i) {
      const uint8_t f = d->refine_flags[i];
      if (f > 1) return fail(RT_ERR_INVALID, "rt_build_grid: refine flag %d at cell %lld", (int)f, i);
      cnt += f;
    }
    if (cnt != d->n_refined[l])
      return fail(RT_ERR_INVALID, "rt_build_grid: level %d has %lld refined cells, n_refined says %lld", l, cnt,
                  (long long)d->n_refined[l]);
  }
  CTX_ENTER(ctx);
  DeviceGuard dg(ctx->device);
  rt_grid* g = new rt_grid();
  g->ctx = ctx;
  g->device = ctx->device;
  memcpy(g->root, d->root, sizeof g->root);
  memcpy(g->box, d->box, sizeof g->box);
  g->h0 = h0;
  g->n_levels = d->n_levels;
  g->n_cells = n;
  g->n0 = off[1];
  g->level_off = off;
  auto cleanup = [&](int rc) -> int {
    rt_grid_free(g);
    return rc;
  };
  uint8_t* flags = nullptr;
  unsigned long long* excl = nullptr;
  double* scal = nullptr;
  int* bad = nullptr;
  const size_t tmpb = scan_tmp_bytes(n);
  void* tmp = nullptr;
  cudaError_t e = cudaSuccess;
#define ALLOC(ptr, bytes)                                                                    \
  do {                                                                                       \
    e = cudaMalloc((void**)&(ptr), (bytes));                                                 \
    if (e != cudaSuccess) {                                                                  \
      cudaFree(flags); cudaFree(excl); cudaFree(scal); cudaFree(bad); cudaFree(tmp);         \
      return cleanup(fail(RT_ERR_OOM, "rt_build_grid: cudaMalloc(%zu): %s", (size_t)(bytes), \
                          cudaGetErrorString(e)));                                           \
    }                                                                                        \
  } while (0)
  ALLOC(g->density, n * sizeof(float));
  ALLOC(g->child, n * sizeof(uint32_t));
  ALLOC(g->level, n * sizeof(uint8_t));
  ALLOC(g->node, n * sizeof(uint32_t));
  ALLOC(g->rho64, n * sizeof(double));
  ALLOC(g->coord, n * sizeof(uint64_t));
  ALLOC(g->scratch, 2 * sizeof(double));
  g->bytes = n * (sizeof(float) + sizeof(uint32_t) * 2 + sizeof(uint8_t) + sizeof(double) + sizeof(uint64_t));
  ALLOC(flags, n);
  ALLOC(excl, n * sizeof(unsigned long long));
  ALLOC(scal, sizeof(double));
  ALLOC(bad, sizeof(int));
  ALLOC(tmp, tmpb);
#undef ALLOC
  auto finish = [&](int rc) -> int {
    cudaFree(flags); cudaFree(excl); cudaFree(scal); cudaFree(bad); cudaFree(tmp);
    if (rc != RT_OK) return cleanup(rc);
    *out = g;
    return RT_OK;
  };
  cudaStream_t s = nullptr;
#define CKG(expr)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (expr);                                                                   \
    if (e_ != cudaSuccess) return finish(fail(RT_ERR_CUDA, "rt_build_grid: %s: %s", #expr, cudaGetErrorString(e_))); \
  } while (0)
  CKG(cudaMemcpyAsync(flags, d->refine_flags, n, cudaMemcpyHostToDevice, s));
  CKG(cudaMemcpyAsync(g->rho64, d->density, n * sizeof(double), cudaMemcpyHostToDevice, s));
  CKG(scan_flags_u8(flags, n, excl, tmp, tmpb, s));
  CKG(build_children(flags, excl, n, off[1], g->child, s));
  CKG(build_levels(off.data(), d->n_levels, g->level, s));
  for (int l = 0; l < d->n_levels; ++l) CKG(build_coords(g->child, off[l], off[l + 1], l == 0 ? d->root : nullptr, g->coord, s));
  CKG(validate_leaf_density(g->rho64, g->child, n, bad, s));
  for (int l = d->n_levels - 2; l >= 0; --l) CKG(build_density(nullptr, g->child, off[l], off[l + 1], g->rho64, s));
  CKG(reduce_max_leaf(g->rho64, g->child, n, scal, s));
  int hbad = 0;
  double hmax = 0.0;
  CKG(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  CKG(cudaMemcpyAsync(&hmax, scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  CKG(cudaStreamSynchronize(s));
  if (hbad) return finish(fail(RT_ERR_INVALID, "rt_build_grid: negative, NaN or infinite leaf density"));
  // f32 node densities span 2^64 down to 2^-126 times rho_scale: the densest
  // leaf sits at 2^64, so leaves down to ~1e-57 of it keep a normal f32
  // density (a near-vacuum cell keeps its absorbed energy per unit mass)
  g->rho_scale = hmax > 0.0 ? std::ldexp(hmax, -64) : 1.0;
  CKG(build_nodes(g->rho64, g->child, n, 1.0 / g->rho_scale, g->density, g->node, s));
  CKG(cudaStreamSynchronize(s));
#undef CKG
  long long leaves = 0;
  for (int l = 0; l < d->n_levels; ++l) leaves += (off[l + 1] - off[l]) - d->n_refined[l];
  g->n_leaves = leaves;
  return finish(RT_OK);
}

extern "C" int rt_grid_get_info(const rt_grid* g, rt_grid_info* o) {
  if (!g || !o) return fail(RT_ERR_INVALID, "rt_grid_get_info: NULL argument");
  o->n_cells = g->n_cells;
  o->n_leaves = g->n_leaves;
  o->depth = g->n_levels - 1;
  memcpy(o->root, g->root, sizeof o->root);
  memcpy(o->box, g->box, sizeof o->box);
  o->bytes = g->bytes;
  o->density = g->density;
  o->child = g->child;
  o->level = g->level;
  o->node = g->node;
  o->density64 = g->rho64;
  o->coord = g->coord;
  o->rho_scale = g->rho_scale;
  return RT_OK;
}

extern "C" void rt_grid_free(rt_grid* g) {
  if (!g) return;
  DeviceGuard dg(g->device);
  cudaFree(g->density);
  cudaFree(g->child);
  cudaFree(g->level);
  cudaFree(g->node);
  cudaFree(g->rho64);
  cudaFree(g->coord);
  cudaFree(g->scratch);
  delete g;
}

// New densities for an existing grid (same tree): upload on the caller's
// stream, validate, interior means, densest leaf (read back: the node words'
// scale), node words.  Nothing is allocated, so work on other streams keeps
// running; the node words are rebuilt stream-ordered after the return.
extern "C" int rt_grid_set_density(rt_ctx* ctx, rt_grid* g, const double* density, void* cuda_stream) {
  if (!ctx || !g || !density) return fail(RT_ERR_INVALID, "rt_grid_set_density: NULL argument");
  if (g->ctx != ctx) return fail(RT_ERR_INVALID, "rt_grid_set_density: the grid belongs to another context");
  CTX_ENTER(ctx);
  DeviceGuard dg(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const long long n = g->n_cells;
  int* bad = reinterpret_cast<int*>(g->scratch + 1);
  int rc = ensure_pin_rb(ctx, 2 * sizeof(double));
  if (rc) return rc;
  CK(cudaMemcpyAsync(g->rho64, density, n * sizeof(double), cudaMemcpyHostToDevice, s));
  CK(validate_leaf_density(g->rho64, g->child, n, bad, s));
  for (int l = g->n_levels - 2; l >= 0; --l)
    CK(build_density(nullptr, g->child, g->level_off[l], g->level_off[l + 1], g->rho64, s));
  CK(reduce_max_leaf(g->rho64, g->child, n, g->scratch, s));
  CK(cudaMemcpyAsync(ctx->pin_rb, g->scratch, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaEventRecord(ctx->ev_c, s));
  rc = ctx_wait(ctx, ctx->ev_c, 3600.0);
  if (rc) return rc;
  double hmax = 0.0;
  int hbad = 0;
  memcpy(&hmax, ctx->pin_rb, sizeof(double));
  memcpy(&hbad, static_cast<char*>(ctx->pin_rb) + sizeof(double), sizeof(int));
  if (hbad)
    return fail(RT_ERR_INVALID, "rt_grid_set_density: negative, NaN or infinite leaf density (the grid's "
                                "densities are undefined until a successful call)");
  g->rho_scale = hmax > 0.0 ? std::ldexp(hmax, -64) : 1.0;
  CK(build_nodes(g->rho64, g->child, n, 1.0 / g->rho_scale, g->density, g->node, s));
  return RT_OK;
}

// ------------------------------------------------------------------------
// job tables
// ------------------------------------------------------------------------
// host-side byte arena mirrored 1:1 into a device buffer
struct Arena {
  std::vector<unsigned char> h;
  size_t put(const void* src, size_t bytes, size_t align = 16) {
    size_t o = (h.size() + align - 1) / align * align;
    h.resize(o + bytes);
    if (src) memcpy(h.data() + o, src, bytes);
    else memset(h.data() + o, 0, bytes);
    return o;
  }
  template <typename T>
  T* at(size_t o) {
    return reinterpret_cast<T*>(h.data() + o);
  }
};

static int check_optics(const rt_optics* op) {
  if (!op || op->n_lambda < 1 || op->n_lambda > RT_MAX_LAMBDA || !op->kappa_ext || !op->albedo || !op->g_hg)
    return fail(RT_ERR_INVALID, "optics: n_lambda must be 1..%d with non-NULL arrays", RT_MAX_LAMBDA);
  for (int b = 0; b < op->n_lambda; ++b) {
    if (!(op->kappa_ext[b] >= 0.0) || !std::isfinite(op->kappa_ext[b]))
      return fail(RT_ERR_INVALID, "optics: kappa_ext[%d] must be finite and >= 0", b);
    if (!(op->albedo[b] >= 0.0 && op->albedo[b] <= 1.0)) return fail(RT_ERR_INVALID, "optics: albedo[%d] not in [0,1]", b);
    if (!(std::fabs(op->g_hg[b]) < 1.0)) return fail(RT_ERR_INVALID, "optics: |g[%d]| must be < 1", b);
  }
  return RT_OK;
}

static int check_dust(const rt_dust* du, int nl) {
  if (!du || du->n_lambda != nl || !du->lambda_um || !du->kappa_abs || !du->dnu)
    return fail(RT_ERR_INVALID, "dust: model must have n_lambda = %d and non-NULL arrays", nl);
  if (!(du->T_min > 0.0) || !(du->T_max > du->T_min) || !std::isfinite(du->T_max))
    return fail(RT_ERR_INVALID, "dust: need 0 < T_min < T_max");
  for (int b = 0; b < nl; ++b)
    if (!(du->lambda_um[b] > 0.0) || !(du->kappa_abs[b] >= 0.0) || !(du->dnu[b] > 0.0) || !std::isfinite(du->kappa_abs[b]))
      return fail(RT_ERR_INVALID, "dust: bad lambda/kappa_abs/dnu at bin %d", b);
  return RT_OK;
}

// Packages per bin in proportion to the bins' energies, at least one in
// every bin that has energy (near-equal package weights, Sect. 4.2).
static void packages_by_energy(const double* e, int n, long long total, long long* out) {
  double tot = 0.0;
  for (int i = 0; i < n; ++i) tot += e[i];
  for (int i = 0; i < n; ++i) {
    long long v = tot > 0 ? (long long)std::floor((double)total * e[i] / tot) : 0;
    if (e[i] > 0 && v == 0) v = 1;
    out[i] = v;
  }
}

// The Lambda drivers' dust: the absorbing part of the optics' extinction,
// kappa_abs = (1 - albedo) kappa_ext (a single dust component, Sect. 3.2),
// when the dust model leaves kappa_abs NULL; else the model as given.
static const rt_dust* resolve_dust(const rt_dust* du, const rt_optics* op, std::vector<double>& kabs, rt_dust& out) {
  if (!du || du->kappa_abs || !op || !op->kappa_ext || !op->albedo || du->n_lambda != op->n_lambda) return du;
  kabs.resize(op->n_lambda);
  for (int b = 0; b < op->n_lambda; ++b) kabs[b] = (1.0 - op->albedo[b]) * op->kappa_ext[b];
  out = *du;
  out.kappa_abs = kabs.data();
  return &out;
}

// upload lambda, kappa_abs, dnu into ctx->dust_arrays (+ table of n_table)
static int upload_dust(rt_ctx* c, const rt_dust* du, int n_table, double** lam, double** kab, double** dnu,
                       double** table, cudaStream_t s) {
  const int nl = du->n_lambda;
  const size_t bytes = sizeof(double) * (3 * (size_t)nl + 3 * (size_t)n_table) + 256;
  int rc = c->dust_arrays.ensure(bytes);
  if (rc) return rc;
  rc = ensure_pinned(c, bytes);
  if (rc) return rc;
  double* hp = reinterpret_cast<double*>(c->pinned);
  memcpy(hp, du->lambda_um, sizeof(double) * nl);
  memcpy(hp + nl, du->kappa_abs, sizeof(double) * nl);
  memcpy(hp + 2 * nl, du->dnu, sizeof(double) * nl);
  double* dp = reinterpret_cast<double*>(c->dust_arrays.p);
  CK(cudaMemcpyAsync(dp, hp, sizeof(double) * 3 * nl, cudaMemcpyHostToDevice, s));
  *lam = dp;
  *kab = dp + nl;
  *dnu = dp + 2 * nl;
  *table = dp + 3 * nl;
  return RT_OK;
}

struct TraceArgs {
  const rt_grid* grid;
  int n_src;
  const rt_source* src;
  const rt_optics* optics;
  const rt_trace_params* prm;
  const rt_observers* obs;
  double* images;
  double* absorbed;
  const rt_peel_tables* tab = nullptr;  // accelerated peel-off tables, or NULL
  int levels = 0;                       // subiterations: absorbed is [n_levels][n_cells] by grid level
  int confine = -1;                     // subiterations: packages leave at grids of level <= confine
  double* self_abs = nullptr;           // ALI: self-absorption tally per cell (levels only)
  double* self_emit = nullptr;          // ALI: energy of the dust packages each cell emitted
  unsigned int* self_cnt = nullptr;     // ALI: their number
  const double* dust_package_energy = nullptr;  // dust sources: host [n_lambda] energy of one package
};

// accelerated peel-off tables (Sect. 2.4)
struct rt_peel_tables {
  rt_ctx* ctx = nullptr;
  const rt_grid* grid = nullptr;
  DevBuf buf;                 // [job record | table]
  const double* table = nullptr;
  long long n = 0;
  PeelTabSpec spec;
  std::vector<double> dirs;   // the observers' directions as given
  int bsh = 0, ssh = 0;
};

// unit observer direction as the job tables compute it
static bool unit_dir(const double* d, double k[3]) {
  const double kn = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  if (!(kn > 0) || !std::isfinite(kn)) return false;
  for (int a = 0; a < 3; ++a) k[a] = d[a] / kn;
  return true;
}

static int max_observers(int n_jobs, const TraceArgs* jobs) {
  int m = 0;
  for (int j = 0; j < n_jobs; ++j)
    if (jobs[j].obs) m = std::max(m, jobs[j].obs->n_obs);
  return m;
}

static void cross3(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

// build the device job table for a list of jobs; returns total packages
static int build_tables(rt_ctx* c, int n_jobs, const TraceArgs* jobs, LedgerDev* led_dev, cudaStream_t s,
                        Arena& A, std::vector<size_t>& job_off, size_t& items_off, int& n_items, long long& total,
                        bool& any_peel, int& precision, int& estimator, DevBuf* table_buf = nullptr,
                        std::vector<DevBuf>* cdf_bufs = nullptr) {
  // device buffers for the table and the dust emission tables: the
  // context's (one-shot calls) or a batch object's (replayed graphs)
  DevBuf& table = table_buf ? *table_buf : c->table;
  std::vector<DevBuf>& cdfv = cdf_bufs ? *cdf_bufs : c->cdf;
  // per job: validate, resolve packages per (source, bin), dust CDFs
  struct Pending {
    size_t ptr_field;  // offset of a pointer field to patch
    size_t target;     // arena offset it must point at
  };
  std::vector<Pending> patches;
  std::vector<ItemDev> items;
  std::vector<std::vector<size_t>> item_patch;  // (bin_prefix, W0, W0f) arena offsets per item
  job_off.assign(n_jobs, 0);
  // the kernel indexes the job records as one contiguous array: reserve it
  // first, per-job data (bins, observers, items) follows
  const size_t jobs_base = A.put(nullptr, sizeof(JobDev) * (size_t)n_jobs);
  total = 0;
  any_peel = false;
  precision = 0;
  int dust_used = 0;
  for (int j = 0; j < n_jobs; ++j) {
    const TraceArgs& T = jobs[j];
    const rt_trace_params* p = T.prm;
    if (!T.grid || !p) return fail(RT_ERR_INVALID, "job %d: NULL grid or params", j);
    if (T.grid->device != c->device) return fail(RT_ERR_INVALID, "job %d: grid belongs to another device", j);
    int rc = check_optics(T.optics);
    if (rc) return rc;
    const int nl = T.optics->n_lambda;
    if (T.n_src < 1 || T.n_src > 256 || !T.src) return fail(RT_ERR_INVALID, "job %d: n_src must be 1..256", j);
    if (p->precision != 32 && p->precision != 64) return fail(RT_ERR_INVALID, "job %d: precision must be 32 or 64", j);
    if (precision && precision != p->precision) return fail(RT_ERR_INVALID, "jobs of one launch must share precision");
    precision = p->precision;
    if (p->estimator != RT_EST_CONTINUOUS && p->estimator != RT_EST_ANALOG)
      return fail(RT_ERR_INVALID, "job %d: unknown estimator", j);
    if (p->packet_offset < 0) return fail(RT_ERR_INVALID, "job %d: packet_offset must be >= 0", j);
    if (j > 0 && p->estimator != estimator) return fail(RT_ERR_INVALID, "jobs of one launch must share the estimator");
    estimator = p->estimator;
    if (p->rr_wmin > 0.0 && !(p->rr_p >= 0.0 && p->rr_p < 1.0)) return fail(RT_ERR_INVALID, "job %d: rr_p must be in [0,1)", j);
    if (p->estimator == RT_EST_ANALOG && p->rr_wmin > 0.0)
      return fail(RT_ERR_INVALID, "job %d: roulette applies to the continuous-absorption estimator only", j);
    if (p->poly_group > 1) {
      if (p->poly_group > 8) return fail(RT_ERR_INVALID, "job %d: poly_group must be 1..8", j);
      if (n_jobs != 1) return fail(RT_ERR_INVALID, "polychromatic packages run one job per call");
      if (p->estimator != RT_EST_CONTINUOUS || p->hits_dev || T.levels || T.tab || p->split_factor > 1)
        return fail(RT_ERR_INVALID, "job %d: polychromatic packages need the continuous estimator, no hits, "
                    "levels, resampling or tabulated peel-off", j);
      for (int si = 0; si < T.n_src; ++si)
        if (T.src[si].kind == RT_SRC_DUST) return fail(RT_ERR_INVALID, "job %d: no polychromatic dust sources", j);
      for (int f = 0; f < nl; f += p->poly_group) {
        const int size = std::min(p->poly_group, nl - f), r = f + (size - 1) / 2;
        bool any = false;
        for (int b = f; b < f + size; ++b) any = any || T.optics->albedo[b] * T.optics->kappa_ext[b] > 0.0;
        if (any && !(T.optics->albedo[r] * T.optics->kappa_ext[r] > 0.0))
          return fail(RT_ERR_INVALID, "job %d: the reference bin %d of a scattering group does not scatter", j, r);
      }
    }
    if (p->split_factor > 1) {
      if (n_jobs != 1) return fail(RT_ERR_INVALID, "resampling runs one job per call");
      if (p->estimator != RT_EST_CONTINUOUS || p->hits_dev || T.levels)
        return fail(RT_ERR_INVALID, "job %d: resampling needs the continuous estimator, no hits or level arrays", j);
      const int depth = T.grid->n_levels - 1;
      const int lm = p->split_max_level < 0 ? depth : std::min(p->split_max_level, depth);
      long long m = 1;
      for (int l = 0; l < lm && m <= 256; ++l) m *= p->split_factor;
      if (m > 256) return fail(RT_ERR_INVALID, "job %d: split_factor^%d exceeds 256 packages per split", j, lm);
    }
    if (T.obs) {
      const rt_observers* o = T.obs;
      if (o->n_obs < 1 || o->n_obs > RT_MAX_OBS || !o->dir || !o->up || o->nx < 1 || o->ny < 1 || !(o->fov[0] > 0) ||
          !(o->fov[1] > 0))
        return fail(RT_ERR_INVALID, "job %d: observers need 1..%d directions, nx, ny, fov > 0", j, RT_MAX_OBS);
      if (!T.images) return fail(RT_ERR_INVALID, "job %d: images buffer is NULL", j);
      any_peel = true;
    }
    const rt_grid* G = T.grid;
    const long long nc = G->n_cells;
    // energies; dust sources: emission per cell and bin (and its totals)
    std::vector<double> energy((size_t)T.n_src * nl, 0.0);
    std::vector<DevBuf*> dust_buf(T.n_src, nullptr);
    for (int si = 0; si < T.n_src; ++si) {
      const rt_source& S = T.src[si];
      if (S.kind == RT_SRC_DUST) {
        if (!S.T_dev) return fail(RT_ERR_INVALID, "job %d source %d: dust source needs T_dev", j, si);
        rc = check_dust(S.dust, nl);
        if (rc) return rc;
        if (nc >= (1ll << 30)) return fail(RT_ERR_INVALID, "job %d source %d: dust sources need < 2^30 cells", j, si);
        if ((int)cdfv.size() <= dust_used) cdfv.resize(dust_used + 1);
        DevBuf& cb = cdfv[dust_used++];
        // [emission nl x nc f64 | first package per cell nl x (nc + 1) i64 | totals nl | w nl]
        rc = cb.ensure(sizeof(double) * ((size_t)nl * nc + (size_t)nl * (nc + 1) + 2 * (size_t)nl) + 256);
        if (rc) return rc;
        double *lam, *kab, *dnu, *tab;
        rc = upload_dust(c, S.dust, 0, &lam, &kab, &dnu, &tab, s);
        if (rc) return rc;
        double* em = reinterpret_cast<double*>(cb.p);
        double* tot = em + (size_t)nl * nc + (size_t)nl * (nc + 1);
        CK(dust_emission(S.T_dev, nc, G->child, G->rho64, G->level, G->h0, lam, kab, dnu, nl, em, s));
        CK(row_sums_f64(em, nl, nc, tot, s));
        rc = ensure_pin_rb(c, sizeof(double) * (size_t)nl);
        if (rc) return rc;
        CK(cudaMemcpyAsync(c->pin_rb, tot, sizeof(double) * (size_t)nl, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int b = 0; b < nl; ++b) energy[(size_t)si * nl + b] = static_cast<const double*>(c->pin_rb)[b];
        dust_buf[si] = &cb;
      } else if (S.kind == RT_SRC_POINT || S.kind == RT_SRC_EXTERNAL || S.kind == RT_SRC_BEAM) {
        if (!S.bin_energy) return fail(RT_ERR_INVALID, "job %d source %d: bin_energy is NULL", j, si);
        for (int b = 0; b < nl; ++b) {
          if (!(S.bin_energy[b] >= 0.0) || !std::isfinite(S.bin_energy[b]))
            return fail(RT_ERR_INVALID, "job %d source %d: bin_energy[%d] must be finite and >= 0", j, si, b);
          energy[(size_t)si * nl + b] = S.bin_energy[b];
        }
        if (S.kind == RT_SRC_BEAM) {
          const double n2 = S.dir[0] * S.dir[0] + S.dir[1] * S.dir[1] + S.dir[2] * S.dir[2];
          if (!(n2 > 0.0) || !std::isfinite(n2)) return fail(RT_ERR_INVALID, "job %d source %d: beam dir is zero", j, si);
        }
        for (int a = 0; a < 3; ++a)
          if (!std::isfinite(S.pos[a])) return fail(RT_ERR_INVALID, "job %d source %d: pos not finite", j, si);
      } else {
        return fail(RT_ERR_INVALID, "job %d source %d: unknown kind %d", j, si, S.kind);
      }
    }
    // packages per (source, bin)
    std::vector<long long> pk((size_t)T.n_src * nl, 0);
    if (p->packets_per_bin > 0) {
      std::fill(pk.begin(), pk.end(), (long long)p->packets_per_bin);
    } else if (p->packets_total > 0) {
      packages_by_energy(energy.data(), (int)energy.size(), p->packets_total, pk.data());
    } else if (p->packets) {
      for (size_t i = 0; i < pk.size(); ++i) {
        if (p->packets[i] < 0) return fail(RT_ERR_INVALID, "job %d: negative package count", j);
        pk[i] = p->packets[i];
      }
    } else {
      return fail(RT_ERR_INVALID, "job %d: set packets_per_bin, packets_total or packets", j);
    }
    if (p->packet_log_dev && p->packet_log_rows <= 0)
      return fail(RT_ERR_INVALID, "job %d: packet_log_rows must give the rows of packet_log_dev", j);
    // polychromatic: packages per group, counted at the group's first bin
    const int poly = p->poly_group > 1 ? p->poly_group : 1;
    if (poly > 1)
      for (int si = 0; si < T.n_src; ++si)
        for (int f = 0; f < nl; f += poly) {
          const int size = std::min(poly, nl - f);
          long long n = 0;
          if (p->packets_per_bin > 0 || p->packets) {
            n = pk[(size_t)si * nl + f];
          } else {
            for (int b = f; b < f + size; ++b) n += pk[(size_t)si * nl + b];
          }
          for (int b = f; b < f + size; ++b) pk[(size_t)si * nl + b] = b == f ? n : 0;
        }
    // Dust sources (Sect. 4.2): every package of a bin carries the same
    // energy w_b (the bin's emission over its packages, or the energy given
    // by the caller), and each cell sends floor(E_bc / w_b + u_bc) of them;
    // pk becomes the packages actually sent
    std::vector<double> w_dust((size_t)T.n_src * nl, 0.0);
    for (int si = 0; si < T.n_src; ++si) {
      if (T.src[si].kind != RT_SRC_DUST) continue;
      double* em = reinterpret_cast<double*>(dust_buf[si]->p);
      long long* first = reinterpret_cast<long long*>(em + (size_t)nl * nc);
      double* wd = em + (size_t)nl * nc + (size_t)nl * (nc + 1) + nl;
      for (int b = 0; b < nl; ++b) {
        const size_t q = (size_t)si * nl + b;
        const double e = energy[q];
        double w = 0.0;
        if (e > 0.0 && pk[q] > 0) w = T.dust_package_energy ? T.dust_package_energy[b] : e / (double)pk[q];
        w_dust[q] = w > 0.0 && std::isfinite(w) ? w : 0.0;
      }
      rc = ensure_pinned(c, sizeof(double) * (size_t)nl);
      if (rc) return rc;
      memcpy(c->pinned, w_dust.data() + (size_t)si * nl, sizeof(double) * (size_t)nl);
      CK(cudaMemcpyAsync(wd, c->pinned, sizeof(double) * (size_t)nl, cudaMemcpyHostToDevice, s));
      CK(dust_counts(em, nc, nl, wd, (uint32_t)p->seed ^ p->job, (uint32_t)(p->seed >> 32) ^ p->iter, (uint32_t)si,
                     first, s));
      rc = c->scan_tmp.ensure(scan_rows_tmp_bytes(nl, nc + 1));
      if (rc) return rc;
      CK(scan_rows_i64_excl(first, nl, nc + 1, c->scan_tmp.p, c->scan_tmp.n, s));
      rc = ensure_pin_rb(c, sizeof(long long) * (size_t)nl);
      if (rc) return rc;
      for (int b = 0; b < nl; ++b)
        CK(cudaMemcpyAsync(static_cast<long long*>(c->pin_rb) + b, first + (size_t)b * (nc + 1) + nc, sizeof(long long),
                           cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (int b = 0; b < nl; ++b) pk[(size_t)si * nl + b] = static_cast<const long long*>(c->pin_rb)[b];
    }
    // job entry
    JobDev J;
    memset(&J, 0, sizeof J);
    J.node = G->node;
    J.rho64 = G->rho64;
    J.coord = G->coord;
    J.level = G->level;
    for (int a = 0; a < 3; ++a) J.root[a] = (uint32_t)G->root[a];
    J.depth = G->n_levels - 1;
    J.h0 = G->h0;
    J.n_lambda = nl;
    J.estimator = p->estimator;
    J.n_cells = nc;
    J.absorbed = T.absorbed;
    J.abs_bins = p->per_lambda ? nl : 1;
    J.img_bins = p->per_lambda ? nl : 1;
    J.images = T.images;
    J.n_obs = T.obs ? T.obs->n_obs : 0;
    J.packet_log = p->packet_log_dev;
    J.hits = p->hits_dev;
    J.ledger = led_dev + j;
    J.seed = p->seed;
    J.job_id = p->job;
    J.iter = p->iter;
    J.rr_wmin = p->rr_wmin;
    J.rr_p = p->rr_p;
    J.step_limit = p->step_limit > 0 ? p->step_limit : 100000000ll;
    J.peel_tau_max = p->peel_tau_max;
    J.rr_wmin_f = (float)p->rr_wmin;
    J.rr_p_f = (float)p->rr_p;
    J.peel_tau_max_f = (float)p->peel_tau_max;
    J.pkt_offset = p->packet_offset;
    J.sub_conf = T.confine;
    J.thin64 = p->thin_f64 ? 1 : 0;
    J.split_n = p->split_factor > 1 ? p->split_factor : 1;
    J.poly_n = poly;
    J.split_lmax = p->split_max_level < 0 ? G->n_levels - 1 : std::min(p->split_max_level, G->n_levels - 1);
    J.self_abs = T.levels ? T.self_abs : nullptr;
    J.self_emit = T.levels ? T.self_emit : nullptr;
    J.self_cnt = T.levels ? T.self_cnt : nullptr;
    if (T.levels && (T.obs || nl < 1)) return fail(RT_ERR_INVALID, "job %d: level arrays exclude peel-off", j);
    if (T.tab) {
      if (T.tab->grid != G || !T.obs || T.obs->n_obs != T.tab->spec.n_obs)
        return fail(RT_ERR_INVALID, "job %d: peel-off tables were built for another grid or observer set", j);
      for (int o = 0; o < T.obs->n_obs; ++o)
        for (int a = 0; a < 3; ++a)
          if (T.obs->dir[3 * o + a] != T.tab->dirs[3 * o + a])
            return fail(RT_ERR_INVALID, "job %d: observer %d differs from the tables' observer", j, o);
      J.ptab = T.tab->table;
      J.ptab_bsh = T.tab->bsh;
      J.ptab_ssh = T.tab->ssh;
      J.ptab_nbx = T.tab->spec.nb[0];
      J.ptab_nby = T.tab->spec.nb[1];
    }
    double w0_max = 0.0;
    for (size_t i = 0; i < pk.size(); ++i)
      if (pk[i] > 0) w0_max = std::max(w0_max, energy[i] / (double)pk[i]);
    J.led_shift = ledger_shift(w0_max, p->rr_wmin, p->rr_p);
    const size_t jo = jobs_base + (size_t)j * sizeof(JobDev);
    memcpy(A.h.data() + jo, &J, sizeof J);
    job_off[j] = jo;
    // bins
    std::vector<BinDev> bins(nl);
    for (int b = 0; b < nl; ++b) {
      BinDev& B = bins[b];
      memset(&B, 0, sizeof B);
      B.kext_d = T.optics->kappa_ext[b] * G->h0;
      B.kext_f = (float)(T.optics->kappa_ext[b] * G->h0 * G->rho_scale);
      B.albedo = (float)T.optics->albedo[b];
      B.g = (float)T.optics->g_hg[b];
      B.albedo_d = T.optics->albedo[b];
      B.g_d = T.optics->g_hg[b];
    }
    const size_t bo = A.put(bins.data(), sizeof(BinDev) * nl);
    patches.push_back({jo + offsetof(JobDev, bins), bo});
    // observers
    if (T.obs) {
      std::vector<ObsDev> ob(T.obs->n_obs);
      for (int o = 0; o < T.obs->n_obs; ++o) {
        ObsDev& O = ob[o];
        memset(&O, 0, sizeof O);
        double k[3];
        if (!unit_dir(&T.obs->dir[3 * o], k)) return fail(RT_ERR_INVALID, "job %d observer %d: zero direction", j, o);
        if (T.tab) {
          O.tab_off = T.tab->spec.off[o];
          O.tab_naxes = T.tab->spec.n_axes[o];
          for (int a = 0; a < 3; ++a) O.tab_slot[a] = 0;
          for (int s2 = 0; s2 < T.tab->spec.n_axes[o]; ++s2) O.tab_slot[T.tab->spec.axes[o][s2]] = s2;
        }
        double ex[3], ey[3];
        cross3(&T.obs->up[3 * o], k, ex);
        const double en = std::sqrt(ex[0] * ex[0] + ex[1] * ex[1] + ex[2] * ex[2]);
        if (!(en > 1e-12)) return fail(RT_ERR_INVALID, "job %d observer %d: up is parallel to dir", j, o);
        for (double& v : ex) v /= en;
        cross3(k, ex, ey);
        for (int a = 0; a < 3; ++a) {
          O.k[a] = k[a];
          O.ex[a] = ex[a];
          O.ey[a] = ey[a];
          O.c[a] = 0.5 * G->root[a];
        }
        O.inv_pix[0] = T.obs->nx * G->h0 / T.obs->fov[0];
        O.inv_pix[1] = T.obs->ny * G->h0 / T.obs->fov[1];
        for (int a = 0; a < 3; ++a) {
          O.kf[a] = (float)O.k[a];
          O.exf[a] = (float)O.ex[a];
          O.eyf[a] = (float)O.ey[a];
          O.cf[a] = (float)O.c[a];
        }
        O.inv_pixf[0] = (float)O.inv_pix[0];
        O.inv_pixf[1] = (float)O.inv_pix[1];
        O.nx = T.obs->nx;
        O.ny = T.obs->ny;
      }
      const size_t oo = A.put(ob.data(), sizeof(ObsDev) * ob.size());
      patches.push_back({jo + offsetof(JobDev, obs), oo});
    }
    // the package log must have a row for every package
    if (p->packet_log_dev) {
      long long n_job = 0;
      for (long long v : pk) n_job += v;
      if (n_job > p->packet_log_rows)
        return fail(RT_ERR_INVALID, "job %d: the launch has %lld packages, packet_log_rows is %lld", j, n_job,
                    (long long)p->packet_log_rows);
    }
    // items
    long long log_off = 0;
    for (int si = 0; si < T.n_src; ++si) {
      const rt_source& S = T.src[si];
      ItemDev I;
      memset(&I, 0, sizeof I);
      I.job = j;
      I.kind = S.kind;
      I.src_index = (uint32_t)si;
      for (int a = 0; a < 3; ++a) I.pos[a] = S.pos[a] / G->h0;
      if (S.kind == RT_SRC_BEAM) {
        const double n2 = std::sqrt(S.dir[0] * S.dir[0] + S.dir[1] * S.dir[1] + S.dir[2] * S.dir[2]);
        for (int a = 0; a < 3; ++a) I.dir[a] = S.dir[a] / n2;
      }
      for (int a = 0; a < 3; ++a) {
        I.posf[a] = (float)I.pos[a];
        I.dirf[a] = (float)I.dir[a];
      }
      std::vector<long long> pref(nl + 1, 0);
      std::vector<double> w0(nl, 0.0);
      std::vector<float> w0f(nl, 0.0f);
      for (int b = 0; b < nl; ++b) {
        const long long np_ = pk[(size_t)si * nl + b];
        pref[b + 1] = pref[b] + np_;
        // polychromatic: every bin of a group shares the group's packages
        const long long ng = poly > 1 ? pk[(size_t)si * nl + (b / poly) * poly] : np_;
        w0[b] = ng > 0 ? energy[(size_t)si * nl + b] / (double)ng : 0.0;
        if (S.kind == RT_SRC_DUST) w0[b] = w_dust[(size_t)si * nl + b];
        w0f[b] = (float)w0[b];
      }
      I.pkt_begin = total;
      I.pkt_end = total + pref[nl];
      I.log_offset = log_off;
      I.dust_first = S.kind == RT_SRC_DUST
                         ? reinterpret_cast<const long long*>(reinterpret_cast<double*>(dust_buf[si]->p) + (size_t)nl * nc)
                         : nullptr;
      total += pref[nl];
      log_off += pref[nl];
      const size_t po = A.put(pref.data(), sizeof(long long) * (nl + 1));
      const size_t wo = A.put(w0.data(), sizeof(double) * nl);
      const size_t wfo = A.put(w0f.data(), sizeof(float) * nl);
      if (pref[nl] == 0) continue;  // nothing to emit
      items.push_back(I);
      item_patch.push_back({po, wo, wfo});
    }
  }
  // items array
  n_items = (int)items.size();
  items_off = A.put(items.data(), sizeof(ItemDev) * std::max<size_t>(items.size(), 1));
  for (int i = 0; i < n_items; ++i) {
    patches.push_back({items_off + i * sizeof(ItemDev) + offsetof(ItemDev, bin_prefix), item_patch[i][0]});
    patches.push_back({items_off + i * sizeof(ItemDev) + offsetof(ItemDev, W0), item_patch[i][1]});
    patches.push_back({items_off + i * sizeof(ItemDev) + offsetof(ItemDev, W0f), item_patch[i][2]});
  }
  // device copy, pointer fix-ups
  int rc = table.ensure(A.h.size() + 256);
  if (rc) return rc;
  char* base = reinterpret_cast<char*>(table.p);
  for (const Pending& pp : patches) {
    void* v = base + pp.target;
    memcpy(A.h.data() + pp.ptr_field, &v, sizeof(void*));
  }
  rc = ensure_pinned(c, A.h.size());
  if (rc) return rc;
  memcpy(c->pinned, A.h.data(), A.h.size());
  CK(cudaMemcpyAsync(base, c->pinned, A.h.size(), cudaMemcpyHostToDevice, s));
  return RT_OK;
}

static int default_refill(int precision, bool peel) {
  (void)precision;
  (void)peel;
  return 8;
}

// launch configuration: explicit params, else the autotuned default, else 256/8
// Levels of the path a tracer lane stores: the deepest grid's depth (at
// most RT_ANC_MAX) when some grid has at least half of its cells below its
// two top levels, else 0 (no path).  Moves out of an octet below level 1
// are what the path shortens; on a grid whose cells are mostly in the top
// two levels they are few, and the path's registers and shared memory cost
// more than it saves (the 256^3 cloud refined 3 levels: 16 % of its cells
// below level 1, tracer 1.6 % and peel-off 8 % slower with the path; the
// same cloud refined to 8 % of the uniform cells, 87 %: 3 % faster; the
// disc, 97 %: 26 % faster).
static int path_levels(int n_jobs, const TraceArgs* jobs) {
  int d = 0;
  bool deep = false;
  for (int j = 0; j < n_jobs; ++j) {
    const rt_grid* G = jobs[j].grid;
    d = std::max(d, G->n_levels - 1);
    if (G->n_levels > 2 && 2 * (G->n_cells - G->level_off[2]) >= G->n_cells) deep = true;
  }
  return deep ? std::min(d, RT_ANC_MAX) : 0;
}

static int make_cfg(rt_ctx* c, int precision, bool peel, const rt_trace_params* lp, int anc, LaunchCfg* cfg) {
  const rt_ctx::Tuned& t = c->tuned[precision == 64][peel ? 1 : 0];
  cfg->block = lp->block_size > 0 ? lp->block_size : (t.set ? t.block : 256);
  if (cfg->block % 32 || cfg->block > 256 || cfg->block < 32)
    return fail(RT_ERR_INVALID, "block_size must be a multiple of 32 in 32..256");
  cfg->anc = anc;
  int occ = 0;
  CK(trace_occupancy(precision, peel, cfg->block, &occ, 0, anc));
  if (occ < 1) occ = 1;
  const int bps = lp->blocks_per_sm > 0 ? lp->blocks_per_sm : (t.set ? t.blocks_per_sm : 0);
  if (bps > 0) occ = std::min(occ, bps);
  cfg->blocks = c->sm_count * occ;
  int occ2 = 0;
  CK(trace_occupancy(precision, peel, cfg->block, &occ2, 2, anc));
  if (occ2 < 1) occ2 = 1;
  if (bps > 0) occ2 = std::min(occ2, bps);
  cfg->blocks_tiled = c->sm_count * occ2;
  cfg->refill = lp->refill_threshold > 0 ? lp->refill_threshold : (t.set ? t.refill : default_refill(precision, peel));
  if (cfg->refill > 32) cfg->refill = 32;
  return RT_OK;
}

// Tiled tracing pays off when one wavelength's working set (4-byte node word
// and 8-byte accumulator per cell) is well above the L2 (129 MB on GB300):
// the root grid is cut into tiles of edge 2^tsh root cells whose working set
// is at most 48 MB.  Single-job launches only.
static bool choose_tiles(const rt_ctx* c, const rt_grid* G, int n_jobs, TileRun* T) {
  if (n_jobs != 1 || c->tile_edge == 0) return false;
  const int* R = G->root;
  auto count = [&](int edge) {
    return (long long)((R[0] + edge - 1) / edge) * ((R[1] + edge - 1) / edge) * ((R[2] + edge - 1) / edge);
  };
  int edge = c->tile_edge;
  if (edge < 0) {
    const double ws = 12.0 * (double)G->n_cells, cap = 48.0 * 1024 * 1024;
    if (ws <= cap) return false;
    const double need = ws / cap;
    edge = 1;
    while (edge * 2 <= std::max(R[0], std::max(R[1], R[2]))) edge *= 2;
    while (edge > 1 && count(edge) < need) edge /= 2;
  }
  while (count(edge) > 512) edge *= 2;  // key space: bins x tiles
  if (count(edge) < 2) return false;
  int tsh = 0;
  while ((1 << tsh) < edge) ++tsh;
  memset(T, 0, sizeof *T);
  T->tsh = tsh;
  T->ntx = (R[0] + edge - 1) / edge;
  T->nty = (R[1] + edge - 1) / edge;
  T->n_tiles = (int)count(edge);
  return true;
}

// Tiled run of one job: emit the packages chunk by chunk into records, then
// sort by (bin, tile) and trace round after round until no package is left.
// With resampling the record buffers also take the copies of split
// packages: the emission chunks are a quarter of the buffer, and each
// round may add as many copies as the buffer has room for beyond its input.
static int run_tiled(rt_ctx* c, TileRun T, int n_lambda, int precision, bool peel, int estimator, bool hits,
                     const JobDev* jobs_dev, const ItemDev* items_dev, int n_items, long long total,
                     const LaunchCfg& cfg, const PeelQueue& q, unsigned long long* counter,
                     unsigned long long* n_out, int* status, double timeout_s, cudaStream_t s,
                     long long* launches, int* rounds, bool levels, bool split, unsigned long long* n_split) {
  const long long cap_max = precision == 64 ? (1ll << 25) : (1ll << 26);
  const long long cap = c->tile_rec_max > 0 ? std::min(c->tile_rec_max, cap_max) : cap_max;
  const long long chunk = std::min<long long>(total, split ? cap / 4 : cap);
  const long long rec_cap = split ? std::min(cap, std::max(16 * chunk, 1ll << 20)) : chunk;
  const size_t rb = tile_record_bytes(precision, levels || split);
#ifndef RT_TILE_SUB_BITS
#define RT_TILE_SUB_BITS 0
#endif
  T.sbits = std::min(RT_TILE_SUB_BITS, T.tsh);
  const int n_keys = (n_lambda * T.n_tiles) << (3 * T.sbits);
  int rc = c->tile_a.ensure(rb * (size_t)rec_cap);
  if (!rc) rc = c->tile_b.ensure(rb * (size_t)rec_cap);
  if (!rc) rc = c->tile_key.ensure(sizeof(uint32_t) * (size_t)rec_cap);
  if (!rc) rc = c->tile_hist.ensure(sizeof(unsigned long long) * ((size_t)n_keys + 1));
  if (rc) return rc;
  T.out_key = reinterpret_cast<uint32_t*>(c->tile_key.p);
  T.n_out = n_out;
  T.cap_out = rec_cap;
  T.status = status;
  T.n_split = n_split;
  T.split_cap = 0;
  for (long long c0 = 0; c0 < total; c0 += chunk) {
    const long long c1 = std::min(total, c0 + chunk);
    CK(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(n_out, 0, sizeof(unsigned long long), s));
    T.in = nullptr;
    T.out = c->tile_a.p;
    T.first = c0;
    T.split_cap = 0;
    CK(launch_trace(precision, peel, estimator, hits, jobs_dev, items_dev, n_items, counter, c1, cfg, q, s, 1, &T,
                    levels, split));
    *launches += 1;
    for (long long round = 0;; ++round) {
      if (round > 10000000) return fail(RT_ERR_CUDA, "tiled tracing did not finish");
      CK(cudaMemcpyAsync(c->pin_count, n_out, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
      CK(cudaEventRecord(c->ev_c, s));
      rc = ctx_wait(c, c->ev_c, timeout_s);
      if (rc) return rc;
      const long long n = (long long)c->pin_count[0];
      if (n == 0) break;
      if (n > rec_cap) return fail(RT_ERR_CUDA, "tile record buffer overflow (%lld > %lld)", n, rec_cap);
      CK(tile_sort(c->tile_a.p, T.out_key, n, (int)rb, n_keys, reinterpret_cast<unsigned long long*>(c->tile_hist.p),
                   c->tile_b.p, s));
      CK(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s));
      CK(cudaMemsetAsync(n_out, 0, sizeof(unsigned long long), s));
      T.in = c->tile_b.p;
      T.out = c->tile_a.p;
      T.first = 0;
      T.split_cap = rec_cap - n;
      if (split) CK(cudaMemsetAsync(n_split, 0, sizeof(unsigned long long), s));
      CK(launch_trace(precision, peel, estimator, hits, jobs_dev, items_dev, n_items, counter, n, cfg, q, s, 2, &T,
                      levels, split));
      *launches += 4;  // histogram, scan, scatter, tracer
      *rounds += 1;
    }
  }
  return RT_OK;
}

// Deferred peel-off records sorted by block of root cells (at most
// RT_PEEL_SORT_KEYS blocks of the first job's root grid: 4^3 root cells on a
// 256^3 root), so that the lanes of a warp march from nearby points: the
// queue length is read back (the tracer has finished), the records are
// counting-sorted into a second buffer.
#ifndef RT_PEEL_SORT
#define RT_PEEL_SORT 1
#endif
#ifndef RT_PEEL_SORT_KEYS
#define RT_PEEL_SORT_KEYS 262144
#endif
static int sort_peel_queue(rt_ctx* c, const PeelQueue& q, int precision, const rt_grid* G, double timeout_s,
                           cudaStream_t s, PeelQueue* out, long long* launches) {
  *out = q;
  CK(cudaMemcpyAsync(c->pin_count, q.count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  CK(cudaEventRecord(c->ev_c, s));
  int rc = ctx_wait(c, c->ev_c, timeout_s);
  if (rc) return rc;
  const long long n = std::min<long long>((long long)c->pin_count[0], q.cap);
  if (n < 64) return RT_OK;
  int bs = 0;
  auto nb = [&](int r) { return (r + (1 << bs) - 1) >> bs; };
  while ((long long)nb(G->root[0]) * nb(G->root[1]) * nb(G->root[2]) > RT_PEEL_SORT_KEYS) ++bs;
  const int n_keys = nb(G->root[0]) * nb(G->root[1]) * nb(G->root[2]);
  const size_t rb = peel_record_bytes(precision);
  rc = c->peel_q2.ensure(rb * (size_t)n);
  if (!rc) rc = c->tile_key.ensure(sizeof(uint32_t) * (size_t)n);
  if (!rc) rc = c->tile_hist.ensure(sizeof(unsigned long long) * ((size_t)n_keys + 1));
  if (rc == RT_ERR_OOM) {
    cudaGetLastError();  // no room for the sorted copy: march the queue as it is
    return RT_OK;
  }
  if (rc) return rc;
  uint32_t* key = reinterpret_cast<uint32_t*>(c->tile_key.p);
  CK(peel_keys(precision, q.rec, n, bs, nb(G->root[0]), nb(G->root[1]), nb(G->root[2]), key, c->sm_count, s));
  CK(tile_sort(q.rec, key, n, (int)rb, n_keys, reinterpret_cast<unsigned long long*>(c->tile_hist.p), c->peel_q2.p,
               s));
  out->rec = c->peel_q2.p;
  *launches += 4;  // keys, histogram, scan, scatter
  return RT_OK;
}

static int run_jobs(rt_ctx* c, int n_jobs, const TraceArgs* jobs, rt_ledger* ledgers, cudaStream_t s,
                    const rt_trace_params* launch_prm) {
  // ledgers + package counter
  int rc = c->small.ensure(sizeof(LedgerDev) * n_jobs + 256);
  if (rc) return rc;
  LedgerDev* led = reinterpret_cast<LedgerDev*>(c->small.p);
  // package counter, peel-off queue length, peel-off work counter
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(led + n_jobs);
  Arena A;
  std::vector<size_t> job_off;
  size_t items_off = 0;
  int n_items = 0, precision = 32, estimator = RT_EST_CONTINUOUS;
  long long total = 0;
  bool peel = false;
  rc = build_tables(c, n_jobs, jobs, led, s, A, job_off, items_off, n_items, total, peel, precision, estimator);
  if (rc) return rc;
  char* base = reinterpret_cast<char*>(c->table.p);
  // counter[0] packages, [1] peel-off queue length, [2] peel-off work,
  // [3] tile records written, [4] tile status, [5] split copies this round
  CK(cudaMemsetAsync(c->small.p, 0, sizeof(LedgerDev) * n_jobs + 6 * sizeof(unsigned long long), s));
  // polychromatic packages: their own tracer, peel-off inline
  const bool poly = n_jobs == 1 && jobs[0].prm->poly_group > 1;
  const PeelQueue q = make_queue(c->peel_q, c->peel_q_max, peel && !poly, n_jobs, total, precision, counter + 1);
  LaunchCfg cfg;
  rc = make_cfg(c, precision, peel, launch_prm, path_levels(n_jobs, jobs), &cfg);
  if (rc) return rc;
  bool hits = false;
  for (int j = 0; j < n_jobs; ++j) hits = hits || jobs[j].prm->hits_dev != nullptr;
  if (hits && (peel || estimator != RT_EST_CONTINUOUS))
    return fail(RT_ERR_INVALID, "hit counting needs rt_trace with the continuous estimator");
  const double to = launch_prm->timeout_s > 0 ? launch_prm->timeout_s : 3600.0;
  TileRun tiles;
  bool tiled = !poly && total > 0 && n_items > 0 && choose_tiles(c, jobs[0].grid, n_jobs, &tiles);
  const bool split = n_jobs == 1 && jobs[0].prm->split_factor > 1;
  if (split && total > 0 && n_items > 0 && !tiled) {
    // resampling runs in the rounds of the tiled tracer: one tile
    const int* R = jobs[0].grid->root;
    int tsh = 0;
    while ((1 << tsh) < std::max(R[0], std::max(R[1], R[2]))) ++tsh;
    memset(&tiles, 0, sizeof tiles);
    tiles.tsh = tsh;
    tiles.ntx = tiles.nty = 1;
    tiles.n_tiles = 1;
    tiled = true;
  }
  int* tile_status = reinterpret_cast<int*>(counter + 4);
  long long n_launch = 0;
  int n_rounds = 0;
  CK(cudaEventRecord(c->ev_a, s));
  if (tiled) {
    rc = run_tiled(c, tiles, jobs[0].optics->n_lambda, precision, peel, estimator, hits,
                   reinterpret_cast<const JobDev*>(base + job_off[0]), reinterpret_cast<const ItemDev*>(base + items_off),
                   n_items, total, cfg, q, counter, counter + 3, tile_status, to, s, &n_launch, &n_rounds,
                   jobs[0].levels != 0, split, counter + 5);
    if (rc) return rc;
  } else if (poly && total > 0 && n_items > 0) {
    CK(launch_poly(precision, jobs[0].prm->poly_group, peel, reinterpret_cast<const JobDev*>(base + job_off[0]),
                   reinterpret_cast<const ItemDev*>(base + items_off), n_items, counter, total, c->sm_count, s));
    n_launch = 1;
  } else if (total > 0 && n_items > 0) {
    CK(launch_trace(precision, peel, estimator, hits, reinterpret_cast<const JobDev*>(base + job_off[0]),
                    reinterpret_cast<const ItemDev*>(base + items_off), n_items, counter, total, cfg, q, s, 0,
                    nullptr, n_jobs == 1 && jobs[0].levels != 0));
    n_launch = 1;
  }
  if (total > 0 && n_items > 0 && q.cap > 0) n_launch += 1;  // the deferred peel-off
  CK(cudaEventRecord(c->ev_m, s));
  if (total > 0 && n_items > 0 && q.cap > 0) {
    PeelQueue qs = q;
#if RT_PEEL_SORT
    rc = sort_peel_queue(c, q, precision, jobs[0].grid, to, s, &qs, &n_launch);
    if (rc) return rc;
#endif
    if (n_jobs == 1 && jobs[0].tab)
      CK(launch_peel_tab(precision, reinterpret_cast<const JobDev*>(base + job_off[0]), qs, counter + 2,
                         max_observers(n_jobs, jobs), cfg.refill, s, cfg.anc));
    else
      CK(launch_peel(precision, reinterpret_cast<const JobDev*>(base + job_off[0]), qs, counter + 2,
                     max_observers(n_jobs, jobs), cfg.refill, s, cfg.anc));
  }
  CK(cudaEventRecord(c->ev_b, s));
  // ledgers and tile status land in the context's pinned read-back area and
  // are read only after the event behind the copies has completed: a wait
  // that runs out leaves no copy pending into caller or stack memory
  const size_t led_bytes = sizeof(LedgerDev) * (size_t)n_jobs;
  rc = ensure_pin_rb(c, led_bytes + sizeof(int));
  if (rc) return rc;
  CK(cudaMemcpyAsync(c->pin_rb, led, led_bytes, cudaMemcpyDeviceToHost, s));
  if (tiled)
    CK(cudaMemcpyAsync(static_cast<char*>(c->pin_rb) + led_bytes, tile_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaEventRecord(c->ev_c, s));
  rc = ctx_wait(c, c->ev_c, to);
  if (rc) return rc;
  std::vector<LedgerDev> hl(n_jobs);
  memcpy(hl.data(), c->pin_rb, led_bytes);
  int tstat = 0;
  if (tiled) memcpy(&tstat, static_cast<const char*>(c->pin_rb) + led_bytes, sizeof(int));
  if (tstat) return fail(RT_ERR_CUDA, "tile record buffer overflow");
  float ms = 0.f, ms_peel = 0.f;
  cudaEventElapsedTime(&ms, c->ev_a, c->ev_m);
  cudaEventElapsedTime(&ms_peel, c->ev_m, c->ev_b);
  int status = RT_OK;
  for (int j = 0; j < n_jobs; ++j) {
    const LedgerDev& L = hl[j];
    if (ledgers) {
      rt_ledger& o = ledgers[j];
      o.emitted = L.emitted;
      o.absorbed = L.absorbed;
      o.escaped = L.escaped;
      o.rr_gain = L.rr_gain;
      o.rr_loss = L.rr_loss;
      o.killed = L.killed;
      o.peeled = L.peeled;
      o.n_packets = L.n_packets;
      o.n_cross = L.n_cross;
      o.n_scatter = L.n_scatter;
      o.n_peel_cross = L.n_peel_cross;
      o.n_killed = L.n_killed;
      o.n_peel_out = L.n_peel_out;
      o.n_peel_deferred = L.n_peel_deferred;
      o.status = L.status ? RT_ERR_STEP_LIMIT : RT_OK;
      o.kernel_ms = ms;
      o.peel_ms = q.cap > 0 ? ms_peel : 0.0;
      o.n_launches = n_launch;
      o.n_tiles = tiled ? tiles.n_tiles : 0;
      o.n_rounds = n_rounds;
      o.n_split = L.n_split;
      o.n_split_skipped = L.n_split_skipped;
    }
    if (L.status) status = RT_ERR_STEP_LIMIT;
  }
  if (status != RT_OK) return fail(status, "some packages were killed by the step limit");
  return RT_OK;
}

extern "C" int rt_trace(rt_ctx* ctx, const rt_grid* grid, int n_src, const rt_source* src, const rt_optics* optics,
                        const rt_trace_params* params, double* absorbed_dev, rt_ledger* ledger, void* cuda_stream) {
  if (!ctx || !grid || !params) return fail(RT_ERR_INVALID, "rt_trace: NULL argument");
  CTX_ENTER(ctx);
  DeviceGuard dg(ctx->device);
  TraceArgs T{grid, n_src, src, optics, params, nullptr, nullptr, absorbed_dev};
  if (ledger) memset(ledger, 0, sizeof *ledger);
  return run_jobs(ctx, 1, &T, ledger, (cudaStream_t)cuda_stream, params);
}

extern "C" int rt_peel(rt_ctx* ctx, const rt_grid* grid, int n_src, const rt_source* src, const rt_optics* optics,
                       const rt_trace_params* params, const rt_observers* obs, double* images_dev,
                       double* absorbed_dev, rt_ledger* ledger, void* cuda_stream) {
  if (!ctx || !grid || !params || !obs) return fail(RT_ERR_INVALID, "rt_peel: NULL argument");
  CTX_ENTER(ctx);
  DeviceGuard dg(ctx->device);
  TraceArgs T{grid, n_src, src, optics, params, obs, images_dev, absorbed_dev};
  if (ledger) memset(ledger, 0, sizeof *ledger);
  return run_jobs(ctx, 1, &T, ledger, (cudaStream_t)cuda_stream, params);
}

extern "C" int rt_peel_tables_create(rt_ctx* ctx, const rt_grid* grid, const rt_observers* obs, int block_edge,
                                     int tiles_per_edge, rt_peel_tables** out, void* cuda_stream) {
  if (!ctx || !grid || !obs || !out) return fail(RT_ERR_INVALID, "rt_peel_tables_create: NULL argument");
  *out = nullptr;
  auto pow2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
  if (!pow2(block_edge) || !pow2(tiles_per_edge) || tiles_per_edge > 4096)
    return fail(RT_ERR_INVALID, "rt_peel_tables_create: block_edge and tiles_per_edge must be powers of two");
  if (obs->n_obs < 1 || obs->n_obs > RT_MAX_OBS || !obs->dir)
    return fail(RT_ERR_INVALID, "rt_peel_tables_create: 1..%d observers", RT_MAX_OBS);
  CTX_ENTER(ctx);
  DeviceGuard dg(ctx->device);
  if (grid->device != ctx->device) return fail(RT_ERR_INVALID, "rt_peel_tables_create: grid on another device");
  rt_peel_tables* t = new rt_peel_tables();
  t->ctx = ctx;
  t->grid = grid;
  PeelTabSpec& S = t->spec;
  memset(&S, 0, sizeof S);
  S.n_obs = obs->n_obs;
  S.block = block_edge;
  S.tiles = tiles_per_edge;
  for (int a = 0; a < 3; ++a) S.nb[a] = (grid->root[a] + block_edge - 1) / block_edge;
  if (S.nb[0] > 1024 || S.nb[1] > 1024 || S.nb[2] > 1024) {
    delete t;
    return fail(RT_ERR_INVALID, "rt_peel_tables_create: at most 1024 blocks per axis");
  }
  while ((1 << t->bsh) < block_edge) ++t->bsh;
  while ((1 << t->ssh) < tiles_per_edge) ++t->ssh;
  const long long nblk = (long long)S.nb[0] * S.nb[1] * S.nb[2];
  t->dirs.assign(obs->dir, obs->dir + 3 * obs->n_obs);
  S.off[0] = 0;
  for (int o = 0; o < obs->n_obs; ++o) {
    if (!unit_dir(&obs->dir[3 * o], S.k[o])) {
      delete t;
      return fail(RT_ERR_INVALID, "rt_peel_tables_create: observer %d has a zero direction", o);
    }
    S.n_axes[o] = 0;
    for (int a = 0; a < 3; ++a)
      if (S.k[o][a] != 0.0) S.axes[o][S.n_axes[o]++] = a;
    S.off[o + 1] = S.off[o] + nblk * S.n_axes[o] * (long long)tiles_per_edge * tiles_per_edge;
  }
  t->n = S.off[obs->n_obs];
  if (t->n > (1ll << 32)) {
    delete t;
    return fail(RT_ERR_INVALID, "rt_peel_tables_create: %lld entries (more than 2^32)", (long long)S.off[obs->n_obs]);
  }
  JobDev J;
  memset(&J, 0, sizeof J);
  J.node = grid->node;
  J.rho64 = grid->rho64;
  for (int a = 0; a < 3; ++a) J.root[a] = (uint32_t)grid->root[a];
  int rc = t->buf.ensure(256 + sizeof(double) * (size_t)std::max<long long>(t->n, 1));
  if (rc) {
    delete t;
    return rc;
  }
  t->table = reinterpret_cast<const double*>(reinterpret_cast<char*>(t->buf.p) + 256);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  rc = ensure_pinned(ctx, sizeof J);
  if (!rc) {
    memcpy(ctx->pinned, &J, sizeof J);
    cudaError_t e = cudaMemcpyAsync(t->buf.p, ctx->pinned, sizeof J, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = build_peel_table(reinterpret_cast<const JobDev*>(t->buf.p), S, const_cast<double*>(t->table), s);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_c, s);
    if (e != cudaSuccess) rc = fail(RT_ERR_CUDA, "rt_peel_tables_create: %s", cudaGetErrorString(e));
  }
  if (!rc) rc = ctx_wait(ctx, ctx->ev_c, 3600.0);
  if (rc) {
    t->buf.release();
    delete t;
    return rc;
  }
  *out = t;
  return RT_OK;
}

extern "C" void rt_peel_tables_destroy(rt_peel_tables* t) {
  if (!t) return;
  DeviceGuard dg(t->ctx->device);
  t->buf.release();
  delete t;
}

extern "C" int64_t rt_peel_tables_size(const rt_peel_tables* t) { return t ? (int64_t)t->n : -1; }

extern "C" int rt_peel_tables_read(const rt_peel_tables* t, double* host, int64_t n) {
  if (!t || !host || n < t->n) return fail(RT_ERR_INVALID, "rt_peel_tables_read: NULL argument or short buffer");
  DeviceGuard dg(t->ctx->device);
  CK(cudaMemcpy(host, t->table, sizeof(double) * (size_t)t->n, cudaMemcpyDeviceToHost));
  return RT_OK;
}

extern "C" int rt_peel_tabulated(rt_ctx* ctx, const rt_grid* grid, int n_src, const rt_source* src,
                                 const rt_optics* optics, const rt_trace_params* params, const rt_observers* obs,
                                 const rt_peel_tables* tables, double* images_dev, double* absorbed_dev,
                                 rt_ledger* ledger, void* cuda_stream) {
  if (!ctx || !grid || !params || !obs || !tables) return fail(RT_ERR_INVALID, "rt_peel_tabulated: NULL argument");
  CTX_ENTER(ctx);
  DeviceGuard dg(ctx->device);
  TraceArgs T{grid, n_src, src, optics, params, obs, images_dev, absorbed_dev, tables};
  if (ledger) memset(ledger, 0, sizeof *ledger);
  return run_jobs(ctx, 1, &T, ledger, (cudaStream_t)cuda_stream, params);
}

// ------------------------------------------------------------------------
// dust
// ------------------------------------------------------------------------
extern "C" int rt_dust_temperature(rt_ctx* ctx, const rt_grid* g, const double* absorbed_dev, int n_bins,
                                   const rt_dust* dust, double* T_dev, void* cuda_stream) {
  if (!ctx || !g || !absorbed_dev || !T_dev || n_bins < 1) return fail(RT_ERR_INVALID, "rt_dust_temperature: bad argument");
  if (!dust) return fail(RT_ERR_INVALID, "rt_dust_temperature: dust is NULL");
  int rc = check_dust(dust, dust->n_lambda);
  if (rc) return rc;
  if (dust->n_lambda < 1 || dust->n_lambda > RT_MAX_LAMBDA) return fail(RT_ERR_INVALID, "dust: n_lambda out of range");
  CTX_ENTER(ctx);
  DeviceGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int n_table = 8192;
  double *lam, *kab, *dnu, *tab;
  rc = upload_dust(ctx, dust, n_table, &lam, &kab, &dnu, &tab, s);
  if (rc) return rc;
  CK(dust_table(lam, kab, dnu, dust->n_lambda, dust->T_min, dust->T_max, n_table, tab, s));
  CK(dust_temperature(absorbed_dev, n_bins, g->n_cells, g->child, g->rho64, g->level, g->h0, lam, kab, dnu,
                      dust->n_lambda, dust->T_min, dust->T_max, tab, n_table, T_dev, s));
  CK(cudaEventRecord(ctx->ev_b, s));
  return ctx_wait(ctx, ctx->ev_b, 3600.0);
}

extern "C" int rt_dust_emission(rt_ctx* ctx, const rt_grid* g, const double* T_dev, const rt_dust* dust,
                                double* emission_dev, double* bin_total_host, void* cuda_stream) {
  if (!ctx || !g || !T_dev || !emission_dev || !dust) return fail(RT_ERR_INVALID, "rt_dust_emission: bad argument");
  int rc = check_dust(dust, dust->n_lambda);
  if (rc) return rc;
  if (dust->n_lambda < 1 || dust->n_lambda > RT_MAX_LAMBDA) return fail(RT_ERR_INVALID, "dust: n_lambda out of range");
  CTX_ENTER(ctx);
  DeviceGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  double *lam, *kab, *dnu, *tab;
  rc = upload_dust(ctx, dust, 0, &lam, &kab, &dnu, &tab, s);
  if (rc) return rc;
  CK(dust_emission(T_dev, g->n_cells, g->child, g->rho64, g->level, g->h0, lam, kab, dnu, dust->n_lambda, emission_dev, s));
  const size_t tb = sizeof(double) * (size_t)dust->n_lambda;
  if (bin_total_host) {
    rc = ctx->small.ensure(tb + 256);
    if (!rc) rc = ensure_pin_rb(ctx, tb);
    if (rc) return rc;
    double* tot = reinterpret_cast<double*>(ctx->small.p);
    CK(row_sums_f64(emission_dev, dust->n_lambda, g->n_cells, tot, s));
    CK(cudaMemcpyAsync(ctx->pin_rb, tot, tb, cudaMemcpyDeviceToHost, s));
  }
  CK(cudaEventRecord(ctx->ev_b, s));
  rc = ctx_wait(ctx, ctx->ev_b, 3600.0);
  if (rc) return rc;
  if (bin_total_host) memcpy(bin_total_host, ctx->pin_rb, tb);
  return RT_OK;
}

// ------------------------------------------------------------------------
// diagnostics
// ------------------------------------------------------------------------
extern "C" int rt_walk(rt_ctx* ctx, const rt_grid* g, int64_t n_rays, const double* origins_dev, const double* dirs_dev,
                       int precision, int64_t max_seg, int64_t* cells_dev, double* lengths_dev, int64_t* counts_dev,
                       void* cuda_stream) {
  if (!ctx || !g || n_rays < 0 || max_seg < 0 || (n_rays > 0 && (!origins_dev || !dirs_dev || !counts_dev)) ||
      (max_seg > 0 && (!cells_dev || !lengths_dev)))
    return fail(RT_ERR_INVALID, "rt_walk: bad argument");
  if (precision != 32 && precision != 64) return fail(RT_ERR_INVALID, "rt_walk: precision must be 32 or 64");
  CTX_ENTER(ctx);
  DeviceGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  JobDev J;
  memset(&J, 0, sizeof J);
  J.node = g->node;
  J.rho64 = g->rho64;
  J.coord = g->coord;
  J.level = g->level;
  for (int a = 0; a < 3; ++a) J.root[a] = (uint32_t)g->root[a];
  J.depth = g->n_levels - 1;
  J.h0 = g->h0;
  J.n_cells = g->n_cells;
  int rc = ctx->table.ensure(sizeof J);
  if (rc) return rc;
  rc = ensure_pinned(ctx, sizeof J);
  if (rc) return rc;
  memcpy(ctx->pinned, &J, sizeof J);
  CK(cudaMemcpyAsync(ctx->table.p, ctx->pinned, sizeof J, cudaMemcpyHostToDevice, s));
  CK(launch_walk(precision, reinterpret_cast<const JobDev*>(ctx->table.p), n_rays, origins_dev, dirs_dev, max_seg,
                 reinterpret_cast<long long*>(cells_dev), lengths_dev, reinterpret_cast<long long*>(counts_dev), s));
  CK(cudaEventRecord(ctx->ev_b, s));
  return ctx_wait(ctx, ctx->ev_b, 3600.0);
}

extern "C" int rt_descent_counts(rt_ctx* ctx, uint64_t* counts, int reset) {
  if (!ctx || !counts) return fail(RT_ERR_INVALID, "rt_descent_counts: NULL argument");
  if (!descents_counted())
    return fail(RT_ERR_INVALID, "rt_descent_counts: this build does not count descents (RT_COUNT_DESCENTS=1)");
  CTX_ENTER(ctx);
  DeviceGuard dg(ctx->device);
  unsigned long long v[2] = {0ull, 0ull};
  CK(cudaDeviceSynchronize());
  CK(descent_counts(v, reset != 0));
  counts[0] = v[0];
  counts[1] = v[1];
  return RT_OK;
}

extern "C" int rt_l2_read_bandwidth(rt_ctx* ctx, void* buf_dev, int64_t bytes, int reps, double* gbs,
                                    void* cuda_stream) {
  if (!ctx || !buf_dev || !gbs || bytes < 16 || reps < 1 || ((uintptr_t)buf_dev & 15))
    return fail(RT_ERR_INVALID, "rt_l2_read_bandwidth: bad argument");
  CTX_ENTER(ctx);
  DeviceGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  CK(launch_l2_read(buf_dev, bytes, reps, ctx->sm_count, s));  // warm-up: fills L2
  double best = 0.0;
  for (int k = 0; k < 5; ++k) {
    CK(cudaEventRecord(ctx->ev_a, s));
    CK(launch_l2_read(buf_dev, bytes, reps, ctx->sm_count, s));
    CK(cudaEventRecord(ctx->ev_b, s));
    const int rc = ctx_wait(ctx, ctx->ev_b, 60.0);
    if (rc) return rc;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev_a, ctx->ev_b);
    if (ms > 0.f) best = std::max(best, (double)(bytes / 16 * 16) * reps / (ms * 1e-3) / 1e9);
  }
  *gbs = best;
  return RT_OK;
}

extern "C" int rt_philox(rt_ctx* ctx, int64_t n, const uint32_t* ctr_dev, const uint32_t* key_dev, uint32_t* out_dev,
                         void* cuda_stream) {
  if (!ctx || n < 0 || (n > 0 && (!ctr_dev || !key_dev || !out_dev))) return fail(RT_ERR_INVALID, "rt_philox: bad argument");
  CTX_ENTER(ctx);
  DeviceGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  CK(launch_philox(n, ctr_dev, key_dev, out_dev, s));
  CK(cudaEventRecord(ctx->ev_b, s));
  return ctx_wait(ctx, ctx->ev_b, 3600.0);
}

// ------------------------------------------------------------------------
// Lambda iteration (Eq. 2, Sect. 3.2)
// ------------------------------------------------------------------------
extern "C" int rt_lambda_iterate(rt_ctx* ctx, const rt_grid* g, int n_src, const rt_source* src, const rt_optics* op,
                                 const rt_dust* du_in, const rt_trace_params* prm, const rt_lambda_params* lp,
                                 double* T_dev, rt_lambda_result* res, void* cuda_stream) {
  std::vector<double> kabs_store;
  rt_dust du_res;
  const rt_dust* du = resolve_dust(du_in, op, kabs_store, du_res);
  if (!ctx || !g || !src || !op || !du || !prm || !lp || !T_dev || !res)
    return fail(RT_ERR_INVALID, "rt_lambda_iterate: NULL argument");
  if (lp->max_iter < 1 || lp->max_iter > 64) return fail(RT_ERR_INVALID, "rt_lambda_iterate: max_iter must be 1..64");
  if (lp->dust_packets_per_bin <= 0 && lp->dust_packets_total <= 0)
    return fail(RT_ERR_INVALID, "rt_lambda_iterate: set dust_packets_total or dust_packets_per_bin");
  int rc = check_optics(op);
  if (rc) return rc;
  rc = check_dust(du, op->n_lambda);
  if (rc) return rc;
  memset(res, 0, sizeof *res);
  CTX_ENTER(ctx);
  DeviceGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const auto t0 = std::chrono::steady_clock::now();
  const long long nc = g->n_cells;
  const size_t fb = sizeof(double) * (size_t)nc;
  rc = ctx->lam.ensure(3 * fb + sizeof(unsigned int) * (size_t)nc + 1024);
  if (rc) return rc;
  char* base = reinterpret_cast<char*>(ctx->lam.p);
  double* A_star = reinterpret_cast<double*>(base);
  double* A = reinterpret_cast<double*>(base + fb);
  double* T_prev = reinterpret_cast<double*>(base + 2 * fb);
  unsigned int* hits = reinterpret_cast<unsigned int*>(base + 3 * fb);
  double* scal = reinterpret_cast<double*>(base + 3 * fb + ((sizeof(unsigned int) * (size_t)nc + 255) / 256) * 256);
  CK(cudaMemsetAsync(A_star, 0, fb, s));
  CK(cudaMemsetAsync(hits, 0, sizeof(unsigned int) * (size_t)nc, s));
  const double to = prm->timeout_s > 0 ? prm->timeout_s : 3600.0;

  // constant sources, traced once and stored (Sect. 3.2)
  rt_trace_params sp = *prm;
  sp.per_lambda = 0;
  sp.hits_dev = hits;
  sp.packet_log_dev = nullptr;
  TraceArgs TS{g, n_src, src, op, &sp, nullptr, nullptr, A_star};
  rc = run_jobs(ctx, 1, &TS, &res->source_ledger, s, &sp);
  if (rc && rc != RT_ERR_STEP_LIMIT) return rc;

  const int n_table = 8192;
  auto solve = [&](const double* absorbed) -> int {
    double *lam, *kab, *dnu, *tab;
    int r = upload_dust(ctx, du, n_table, &lam, &kab, &dnu, &tab, s);
    if (r) return r;
    CK(dust_table(lam, kab, dnu, du->n_lambda, du->T_min, du->T_max, n_table, tab, s));
    CK(dust_temperature(absorbed, 1, nc, g->child, g->rho64, g->level, g->h0, lam, kab, dnu, du->n_lambda, du->T_min,
                        du->T_max, tab, n_table, T_dev, s));
    return RT_OK;
  };
  rc = solve(A_star);
  if (rc) return rc;

  // dust re-emission: same streams every iteration (key iter = params.iter + 1)
  rt_source ds;
  memset(&ds, 0, sizeof ds);
  ds.kind = RT_SRC_DUST;
  ds.T_dev = T_prev;
  ds.dust = du;
  rt_trace_params dp = *prm;
  dp.per_lambda = 0;
  dp.iter = prm->iter + 1;
  dp.packets = nullptr;
  dp.packet_log_dev = nullptr;
  dp.packets_per_bin = lp->dust_packets_per_bin > 0 ? lp->dust_packets_per_bin : 0;
  dp.packets_total = lp->dust_packets_per_bin > 0 ? 0 : lp->dust_packets_total;
  for (int it = 1; it <= lp->max_iter; ++it) {
    CK(cudaMemcpyAsync(T_prev, T_dev, fb, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(A, A_star, fb, cudaMemcpyDeviceToDevice, s));
    dp.hits_dev = it == 1 ? hits : nullptr;
    TraceArgs TD{g, 1, &ds, op, &dp, nullptr, nullptr, A};
    rc = run_jobs(ctx, 1, &TD, &res->dust_ledger, s, &dp);
    if (rc && rc != RT_ERR_STEP_LIMIT) return rc;
    rc = solve(A);
    if (rc) return rc;
    CK(max_rel_change(T_dev, T_prev, hits, g->child, nc, lp->min_hits, scal, s));
    CK(cudaMemcpyAsync(ctx->pin_count, scal, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(ctx->ev_c, s));
    rc = ctx_wait(ctx, ctx->ev_c, to);
    if (rc) return rc;
    double v = 0.0;
    memcpy(&v, ctx->pin_count, sizeof v);
    res->history[it - 1] = v;
    res->n_iter = it;
    if (v < lp->tol) break;
  }
  res->ms = 1e3 * std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return RT_OK;
}

// ------------------------------------------------------------------------
// Lambda iteration with subiterations (Sect. 3.2, App. B)
// ------------------------------------------------------------------------
extern "C" int rt_lambda_subiterate(rt_ctx* ctx, const rt_grid* g, int n_src, const rt_source* src,
                                    const rt_optics* op, const rt_dust* du_in, const rt_trace_params* prm,
                                    const rt_lambda_params* lp, const rt_subiter_params* sp, double* T_dev,
                                    rt_subiter_result* res, void* cuda_stream) {
  std::vector<double> kabs_store;
  rt_dust du_res;
  const rt_dust* du = resolve_dust(du_in, op, kabs_store, du_res);
  if (!ctx || !g || !src || !op || !du || !prm || !lp || !sp || !T_dev || !res)
    return fail(RT_ERR_INVALID, "rt_lambda_subiterate: NULL argument");
  const int n_steps = sp->n_steps > 0 ? sp->n_steps : lp->max_iter;
  if (n_steps < 1 || n_steps > 64) return fail(RT_ERR_INVALID, "rt_lambda_subiterate: 1..64 steps");
  if (sp->n_steps > 0 && !sp->schedule) return fail(RT_ERR_INVALID, "rt_lambda_subiterate: schedule is NULL");
  if (sp->sub_level < 0 || sp->sub_level >= g->n_levels - 1)
    return fail(RT_ERR_INVALID, "rt_lambda_subiterate: sub_level must be 0..%d", g->n_levels - 2);
  if (lp->dust_packets_per_bin <= 0 && lp->dust_packets_total <= 0)
    return fail(RT_ERR_INVALID, "rt_lambda_subiterate: set dust_packets_total or dust_packets_per_bin");
  int rc = check_optics(op);
  if (rc) return rc;
  rc = check_dust(du, op->n_lambda);
  if (rc) return rc;
  memset(res, 0, sizeof *res);
  CTX_ENTER(ctx);
  DeviceGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const auto t0 = std::chrono::steady_clock::now();
  const long long nc = g->n_cells;
  const int nlev = g->n_levels, L = sp->sub_level;
  const size_t fb = sizeof(double) * (size_t)nc, hb = sizeof(unsigned int) * (size_t)nc;
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  // A_star, A, T_prev, T_emit | I (levels) | I_step (levels) | hits_star, hits_step | scalars
  // (scal[0] max dT/T, scal[1..6] level_imbalance sums) | ALI: self, emitted, weights (bins x
  // cells each), right-hand side, package count, use flag
  const int nlb = op->n_lambda;
  const size_t ali_bytes = sp->ali ? 3 * al(fb * nlb) + al(fb) + al(hb) + al((size_t)nc) : 0;
  const size_t scal_bytes = al(sizeof(double) * (16 + RT_MAX_LAMBDA));  // + per-bin emission totals at scal + 16
  rc = ctx->lam.ensure(4 * al(fb) + 2 * al(fb * nlev) + 2 * al(hb) + scal_bytes + ali_bytes);
  if (rc) return rc;
  char* base = reinterpret_cast<char*>(ctx->lam.p);
  double* A_star = reinterpret_cast<double*>(base);
  double* A = reinterpret_cast<double*>(base + al(fb));
  double* T_prev = reinterpret_cast<double*>(base + 2 * al(fb));
  double* T_emit = reinterpret_cast<double*>(base + 3 * al(fb));
  double* I = reinterpret_cast<double*>(base + 4 * al(fb));
  double* I_step = reinterpret_cast<double*>(base + 4 * al(fb) + al(fb * nlev));
  unsigned int* hits_star = reinterpret_cast<unsigned int*>(base + 4 * al(fb) + 2 * al(fb * nlev));
  unsigned int* hits_step = reinterpret_cast<unsigned int*>(base + 4 * al(fb) + 2 * al(fb * nlev) + al(hb));
  double* scal = reinterpret_cast<double*>(base + 4 * al(fb) + 2 * al(fb * nlev) + 2 * al(hb));
  char* ali_base = base + 4 * al(fb) + 2 * al(fb * nlev) + 2 * al(hb) + scal_bytes;
  double* self_abs = reinterpret_cast<double*>(ali_base);
  double* self_emit = reinterpret_cast<double*>(ali_base + al(fb * nlb));
  double* ali_w = reinterpret_cast<double*>(ali_base + 2 * al(fb * nlb));
  double* ali_rhs = reinterpret_cast<double*>(ali_base + 3 * al(fb * nlb));
  unsigned int* self_cnt = reinterpret_cast<unsigned int*>(ali_base + 3 * al(fb * nlb) + al(fb));
  uint8_t* ali_use = reinterpret_cast<uint8_t*>(ali_base + 3 * al(fb * nlb) + al(fb) + al(hb));
  CK(cudaMemsetAsync(A_star, 0, fb, s));
  CK(cudaMemsetAsync(hits_star, 0, hb, s));
  CK(cudaMemsetAsync(I, 0, fb * nlev, s));
  const double to = prm->timeout_s > 0 ? prm->timeout_s : 3600.0;

  // constant sources, traced once and stored (Sect. 3.2)
  rt_trace_params stp = *prm;
  stp.per_lambda = 0;
  stp.hits_dev = hits_star;
  stp.packet_log_dev = nullptr;
  TraceArgs TS{g, n_src, src, op, &stp, nullptr, nullptr, A_star};
  rc = run_jobs(ctx, 1, &TS, &res->lambda.source_ledger, s, &stp);
  if (rc && rc != RT_ERR_STEP_LIMIT) return rc;
  CK(cudaMemcpyAsync(A, A_star, fb, cudaMemcpyDeviceToDevice, s));

  const int n_table = 8192;
  double *lam, *kab, *dnu, *tab;
  auto upload = [&]() -> int {
    int r = upload_dust(ctx, du, n_table, &lam, &kab, &dnu, &tab, s);
    if (r) return r;
    CK(dust_table(lam, kab, dnu, du->n_lambda, du->T_min, du->T_max, n_table, tab, s));
    return RT_OK;
  };
  auto solve = [&](const double* absorbed) -> int {
    int r = upload();
    if (r) return r;
    CK(dust_temperature(absorbed, 1, nc, g->child, g->rho64, g->level, g->h0, lam, kab, dnu, du->n_lambda, du->T_min,
                        du->T_max, tab, n_table, T_dev, s));
    return RT_OK;
  };
  auto read_scalars = [&](double* out, int n) -> int {
    CK(cudaMemcpyAsync(ctx->pin_count, scal, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(ctx->ev_c, s));
    int r = ctx_wait(ctx, ctx->ev_c, to);
    if (r) return r;
    memcpy(out, ctx->pin_count, sizeof(double) * n);
    return RT_OK;
  };
  rc = solve(A_star);
  if (rc) return rc;

  rt_source ds;
  memset(&ds, 0, sizeof ds);
  ds.kind = RT_SRC_DUST;
  ds.T_dev = T_emit;
  ds.dust = du;
  rt_trace_params dp = *prm;
  dp.per_lambda = 0;
  dp.iter = prm->iter + 1;  // the same streams every step
  dp.packets = nullptr;
  dp.packet_log_dev = nullptr;
  dp.hits_dev = hits_step;
  dp.packets_per_bin = lp->dust_packets_per_bin > 0 ? lp->dust_packets_per_bin : 0;
  dp.packets_total = lp->dust_packets_per_bin > 0 ? 0 : lp->dust_packets_total;
  double imb_low = 0.0, imb_deep = 0.0;  // mass-weighted mean imbalance at levels <= L and > L
  double e_ref = -1.0;                   // emission below L after the last full step
  int last_kind = 0;
  for (int it = 1; it <= n_steps; ++it) {
    const auto ts = std::chrono::steady_clock::now();
    // emission at levels <= L and below L with the current temperatures
    double e[7] = {0, 0, 0, 0, 0, 0, 0};
    if (it > 1) {
      rc = upload();
      if (rc) return rc;
      CK(level_imbalance(A, T_dev, g->child, g->rho64, g->level, g->h0, tab, n_table, nc, L, scal + 1, s));
      rc = read_scalars(e, 7);
      if (rc) return rc;
      if (last_kind == 0) e_ref = e[6];
    }
    int kind;
    if (sp->n_steps > 0) {
      kind = sp->schedule[it - 1] ? 1 : 0;
    } else if (it == 1) {
      kind = 0;
    } else {
      // Sect. 3.3: iterate the upper levels when their imbalance is a
      // sizeable fraction of the largest, or when the radiation they receive
      // from below (tracked by the emission below L) has changed
      // appreciably since they were last included
      const bool tagged = sp->flux_frac > 0 && e_ref > 0 && std::fabs(e[6] - e_ref) >= sp->flux_frac * e_ref;
      kind = tagged || imb_low >= sp->select_frac * std::max(imb_low, imb_deep) ? 0 : 1;
    }
    last_kind = kind;
    CK(cudaMemcpyAsync(T_prev, T_dev, fb, cudaMemcpyDeviceToDevice, s));
    if (kind == 1) CK(mask_levels(T_dev, g->level, nc, L, T_emit, s));
    else CK(cudaMemcpyAsync(T_emit, T_dev, fb, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(hits_step, hits_star, hb, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(I_step, 0, fb * nlev, s));
    // a subiteration sends from each cell the packages a full step would
    // (App. B): the package energy of the full step's emission, so every
    // cell of the subtrees sends the packages, with the streams, it would
    // send in a full step
    std::vector<double> w_full;
    if (kind == 1) {
      rc = upload();
      if (rc) return rc;
      CK(dust_emission_totals(T_dev, nc, g->child, g->rho64, g->level, g->h0, lam, kab, dnu, nlb, scal + 16, s));
      rc = ensure_pin_rb(ctx, sizeof(double) * (size_t)nlb);
      if (rc) return rc;
      CK(cudaMemcpyAsync(ctx->pin_rb, scal + 16, sizeof(double) * (size_t)nlb, cudaMemcpyDeviceToHost, s));
      CK(cudaEventRecord(ctx->ev_c, s));
      rc = ctx_wait(ctx, ctx->ev_c, to);
      if (rc) return rc;
      std::vector<double> ef(static_cast<const double*>(ctx->pin_rb), static_cast<const double*>(ctx->pin_rb) + nlb);
      std::vector<long long> nf(nlb);
      if (lp->dust_packets_per_bin > 0) {
        for (int b = 0; b < nlb; ++b) nf[b] = ef[b] > 0 ? lp->dust_packets_per_bin : 0;
      } else {
        packages_by_energy(ef.data(), nlb, lp->dust_packets_total, nf.data());
      }
      w_full.assign(nlb, 0.0);
      for (int b = 0; b < nlb; ++b) w_full[b] = nf[b] > 0 ? ef[b] / (double)nf[b] : 0.0;
    }
    TraceArgs TD{g, 1, &ds, op, &dp, nullptr, nullptr, I_step};
    TD.dust_package_energy = kind == 1 ? w_full.data() : nullptr;
    TD.levels = 1;
    TD.confine = kind == 1 ? L : -1;
    if (sp->ali) {
      CK(cudaMemsetAsync(self_abs, 0, fb * nlb, s));
      CK(cudaMemsetAsync(self_emit, 0, fb * nlb, s));
      CK(cudaMemsetAsync(self_cnt, 0, hb, s));
      TD.self_abs = self_abs;
      TD.self_emit = self_emit;
      TD.self_cnt = self_cnt;
    }
    rc = run_jobs(ctx, 1, &TD, &res->lambda.dust_ledger, s, &dp);
    if (rc && rc != RT_ERR_STEP_LIMIT) return rc;
    // a full step replaces every level array, a subiteration those below L
    const int first = kind == 1 ? L + 1 : 0;
    CK(cudaMemcpyAsync(I + (size_t)first * nc, I_step + (size_t)first * nc, fb * (size_t)(nlev - first),
                       cudaMemcpyDeviceToDevice, s));
    CK(sum_levels(I, nlev, nc, A_star, A, s));
    // imbalance of the new field against the emission that produced it
    rc = upload();
    if (rc) return rc;
    CK(level_imbalance(A, T_prev, g->child, g->rho64, g->level, g->h0, tab, n_table, nc, L, scal + 1, s));
    rc = solve(A);
    if (!rc && sp->ali) {
      // Eq. 3 per frequency: the cells' own re-absorption solved with the
      // new temperature, from the plain solve's T
      const double lam_max = sp->ali_max_lambda > 0.0 && sp->ali_max_lambda < 1.0 ? sp->ali_max_lambda : 0.999;
      CK(ali_weights(A, self_abs, self_emit, self_cnt, kab, (unsigned)std::max(1, sp->ali_min_packages), lam_max,
                     nlb, nc, ali_rhs, ali_w, ali_use, s));
      CK(dust_temperature_weighted(ali_rhs, ali_w, ali_use, nc, g->child, g->rho64, g->level, g->h0, lam, kab, dnu,
                                   du->n_lambda, du->T_min, du->T_max, T_dev, s));
    }
    if (rc) return rc;
    CK(max_rel_change(T_dev, T_prev, hits_step, g->child, nc, lp->min_hits, scal, s));
    double v[7];
    rc = read_scalars(v, 7);
    if (rc) return rc;
    if (kind == 0) imb_low = v[2] > 0 ? v[1] / v[2] : 0.0;
    imb_deep = v[4] > 0 ? v[3] / v[4] : 0.0;
    res->lambda.history[it - 1] = v[0];
    res->lambda.n_iter = it;
    res->step_kind[it - 1] = kind;
    res->imbalance[it - 1][0] = imb_low;
    res->imbalance[it - 1][1] = imb_deep;
    res->step_ms[it - 1] = 1e3 * std::chrono::duration<double>(std::chrono::steady_clock::now() - ts).count();
    if (v[0] < lp->tol) break;
  }
  res->lambda.ms = 1e3 * std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return RT_OK;
}

// ------------------------------------------------------------------------
// batches: many models in one persistent launch
// ------------------------------------------------------------------------
static int jobs_to_args(int n_jobs, const rt_job* jobs, std::vector<TraceArgs>& out) {
  if (n_jobs < 1 || !jobs) return fail(RT_ERR_INVALID, "batch: need at least one job");
  out.resize(n_jobs);
  for (int j = 0; j < n_jobs; ++j) {
    const rt_job& J = jobs[j];
    if (!J.grid || !J.params) return fail(RT_ERR_INVALID, "batch job %d: NULL grid or params", j);
    out[j] = TraceArgs{J.grid, J.n_src, J.src, J.optics, J.params, J.obs, J.images_dev, J.absorbed_dev};
  }
  return RT_OK;
}

extern "C" int rt_trace_batch(rt_ctx* ctx, int n_jobs, const rt_job* jobs, rt_ledger* ledgers, void* cuda_stream) {
  if (!ctx) return fail(RT_ERR_INVALID, "rt_trace_batch: NULL context");
  std::vector<TraceArgs> args;
  int rc = jobs_to_args(n_jobs, jobs, args);
  if (rc) return rc;
  CTX_ENTER(ctx);
  DeviceGuard dg(ctx->device);
  if (ledgers) memset(ledgers, 0, sizeof(rt_ledger) * n_jobs);
  return run_jobs(ctx, n_jobs, args.data(), ledgers, (cudaStream_t)cuda_stream, jobs[0].params);
}

struct rt_batch {
  rt_ctx* ctx = nullptr;
  int n_jobs = 0;
  DevBuf table, small, peel_q;
  std::vector<DevBuf> cdf;
  LedgerDev* host_led = nullptr;  // pinned, written by the graph
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  long long launches = 0;  // kernels per replay (tracer, peel-off)
};

extern "C" void rt_batch_destroy(rt_batch* b) {
  if (!b) return;
  DeviceGuard dg(b->ctx->device);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  if (b->host_led) cudaFreeHost(b->host_led);
  b->table.release();
  b->small.release();
  b->peel_q.release();
  for (auto& d : b->cdf) d.release();
  delete b;
}

extern "C" int rt_batch_create(rt_ctx* ctx, int n_jobs, const rt_job* jobs, rt_batch** out) {
  if (!ctx || !out) return fail(RT_ERR_INVALID, "rt_batch_create: NULL argument");
  *out = nullptr;
  std::vector<TraceArgs> args;
  int rc = jobs_to_args(n_jobs, jobs, args);
  if (rc) return rc;
  CTX_ENTER(ctx);
  DeviceGuard dg(ctx->device);
  rt_batch* b = new rt_batch();
  b->ctx = ctx;
  b->n_jobs = n_jobs;
  auto bail = [&](int code) -> int {
    rt_batch_destroy(b);
    return code;
  };
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev1);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->host_led, sizeof(LedgerDev) * n_jobs);
  if (e != cudaSuccess) return bail(fail(RT_ERR_CUDA, "rt_batch_create: %s", cudaGetErrorString(e)));
  rc = b->small.ensure(sizeof(LedgerDev) * n_jobs + 256);
  if (rc) return bail(rc);
  LedgerDev* led = reinterpret_cast<LedgerDev*>(b->small.p);
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(led + n_jobs);
  Arena A;
  std::vector<size_t> job_off;
  size_t items_off = 0;
  int n_items = 0, precision = 32, estimator = RT_EST_CONTINUOUS;
  long long total = 0;
  bool peel = false;
  rc = build_tables(ctx, n_jobs, args.data(), led, b->cap, A, job_off, items_off, n_items, total, peel, precision,
                    estimator, &b->table, &b->cdf);
  if (rc) return bail(rc);
  for (int j = 0; j < n_jobs; ++j)
    if (args[j].prm->hits_dev || args[j].prm->split_factor > 1 || args[j].prm->poly_group > 1)
      return bail(fail(RT_ERR_INVALID, "rt_batch_create: hit counting, resampling and polychromatic packages are "
                                       "not batched"));
  e = cudaStreamSynchronize(b->cap);
  if (e != cudaSuccess) return bail(fail(RT_ERR_CUDA, "rt_batch_create: %s", cudaGetErrorString(e)));
  LaunchCfg cfg;
  rc = make_cfg(ctx, precision, peel, jobs[0].params, path_levels(n_jobs, args.data()), &cfg);
  if (rc) return bail(rc);
  const PeelQueue q = make_queue(b->peel_q, ctx->peel_q_max, peel, n_jobs, total, precision, counter + 1);
  // capture: zero every job's outputs and the ledgers, run the tracer and
  // the deferred peel-off, read back
  char* base = reinterpret_cast<char*>(b->table.p);
  e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  for (int j = 0; j < n_jobs && e == cudaSuccess; ++j) {
    const TraceArgs& T = args[j];
    const int bins = T.prm->per_lambda ? T.optics->n_lambda : 1;
    if (T.absorbed) e = cudaMemsetAsync(T.absorbed, 0, sizeof(double) * (size_t)bins * T.grid->n_cells, b->cap);
    if (e == cudaSuccess && T.obs && T.images)
      e = cudaMemsetAsync(T.images, 0, sizeof(double) * (size_t)T.obs->n_obs * bins * T.obs->nx * T.obs->ny, b->cap);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(led, 0, sizeof(LedgerDev) * n_jobs + 3 * sizeof(unsigned long long), b->cap);
  if (e == cudaSuccess && total > 0 && n_items > 0)
    e = launch_trace(precision, peel, estimator, false, reinterpret_cast<const JobDev*>(base + job_off[0]),
                     reinterpret_cast<const ItemDev*>(base + items_off), n_items, counter, total, cfg, q, b->cap);
  if (e == cudaSuccess && total > 0 && n_items > 0 && q.cap > 0)
    e = launch_peel(precision, reinterpret_cast<const JobDev*>(base + job_off[0]), q, counter + 2,
                    max_observers(n_jobs, args.data()), cfg.refill, b->cap, cfg.anc);
  b->launches = (total > 0 && n_items > 0) ? 1 + (q.cap > 0 ? 1 : 0) : 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->host_led, led, sizeof(LedgerDev) * n_jobs, cudaMemcpyDeviceToHost, b->cap);
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
  b->graph = g;
  if (e != cudaSuccess || e2 != cudaSuccess)
    return bail(fail(RT_ERR_CUDA, "rt_batch_create: capture failed: %s",
                     cudaGetErrorString(e != cudaSuccess ? e : e2)));
  e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) return bail(fail(RT_ERR_CUDA, "rt_batch_create: instantiate: %s", cudaGetErrorString(e)));
  *out = b;
  return RT_OK;
}

extern "C" int rt_batch_run(rt_batch* b, rt_ledger* ledgers, double timeout_s, void* cuda_stream) {
  if (!b) return fail(RT_ERR_INVALID, "rt_batch_run: NULL batch");
  CTX_ENTER(b->ctx);
  DeviceGuard dg(b->ctx->device);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  CK(cudaEventRecord(b->ev0, s));
  CK(cudaGraphLaunch(b->exec, s));
  CK(cudaEventRecord(b->ev1, s));
  int rc = ctx_wait(b->ctx, b->ev1, timeout_s > 0 ? timeout_s : 3600.0);
  if (rc) return rc;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, b->ev0, b->ev1);
  int status = RT_OK;
  for (int j = 0; j < b->n_jobs; ++j) {
    const LedgerDev& L = b->host_led[j];
    if (ledgers) {
      rt_ledger& o = ledgers[j];
      o.emitted = L.emitted; o.absorbed = L.absorbed; o.escaped = L.escaped; o.rr_gain = L.rr_gain;
      o.rr_loss = L.rr_loss; o.killed = L.killed; o.peeled = L.peeled; o.n_packets = L.n_packets;
      o.n_cross = L.n_cross; o.n_scatter = L.n_scatter; o.n_peel_cross = L.n_peel_cross; o.n_killed = L.n_killed;
      o.n_peel_out = L.n_peel_out; o.n_peel_deferred = L.n_peel_deferred;
      o.status = L.status ? RT_ERR_STEP_LIMIT : RT_OK; o.kernel_ms = ms; o.peel_ms = 0.0;
      o.n_launches = b->launches; o.n_tiles = 0; o.n_rounds = 0;
    }
    if (L.status) status = RT_ERR_STEP_LIMIT;
  }
  if (status != RT_OK) return fail(status, "rt_batch_run: some packages hit the step limit");
  return RT_OK;
}

// ------------------------------------------------------------------------
// autotuner: block size and refill threshold from short trial launches
// ------------------------------------------------------------------------
extern "C" int rt_autotune(rt_ctx* ctx, int n_jobs, const rt_job* jobs, double sample_fraction, rt_tune_result* best) {
  if (!ctx || !best) return fail(RT_ERR_INVALID, "rt_autotune: NULL argument");
  if (!(sample_fraction > 0.0 && sample_fraction <= 1.0)) return fail(RT_ERR_INVALID, "rt_autotune: fraction in (0,1]");
  std::vector<TraceArgs> args;
  int rc = jobs_to_args(n_jobs, jobs, args);
  if (rc) return rc;
  CTX_ENTER(ctx);
  DeviceGuard dg(ctx->device);
  // trial copies of the jobs with scaled package counts and private outputs
  std::vector<rt_trace_params> prm(n_jobs);
  std::vector<std::vector<int64_t>> pk(n_jobs);
  bool peel = false;
  for (int j = 0; j < n_jobs; ++j) {
    prm[j] = *args[j].prm;
    prm[j].packet_log_dev = nullptr;
    prm[j].hits_dev = nullptr;
    if (prm[j].packets_per_bin > 0) prm[j].packets_per_bin = std::max<int64_t>(1, (int64_t)(prm[j].packets_per_bin * sample_fraction));
    else if (prm[j].packets_total > 0) prm[j].packets_total = std::max<int64_t>(1, (int64_t)(prm[j].packets_total * sample_fraction));
    else if (prm[j].packets) {
      const int nl = args[j].optics ? args[j].optics->n_lambda : 0;
      pk[j].resize((size_t)args[j].n_src * nl);
      for (size_t i = 0; i < pk[j].size(); ++i) pk[j][i] = (int64_t)(prm[j].packets[i] * sample_fraction);
      prm[j].packets = pk[j].data();
    }
    args[j].prm = &prm[j];
    peel = peel || args[j].obs != nullptr;
  }
  const int precision = prm[0].precision;
  const int blocks[2] = {128, 256};
  const int refills[5] = {2, 4, 8, 12, 16};
  rt_tune_result res;
  res.crossings_per_ms = -1.0;
  res.block_size = 256;
  res.refill_threshold = 8;
  res.blocks_per_sm = 0;
  std::vector<rt_ledger> led(n_jobs);
  for (int bi = 0; bi < 2; ++bi)
    for (int ri = 0; ri < 5; ++ri) {
      for (int j = 0; j < n_jobs; ++j) {
        prm[j].block_size = blocks[bi];
        prm[j].refill_threshold = refills[ri];
        prm[j].blocks_per_sm = 0;
      }
      // outputs are accumulated into the real buffers: zero them after tuning
      rc = run_jobs(ctx, n_jobs, args.data(), led.data(), nullptr, &prm[0]);
      if (rc && rc != RT_ERR_STEP_LIMIT) return rc;
      double cross = 0.0;
      for (auto& L : led) cross += (double)L.n_cross + (double)L.n_peel_cross;
      const double ms = led[0].kernel_ms + led[0].peel_ms;  // tracer + deferred peel-off
      const double rate = ms > 0 ? cross / ms : 0.0;
      if (rate > res.crossings_per_ms) {
        res.crossings_per_ms = rate;
        res.block_size = blocks[bi];
        res.refill_threshold = refills[ri];
      }
    }
  // clear what the trials accumulated
  for (int j = 0; j < n_jobs; ++j) {
    const TraceArgs& T = args[j];
    const int bins = T.prm->per_lambda ? T.optics->n_lambda : 1;
    if (T.absorbed) CK(cudaMemset(T.absorbed, 0, sizeof(double) * (size_t)bins * T.grid->n_cells));
    if (T.obs && T.images)
      CK(cudaMemset(T.images, 0, sizeof(double) * (size_t)T.obs->n_obs * bins * T.obs->nx * T.obs->ny));
  }
  rt_ctx::Tuned& t = ctx->tuned[precision == 64][peel ? 1 : 0];
  t.set = true;
  t.block = res.block_size;
  t.refill = res.refill_threshold;
  t.blocks_per_sm = 0;
  *best = res;
  return RT_OK;
}

extern "C" int rt_tune_save(const rt_ctx* ctx, const char* path) {
  if (!ctx || !path) return fail(RT_ERR_INVALID, "rt_tune_save: NULL argument");
  FILE* f = fopen(path, "w");
  if (!f) return fail(RT_ERR_INVALID, "rt_tune_save: cannot open %s", path);
  fprintf(f, "# arch precision peel block refill blocks_per_sm\n");
  for (int p = 0; p < 2; ++p)
    for (int q = 0; q < 2; ++q) {
      const rt_ctx::Tuned& t = ctx->tuned[p][q];
      if (t.set)
        fprintf(f, "sm_%d%d %d %d %d %d %d\n", ctx->cc_major, ctx->cc_minor, p ? 64 : 32, q, t.block, t.refill,
                t.blocks_per_sm);
    }
  fclose(f);
  return RT_OK;
}

extern "C" int rt_tune_load(rt_ctx* ctx, const char* path) {
  if (!ctx || !path) return fail(RT_ERR_INVALID, "rt_tune_load: NULL argument");
  FILE* f = fopen(path, "r");
  if (!f) return fail(RT_ERR_INVALID, "rt_tune_load: cannot open %s", path);
  char line[256];
  char arch[32];
  char mine[32];
  snprintf(mine, sizeof mine, "sm_%d%d", ctx->cc_major, ctx->cc_minor);
  int loaded = 0;
  while (fgets(line, sizeof line, f)) {
    if (line[0] == '#') continue;
    int prec, peel, block, refill, bps;
    if (sscanf(line, "%31s %d %d %d %d %d", arch, &prec, &peel, &block, &refill, &bps) != 6) continue;
    if (strcmp(arch, mine) != 0 || (prec != 32 && prec != 64) || (peel != 0 && peel != 1)) continue;
    if (block < 32 || block > 256 || block % 32 || refill < 1 || refill > 32 || bps < 0) continue;
    rt_ctx::Tuned& t = ctx->tuned[prec == 64][peel];
    t.set = true;
    t.block = block;
    t.refill = refill;
    t.blocks_per_sm = bps;
    ++loaded;
  }
  fclose(f);
  return loaded > 0 ? RT_OK : fail(RT_ERR_INVALID, "rt_tune_load: no entry for %s in %s", mine, path);
}

// ------------------------------------------------------------------------
// hierarchical model from a full-resolution cube (Sect. 4.1)
// ------------------------------------------------------------------------
extern "C" int rt_merge_uniform(rt_ctx* ctx, const int* root, const double* box, int n_fine_levels,
                                const double* rho_dev, double kappa, double tau_max, double contrast_max,
                                int64_t cap_cells, uint8_t* refine_flags_host, double* density_host,
                                int64_t* n_refined_host, int* n_levels_out, int64_t* n_cells_out, void* cuda_stream) {
  if (!ctx || !root || !box || !rho_dev || !n_refined_host || !n_levels_out || !n_cells_out)
    return fail(RT_ERR_INVALID, "rt_merge_uniform: NULL argument");
  if (cap_cells > 0 && (!refine_flags_host || !density_host))
    return fail(RT_ERR_INVALID, "rt_merge_uniform: output arrays are NULL");
  if (n_fine_levels < 0 || n_fine_levels > 20) return fail(RT_ERR_INVALID, "rt_merge_uniform: n_fine_levels must be 0..20");
  for (int a = 0; a < 3; ++a) {
    if (root[a] < 1 || ((long long)root[a] << n_fine_levels) > (1ll << RT_COORD_BITS))
      return fail(RT_ERR_INVALID, "rt_merge_uniform: root dims must be >= 1 with root * 2^L <= 2^%d", RT_COORD_BITS);
    if (!(box[a] > 0.0) || !std::isfinite(box[a])) return fail(RT_ERR_INVALID, "rt_merge_uniform: bad box size");
  }
  const double h0 = box[0] / root[0];
  for (int a = 1; a < 3; ++a)
    if (std::fabs(box[a] / root[a] - h0) > 1e-12 * h0) return fail(RT_ERR_INVALID, "rt_merge_uniform: cells are not cubic");
  if (!(kappa >= 0.0) || !std::isfinite(kappa) || !(tau_max > 0.0) || !(contrast_max >= 1.0))
    return fail(RT_ERR_INVALID, "rt_merge_uniform: need kappa >= 0, tau_max > 0, contrast_max >= 1");
  CTX_ENTER(ctx);
  DeviceGuard dg(ctx->device);
  const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  long long nref[24] = {0};
  long long nc = 0;
  int nlev = 0;
  const int rc = rtk::merge_uniform(root, h0, n_fine_levels, rho_dev, kappa, tau_max, contrast_max, cap_cells,
                                    refine_flags_host, density_host, nref, &nlev, &nc, s);
  *n_cells_out = nc;
  *n_levels_out = nlev;
  for (int l = 0; l < nlev; ++l) n_refined_host[l] = nref[l];
  return rc;
}
