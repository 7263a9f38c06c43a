// nrr_api.cu -- the C ABI of libnrr (declared in include/nrr.h) and the host
// driver of the relaxation loop (arXiv 2501.14030, Alg. 1).
//
// Set-up runs once per grid on the device; the relaxation loop is a CUDA
// graph of `check_every` RK4 steps (4 fused stage kernels each) followed by
// the residual and its norm, replayed until the norm falls below tol.  The
// only host<->device traffic per chunk is the 8-byte norm.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/nrr.h"
#include "nrr_debug.cuh"
#include "nrr_internal.h"

using namespace nrr;

// ---- NRR_DEBUG address registry (no-ops in the release build) --------------
namespace nrr {
namespace dbgreg {
struct DbgRegistry {
  std::mutex mu;
  std::vector<std::pair<uintptr_t, uintptr_t>> ranges;
  std::vector<std::pair<DbgSync, DbgRead>> units;
  bool overflow = false;
};
DbgRegistry &dbg_registry() {
  static DbgRegistry r;
  return r;
}
#if NRR_DEBUG
// Copies the range list into every translation unit's device table; the
// device is idle first, so that no kernel reads a half-written table.
void dbg_publish(DbgRegistry &r) {
  DbgTable t{};
  t.n = (int)std::min<size_t>(r.ranges.size(), kDbgRanges);
  for (int i = 0; i < t.n; i++) {
    t.lo[i] = r.ranges[i].first;
    t.hi[i] = r.ranges[i].second;
  }
  cudaDeviceSynchronize();
  for (auto &u : r.units) u.first(t);
}
#endif
}  // namespace dbgreg
using dbgreg::DbgRegistry;
using dbgreg::dbg_registry;

void dbg_add_unit(DbgSync sync, DbgRead read) {
  DbgRegistry &r = dbg_registry();
  std::lock_guard<std::mutex> lock(r.mu);
  r.units.emplace_back(sync, read);
}

void dbg_register(const void *p, size_t bytes) {
#if NRR_DEBUG
  // NaN poison (all bits set is a NaN in FP32 and FP64): a kernel that reads
  // memory the library never wrote then produces NaN instead of plausible
  // numbers
  cudaMemset(const_cast<void *>(p), 0xFF, bytes);
  DbgRegistry &r = dbg_registry();
  std::lock_guard<std::mutex> lock(r.mu);
  if (r.ranges.size() >= (size_t)kDbgRanges) r.overflow = true;
  r.ranges.emplace_back((uintptr_t)p, (uintptr_t)p + bytes);
  dbgreg::dbg_publish(r);
#else
  (void)p;
  (void)bytes;
#endif
}

void dbg_unregister(const void *p) {
#if NRR_DEBUG
  DbgRegistry &r = dbg_registry();
  std::lock_guard<std::mutex> lock(r.mu);
  for (size_t i = 0; i < r.ranges.size(); i++)
    if (r.ranges[i].first == (uintptr_t)p) {
      r.ranges.erase(r.ranges.begin() + (long)i);
      break;
    }
  dbgreg::dbg_publish(r);
#else
  (void)p;
#endif
}
}  // namespace nrr

namespace {

thread_local std::string g_last_error;
std::atomic<int64_t> g_launches{0};

nrr_status fail(nrr_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

#define CUDA_TRY(call)                                                     \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess)                                                 \
      return fail(NRR_ERR_CUDA, "%s: %s (%s:%d)", #call,                   \
                  cudaGetErrorString(e_), __FILE__, __LINE__);             \
  } while (0)

#define TRY(expr)                     \
  do {                                \
    nrr_status s_ = (expr);           \
    if (s_ != NRR_OK) return s_;      \
  } while (0)

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

void nrr::set_last_error(const char *msg) { g_last_error = msg; }

struct GraphKey {
  int mode, steps;
  double dt, eta, r_int;
  bool operator<(const GraphKey &o) const {
    return std::tie(mode, steps, dt, eta, r_int) <
           std::tie(o.mode, o.steps, o.dt, o.eta, o.r_int);
  }
};

// Control block of a relaxation whose stop test runs on the device (Alg. 1:
// evaluate the norm, stop below tol, else take more RK steps): the host
// writes the first three fields, the control kernel the rest.
struct RelaxCtl {
  double tol;
  long long max_chunks;            // chunks of check_every steps allowed
  unsigned long long timeout_ns;   // 0: no limit
  long long chunks;                // chunks completed
  double norm;                     // the last norm
  unsigned long long t0_ns;        // %globaltimer at the first test
  int timed_out;
  int pad;
};

namespace {

// After each norm evaluation: counts the chunk, keeps the norm, and lets the
// WHILE node run the body again while the norm is finite and >= tol, the
// chunk limit is not reached and the device-timed limit has not passed.
__global__ void relax_control_kernel(const double *norm, RelaxCtl *c,
                                     cudaGraphConditionalHandle h, int first) {
  unsigned long long now;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
  if (first) {
    c->t0_ns = now;
    c->chunks = 0;
    c->timed_out = 0;
  } else {
    c->chunks += 1;
  }
  const double n = *norm;
  c->norm = n;
  bool go = isfinite(n) && n >= c->tol && c->chunks < c->max_chunks;
  if (go && c->timeout_ns > 0 && now - c->t0_ns > c->timeout_ns) {
    c->timed_out = 1;
    go = false;
  }
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

// The defect correction's increment (d, w) starts from rest.
__global__ void zero2_kernel(float *a, float *b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    a[i] = 0.f;
    b[i] = 0.f;
  }
}

}  // namespace

struct nrr_grid {
  nrr_grid_desc desc{};
  Geo geo{};
  cudaStream_t stream = nullptr;       // the grid's own work stream
  cudaStream_t user_stream = nullptr;  // caller's stream (ordering only)
  cudaEvent_t order_ev = nullptr;
  int device = 0;
  LaunchCfg res_cfg{128, 2};  // residual kernels (fixed: sizes the partials)
  LaunchCfg stage_cfg[2];  // stage kernels, [0] FP64, [1] FP32 (autotuned)
  std::vector<void *> allocs;

  FieldSet<double> f64;
  FieldSet<float> f32;
  ColumnSet<double> c64;
  ColumnSet<float> c32;
  CartCoef cart{};
  // column geometry
  double *h = nullptr, *gl = nullptr, *rad = nullptr, *drdxx0 = nullptr,
         *jac = nullptr, *dsmin = nullptr;
  double *scalars = nullptr;   // [0] dsmin_global, [1..3] norm out
  double *partials = nullptr;
  int *flag = nullptr;
  double *host_pinned = nullptr;  // norm read-back
  // defect correction
  double *res64 = nullptr;
  double *u_save = nullptr;
  float *acoef32 = nullptr;
  float *rhs32 = nullptr;
  float *fu32 = nullptr;

  double dsmin_global = 0.0;
  bool have_source = false;
  PunctureSet punct{};  // the last set of punctures (source recomputation)
  int state_prec = 64;  // which FieldSet holds the current state
  std::map<GraphKey, cudaGraphExec_t> graphs;
  std::map<GraphKey, int64_t> graph_kernels;
  // whole-solve graphs (conditional WHILE node): kernels of the prologue and
  // of one chunk of the loop body
  std::map<GraphKey, std::pair<int64_t, int64_t>> loop_kernels;
  int device_loop = 1;          // stop test on the device (one graph launch)
  struct RelaxCtl *ctl = nullptr;       // device control block
  struct RelaxCtl *ctl_host = nullptr;  // pinned mirror
};

namespace {

// Autotuned launch shapes, remembered per (coordinates, n, order, precision)
// for the life of the process.
struct TuneKey {
  int coord, n0, n1, n2, ng, prec;
  bool operator<(const TuneKey &o) const {
    return std::tie(coord, n0, n1, n2, ng, prec) <
           std::tie(o.coord, o.n0, o.n1, o.n2, o.ng, o.prec);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, LaunchCfg> g_tuned;

TuneKey tune_key(const Geo &g, int prec) {
  return TuneKey{g.coord, g.n0, g.n1, g.n2, g.ng, prec};
}

LaunchCfg tuned_or_default(const Geo &g, int prec) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tuned.find(tune_key(g, prec));
  return it != g_tuned.end() ? it->second : LaunchCfg{};
}

// Whether a launch shape is one nrr_set_launch accepts.
bool valid_shape(const LaunchCfg &c) {
  const bool zc_ok =
      c.variant == 0   ? (c.zc == 1 || c.zc == 2 || c.zc == 4)
      : (c.variant == 1 || c.variant == 3 || c.variant == 5)
          ? (c.zc == 2 || c.zc == 4 || c.zc == 8 || c.zc == 16)
          : (c.variant == 2 || c.variant == 4 || c.variant == 6) && c.zc == 1;
  return c.variant >= 0 && c.variant <= 6 && zc_ok &&
         (c.block == 32 || c.block == 64 || c.block == 128 || c.block == 256) &&
         (c.pdl == 0 || c.pdl == 1);
}

// Integer value of "key": in [b, e) of a JSON object; false if absent.
bool json_int(const char *b, const char *e, const char *key, int *out) {
  char pat[64];
  snprintf(pat, sizeof pat, "\"%s\"", key);
  const size_t n = strlen(pat);
  for (const char *p = b; p + n <= e; p++) {
    if (strncmp(p, pat, n) != 0) continue;
    p += n;
    while (p < e && (*p == ' ' || *p == ':' || *p == '\t' || *p == '\n' || *p == '[')) p++;
    char *end = nullptr;
    long v = strtol(p, &end, 10);
    if (end == p || end > e) return false;
    *out = (int)v;
    return true;
  }
  return false;
}

// The three integers of "n": [a, b, c].
bool json_int3(const char *b, const char *e, const char *key, int out[3]) {
  char pat[64];
  snprintf(pat, sizeof pat, "\"%s\"", key);
  const char *p = strstr(b, pat);
  if (!p || p >= e) return false;
  p = strchr(p, '[');
  if (!p || p >= e) return false;
  p++;
  for (int i = 0; i < 3; i++) {
    char *end = nullptr;
    long v = strtol(p, &end, 10);
    if (end == p || end > e) return false;
    out[i] = (int)v;
    p = end;
    while (p < e && (*p == ',' || *p == ' ')) p++;
  }
  return true;
}

template <typename T>
nrr_status dev_alloc(nrr_grid *g, T **p, size_t count) {
  void *ptr = nullptr;
  cudaError_t e = cudaMalloc(&ptr, count * sizeof(T));
  if (e != cudaSuccess)
    return fail(NRR_ERR_OOM, "cudaMalloc of %zu bytes: %s", count * sizeof(T),
                cudaGetErrorString(e));
  g->allocs.push_back(ptr);
  dbg_register(ptr, count * sizeof(T));
  *p = static_cast<T *>(ptr);
  return NRR_OK;
}

size_t footprint_bytes(const Geo &geo) {
  size_t n = (size_t)geo.npts, nc = (size_t)geo.ncol;
  size_t b = 0;
  b += n * (10 * 8 + 10 * 4);          // FP64 + FP32 field sets
  b += n * (8 + 8 + 4 + 4 + 4);        // defect-correction buffers
  b += nc * 8 * (3 + 2 + 4);           // column geometry
  b += nc * (8 + 4) * (ncoef(geo.ng) + 5);
  b += (size_t)(geo.ncol / 32 + 16) * 16 * ((geo.n2 + 1)) + (1 << 20);
  return b;
}

}  // namespace

nrr_status nrr::check_grid_desc(const nrr_grid_desc *d) {
  if (!d) return fail(NRR_ERR_INVALID_ARG, "null grid descriptor");
  if (d->coord < NRR_SINHSYMTP || d->coord > NRR_SINHCYLINDRICAL)
    return fail(NRR_ERR_INVALID_ARG, "unknown coordinate system %d", d->coord);
  if (d->fd_order != 4 && d->fd_order != 8 && d->fd_order != 10)
    return fail(NRR_ERR_INVALID_ARG, "fd_order must be 4, 8 or 10 (got %d)",
                d->fd_order);
  int ng = d->fd_order / 2;
  for (int i = 0; i < 3; i++)
    if (d->n[i] < 1 || d->n[i] > (1 << 16))
      return fail(NRR_ERR_INVALID_ARG, "n[%d] = %d out of range", i, d->n[i]);
  // Per-column arrays are indexed with 32-bit integers: the padded plane
  // s0*s1 (computed in 64 bits here) must fit.
  const int64_t plane = (int64_t)(d->n[0] + 2 * ng) * (int64_t)(d->n[1] + 2 * ng);
  if (plane > (int64_t)INT32_MAX)
    return fail(NRR_ERR_INVALID_ARG, "padded plane s0*s1 = %lld exceeds 2^31 - 1",
                (long long)plane);
  if (d->coord != NRR_CARTESIAN) {
    if (d->n[2] & 1)
      return fail(NRR_ERR_INVALID_ARG, "n2 must be even on curvilinear grids");
    if (d->n[1] < ng)
      return fail(NRR_ERR_INVALID_ARG, "n1 must be >= fd_order/2");
    if (d->n[0] < ng)
      return fail(NRR_ERR_INVALID_ARG, "n0 must be >= fd_order/2");
  } else {
    for (int i = 0; i < 3; i++)
      if (d->n[i] < 2)
        return fail(NRR_ERR_INVALID_ARG, "Cartesian n must be >= 2");
  }
  if (d->coord == NRR_SINHSYMTP &&
      !(d->amax > 0 && d->sinhwaa > 0 && d->bscale >= 0))
    return fail(NRR_ERR_INVALID_ARG, "SinhSymTP needs amax > 0, sinhwaa > 0");
  if (d->coord == NRR_SPHERICAL && !(d->rmax > 0))
    return fail(NRR_ERR_INVALID_ARG, "Spherical needs rmax > 0");
  if (d->coord == NRR_SINHSPHERICAL && !(d->amax > 0 && d->sinhwaa > 0))
    return fail(NRR_ERR_INVALID_ARG, "SinhSpherical needs amax > 0, sinhwaa > 0");
  if (d->coord == NRR_CARTESIAN && !(d->xmax > 0))
    return fail(NRR_ERR_INVALID_ARG, "Cartesian needs xmax > 0");
  if (d->coord == NRR_SINHCYLINDRICAL &&
      !(d->amax > 0 && d->sinhwaa > 0 && d->zmax > 0 && d->sinhwz > 0))
    return fail(NRR_ERR_INVALID_ARG,
                "SinhCylindrical needs amax, sinhwaa, zmax, sinhwz > 0");
  return NRR_OK;
}

Geo nrr::grid_geo(const nrr_grid_desc *d) {
  Geo g{};
  g.coord = d->coord;
  g.n0 = d->n[0];
  g.n1 = d->n[1];
  g.n2 = d->n[2];
  g.ng = d->fd_order / 2;
  g.s0 = g.n0 + 2 * g.ng;
  g.s1 = g.n1 + 2 * g.ng;
  g.s2 = g.n2 + 2 * g.ng;
  g.ncol = g.s0 * g.s1;
  g.npts = (int64_t)g.ncol * g.s2;
  double xmin[3], xmax[3];
  if (d->coord == NRR_CARTESIAN) {
    for (int i = 0; i < 3; i++) {
      xmin[i] = -d->xmax;
      xmax[i] = d->xmax;
    }
  } else {
    xmin[0] = 0.0;
    xmax[0] = (d->coord == NRR_SINHSYMTP || d->coord == NRR_SINHSPHERICAL ||
               d->coord == NRR_SINHCYLINDRICAL) ? 1.0 : d->rmax;
    xmin[1] = d->coord == NRR_SINHCYLINDRICAL ? -1.0 : 0.0;
    xmax[1] = d->coord == NRR_SINHCYLINDRICAL ? 1.0 : M_PI;
    xmin[2] = -M_PI;
    xmax[2] = M_PI;
  }
  int n[3] = {g.n0, g.n1, g.n2};
  for (int i = 0; i < 3; i++) {
    g.xxmin[i] = xmin[i];
    g.dxx[i] = (xmax[i] - xmin[i]) / n[i];
  }
  g.amax = d->amax;
  g.bscale = d->bscale;
  g.sinhwaa = d->sinhwaa;
  g.zmax = d->zmax;
  g.sinhwz = d->sinhwz;
  return g;
}

namespace {

template <typename R>
StageArgs<R> stage_args(const nrr_grid *g, const FieldSet<R> &f,
                        const ColumnSet<R> &c, int stage, double dt,
                        double eta) {
  return rk4_stage_args<R>(f, c, g->cart, g->flag + 2, stage, dt, eta);
}

template <typename R>
void launch_rk4_steps(const nrr_grid *g, const FieldSet<R> &f,
                      const ColumnSet<R> &c, double dt, double eta,
                      int64_t steps) {
  static const int kinds[4] = {STAGE_FIRST, STAGE_MID, STAGE_MID, STAGE_LAST};
  const LaunchCfg &cfg = g->stage_cfg[sizeof(R) == 4];
  if constexpr (sizeof(R) == 4) {
    if (cfg.variant == 6 && stage2_ok(g->geo)) {
      // two stages per launch over an even number of steps (the state
      // returns to f.y), then one step of single-stage launches if odd
      const int64_t pairs = steps - (steps & 1);
      g_launches += 2 * pairs;
      launch_stage2_steps(g->geo, f, c, dt, eta, pairs, cfg.pdl, g->stream);
      if (steps & 1) {
        LaunchCfg col = cfg;
        col.variant = 0;
        col.zc = 2;
        g_launches += 4;
        for (int k = 0; k < 4; k++)
          launch_stage<R>(g->geo, kinds[k], stage_args<R>(g, f, c, k, dt, eta), col,
                          g->stream);
      }
      return;
    }
  }
  if ((cfg.variant == 4 || cfg.variant == 5) && g->geo.coord != CARTESIAN &&
      g->geo.coord != SINHCYLINDRICAL) {
    // all steps in one cooperative launch (grid barriers between stages)
    StageArgs<R> sa[4];
    for (int k = 0; k < 4; k++) sa[k] = stage_args<R>(g, f, c, k, dt, eta);
    g_launches += 1;
    launch_stage_steps<R>(g->geo, sa, (int)steps,
                          reinterpret_cast<unsigned *>(g->flag + 3), cfg, g->stream);
    return;
  }
  g_launches += 4 * steps;
  for (int64_t s = 0; s < steps; s++)
    for (int k = 0; k < 4; k++)
      launch_stage<R>(g->geo, kinds[k], stage_args<R>(g, f, c, k, dt, eta), cfg,
                      g->stream);
}

// Residual + norm of the current state in precision R into scalars[1..3].
template <typename R>
void launch_norm(const nrr_grid *g, const FieldSet<R> &f, const ColumnSet<R> &c,
                 double r_int, double *h_out) {
  int nb = 0;
  g_launches += 2;
  launch_residual<R>(g->geo, f.y[0], f.alpha, f.bc2, c, g->cart, g->jac,
                     g->rad, r_int, h_out, g->partials, &nb, g->res_cfg,
                     g->stream, f.lin);
  launch_norm_finalize(g->partials, nb, g->scalars + 1, g->stream);
}

// After the stream has drained: NRR_ERR_TIMEOUT (and the flag cleared) if a
// stage kernel's bounded wait -- for its tensor copies or at a grid barrier --
// expired since the flag was last cleared.
nrr_status take_stage_error(nrr_grid *g) {
  int stage_err = 0;
  CUDA_TRY(cudaMemcpyAsync(&stage_err, g->flag + 2, sizeof(int),
                           cudaMemcpyDeviceToHost, g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  if (!stage_err) return NRR_OK;
  CUDA_TRY(cudaMemsetAsync(g->flag + 2, 0, sizeof(int), g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  return fail(NRR_ERR_TIMEOUT, "a stage kernel's bounded wait expired");
}

nrr_status sync_read_norm(nrr_grid *g, double *out) {
  CUDA_TRY(cudaMemcpyAsync(g->host_pinned, g->scalars + 1, sizeof(double),
                           cudaMemcpyDeviceToHost, g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  *out = g->host_pinned[0];
  return NRR_OK;
}

// Make the requested precision hold the current state.
nrr_status ensure_state(nrr_grid *g, int prec) {
  if (g->state_prec == prec) return NRR_OK;
  int64_t n = g->geo.npts;
  for (int c = 0; c < 2; c++) {
    if (prec == 32)
      launch_convert(g->f64.y[c], g->f32.y[c], n, g->stream);
    else
      launch_convert(g->f32.y[c], g->f64.y[c], n, g->stream);
  }
  CUDA_TRY(cudaGetLastError());
  g->state_prec = prec;
  return NRR_OK;
}

// The FP32 field set of the defect correction's increment equation: (d, w)
// in the FP32 state buffers, with c^2 a in place of alpha and the FP64
// defect (f_u, f_v) as forcing.
FieldSet<float> dc_fields(const nrr_grid *g) {
  FieldSet<float> dc = g->f32;
  dc.alpha = g->acoef32;
  dc.bc2 = g->rhs32;
  dc.fu = g->fu32;
  dc.lin = 1;
  return dc;
}

nrr_status get_graph(nrr_grid *g, int mode, int steps, double dt, double eta,
                     double r_int, cudaGraphExec_t *out) {
  GraphKey key{mode, steps, dt, eta, r_int};
  auto it = g->graphs.find(key);
  if (it != g->graphs.end()) {
    *out = it->second;
    return NRR_OK;
  }
  cudaGraph_t graph;
  int64_t before = g_launches.load();
  CUDA_TRY(cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
  if (mode == NRR_FP32) {
    launch_rk4_steps<float>(g, g->f32, g->c32, dt, eta, steps);
    launch_norm<float>(g, g->f32, g->c32, r_int, nullptr);
  } else if (mode == NRR_FP32_DC) {
    // defect-correction inner steps, FP64 update, FP64 norm
    FieldSet<float> dc = dc_fields(g);
    launch_rk4_steps<float>(g, dc, g->c32, dt, eta, steps);
    launch_dc_update(g->f64.y[0], g->f64.y[1], g->f32.y[0], g->f32.y[1],
                     g->geo.npts, g->stream);
    g_launches += 1;
    launch_norm<double>(g, g->f64, g->c64, r_int, nullptr);
  } else {
    launch_rk4_steps<double>(g, g->f64, g->c64, dt, eta, steps);
    launch_norm<double>(g, g->f64, g->c64, r_int, nullptr);
  }
  cudaError_t e = cudaStreamEndCapture(g->stream, &graph);
  if (e != cudaSuccess)
    return fail(NRR_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
  cudaGraphExec_t exec;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess)
    return fail(NRR_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  g->graphs[key] = exec;
  // captured launches are not executed: count them once per replay instead
  g->graph_kernels[key] = g_launches.load() - before;
  g_launches -= g->graph_kernels[key];
  *out = exec;
  return NRR_OK;
}

nrr_status check_grid(const nrr_grid *g) {
  if (!g) return fail(NRR_ERR_INVALID_ARG, "null grid");
  return NRR_OK;
}

// Every call starts by making the grid's work stream wait for the work the
// caller has queued on its own stream (inputs produced there), and ends
// after the work stream has drained.
nrr_status set_device(const nrr_grid *g) {
  CUDA_TRY(cudaSetDevice(g->device));
  CUDA_TRY(cudaEventRecord(g->order_ev, g->user_stream));
  CUDA_TRY(cudaStreamWaitEvent(g->stream, g->order_ev, 0));
  return NRR_OK;
}

// Relaxes the current state chunk by chunk (check_every steps, then the norm)
// in the given mode; *norm holds the last norm.  Stops below tol, at
// max_steps, on a non-finite norm or at the wall-clock limit.
nrr_status relax_chunks(nrr_grid *g, int mode, double dt, double eta,
                        double tol, double r_int, int check_every,
                        int64_t max_steps, double t_start, int64_t timeout_ms,
                        int64_t *steps_done, double *norm, nrr_status *why) {
  int64_t it = 0;
  *why = NRR_ERR_NOT_CONVERGED;
  for (;;) {
    if (!std::isfinite(*norm)) {
      *why = NRR_ERR_DIVERGED;
      break;
    }
    if (*norm < tol) {
      *why = NRR_OK;
      break;
    }
    if (it >= max_steps) break;
    if (timeout_ms > 0 && (now_s() - t_start) * 1e3 > (double)timeout_ms) {
      *why = NRR_ERR_TIMEOUT;
      break;
    }
    int64_t m = check_every;
    if (max_steps - it < m) m = max_steps - it;
    if (m == check_every) {
      cudaGraphExec_t exec;
      TRY(get_graph(g, mode, (int)m, dt, eta, r_int, &exec));
      CUDA_TRY(cudaGraphLaunch(exec, g->stream));
      g_launches += g->graph_kernels[GraphKey{mode, (int)m, dt, eta, r_int}];
    } else if (mode == NRR_FP32) {
      launch_rk4_steps<float>(g, g->f32, g->c32, dt, eta, m);
      launch_norm<float>(g, g->f32, g->c32, r_int, nullptr);
    } else {
      launch_rk4_steps<double>(g, g->f64, g->c64, dt, eta, m);
      launch_norm<double>(g, g->f64, g->c64, r_int, nullptr);
    }
    CUDA_TRY(cudaGetLastError());
    TRY(sync_read_norm(g, norm));
    it += m;
  }
  *steps_done = it;
  return NRR_OK;
}

// The start of one defect-correction outer iteration: the FP64 defect
// F = the relaxation system's right-hand side at (u, v) (into the FP64 t
// buffers), the FP32 coefficient c^2 a and forcings from it, and the
// increment (d, w) set to rest.
void launch_dc_outer_prep(const nrr_grid *g, double eta, cudaStream_t st) {
  const Geo &geo = g->geo;
  double *Fu = g->f64.t[0], *Fv = g->f64.t[1];
  StageArgs<double> ra{};
  ra.su = g->f64.y[0];
  ra.sv = g->f64.y[1];
  ra.ou = Fu;
  ra.ov = Fv;
  ra.alpha = g->f64.alpha;
  ra.bc2 = g->f64.bc2;
  ra.col = g->c64;
  ra.cart = g->cart;
  ra.eta = eta;
  ra.err = g->flag + 2;  // a tensor-copy variant's bounded-wait flag
  launch_stage<double>(geo, STAGE_RAW, ra, g->stage_cfg[0], st);
  launch_dc_prepare(geo, g->f64.y[0], g->f64.alpha, g->f64.bc2, Fu, Fv,
                    g->acoef32, g->fu32, g->rhs32, st);
  const int64_t n = geo.npts;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
  zero2_kernel<<<blocks, 256, 0, st>>>(g->f32.y[0], g->f32.y[1], n);
  g_launches += 3;
}
void launch_dc_outer_prep(const nrr_grid *g, double eta) {
  launch_dc_outer_prep(g, eta, g->stream);
}

// One whole solve as one graph: the norm of the current state and the stop
// test (prologue), then a conditional WHILE node whose body is one chunk --
// check_every RK4 steps (FP64 or FP32), or one defect-correction outer
// iteration of `every` FP32 steps with its FP64 update -- followed by the
// norm and the stop test.  The control block's tol, chunk limit and timeout
// are read on the device at each replay.
nrr_status get_loop_graph(nrr_grid *g, int mode, int every, double dt,
                          double eta, double r_int, cudaGraphExec_t *out,
                          std::pair<int64_t, int64_t> *kernels) {
  GraphKey key{mode + 100, every, dt, eta, r_int};
  auto it = g->graphs.find(key);
  if (it != g->graphs.end()) {
    *out = it->second;
    *kernels = g->loop_kernels[key];
    return NRR_OK;
  }
  cudaGraph_t graph;
  CUDA_TRY(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle handle;
  cudaError_t e = cudaGraphConditionalHandleCreate(&handle, graph, 1,
                                                   cudaGraphCondAssignDefault);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return fail(NRR_ERR_CUDA, "conditional handle: %s", cudaGetErrorString(e));
  }
  int64_t before = g_launches.load();
  e = cudaStreamBeginCaptureToGraph(g->stream, graph, nullptr, nullptr, 0,
                                    cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return fail(NRR_ERR_CUDA, "prologue capture: %s", cudaGetErrorString(e));
  }
  if (mode == NRR_FP32)
    launch_norm<float>(g, g->f32, g->c32, r_int, nullptr);
  else
    launch_norm<double>(g, g->f64, g->c64, r_int, nullptr);
  relax_control_kernel<<<1, 1, 0, g->stream>>>(g->scalars + 1, g->ctl, handle, 1);
  g_launches += 1;
  cudaGraph_t captured = nullptr;
  e = cudaStreamEndCapture(g->stream, &captured);
  const int64_t n_pro = g_launches.load() - before;
  if (e != cudaSuccess) {
    g_launches -= n_pro;
    cudaGraphDestroy(graph);
    return fail(NRR_ERR_CUDA, "prologue capture: %s", cudaGetErrorString(e));
  }
  // the WHILE node after the prologue's last node
  size_t nn = 0;
  std::vector<cudaGraphNode_t> nodes, sinks;
  e = cudaGraphGetNodes(graph, nullptr, &nn);
  if (e == cudaSuccess) {
    nodes.resize(nn);
    e = cudaGraphGetNodes(graph, nodes.data(), &nn);
  }
  for (size_t i = 0; e == cudaSuccess && i < nn; i++) {
    size_t nout = 0;
    e = cudaGraphNodeGetDependentNodes(nodes[i], nullptr, nullptr, &nout);
    if (e == cudaSuccess && nout == 0) sinks.push_back(nodes[i]);
  }
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = handle;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t wnode;
  if (e == cudaSuccess)
    e = cudaGraphAddNode(&wnode, graph, sinks.data(), nullptr, sinks.size(), &cp);
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(g->stream, cp.conditional.phGraph_out[0],
                                      nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    g_launches -= n_pro;
    cudaGraphDestroy(graph);
    return fail(NRR_ERR_CUDA, "loop graph: %s", cudaGetErrorString(e));
  }
  const int64_t before_body = g_launches.load();
  if (mode == NRR_FP32_DC) {
    launch_dc_outer_prep(g, eta);
    FieldSet<float> dc = dc_fields(g);
    launch_rk4_steps<float>(g, dc, g->c32, dt, eta, every);
    launch_dc_update(g->f64.y[0], g->f64.y[1], g->f32.y[0], g->f32.y[1],
                     g->geo.npts, g->stream);
    g_launches += 1;
    launch_norm<double>(g, g->f64, g->c64, r_int, nullptr);
  } else if (mode == NRR_FP32) {
    launch_rk4_steps<float>(g, g->f32, g->c32, dt, eta, every);
    launch_norm<float>(g, g->f32, g->c32, r_int, nullptr);
  } else {
    launch_rk4_steps<double>(g, g->f64, g->c64, dt, eta, every);
    launch_norm<double>(g, g->f64, g->c64, r_int, nullptr);
  }
  relax_control_kernel<<<1, 1, 0, g->stream>>>(g->scalars + 1, g->ctl, handle, 0);
  g_launches += 1;
  e = cudaStreamEndCapture(g->stream, &captured);
  const int64_t n_body = g_launches.load() - before_body;
  g_launches -= n_pro + n_body;  // captured, not executed
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return fail(NRR_ERR_CUDA, "loop body capture: %s", cudaGetErrorString(e));
  }
  cudaGraphExec_t exec;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess)
    return fail(NRR_ERR_CUDA, "loop graph instantiate: %s", cudaGetErrorString(e));
  g->graphs[key] = exec;
  g->loop_kernels[key] = {n_pro, n_body};
  *out = exec;
  *kernels = {n_pro, n_body};
  return NRR_OK;
}

// Up to max_chunks chunks of `every` steps with the stop test on the device,
// in one graph launch and one read-back of the control block.  *chunks,
// *norm: chunks done and the last norm; *timed_out: the device-timed limit
// stopped it.
nrr_status relax_device_loop(nrr_grid *g, int mode, int every, double dt,
                             double eta, double tol, double r_int,
                             int64_t max_chunks, int64_t timeout_ms,
                             double t_start, int64_t *chunks, double *norm,
                             bool *timed_out) {
  cudaGraphExec_t exec;
  std::pair<int64_t, int64_t> kern;
  TRY(get_loop_graph(g, mode, every, dt, eta, r_int, &exec, &kern));
  RelaxCtl *h = g->ctl_host;
  memset(h, 0, sizeof *h);
  h->tol = tol;
  h->max_chunks = max_chunks;
  if (timeout_ms > 0) {
    const double left_ms = (double)timeout_ms - (now_s() - t_start) * 1e3;
    h->timeout_ns = left_ms > 1e-3 ? (unsigned long long)(left_ms * 1e6) : 1ull;
  }
  CUDA_TRY(cudaMemcpyAsync(g->ctl, h, sizeof *h, cudaMemcpyHostToDevice, g->stream));
  CUDA_TRY(cudaGraphLaunch(exec, g->stream));
  CUDA_TRY(cudaMemcpyAsync(h, g->ctl, sizeof *h, cudaMemcpyDeviceToHost, g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  *chunks = h->chunks;
  *norm = h->norm;
  *timed_out = h->timed_out != 0;
  g_launches += kern.first + h->chunks * kern.second;
  return NRR_OK;
}

// Defect correction of the relaxation itself.  Outer iteration, in FP64:
// the full right-hand side F of the relaxation system (with its boundary
// conditions) at the current state (u, v) -- the defect -- and the
// linearisation coefficient a of the source at u.  Inner, in FP32: the
// increment (d, w) from rest by `inner_steps` RK4 steps of
//   dd/dt = w - eta d + F_u,   dw/dt = c^2 (lap d - a d) + F_v
// (radiation condition plus F on the outer shell).  Then (u, v) += (d, w) in
// FP64 and the FP64 residual norm decides whether to stop.  The fixed point
// has F = 0, i.e. the FP64 discrete solution; FP32 rounding enters only
// through the increments.
nrr_status relax_defect_correction(nrr_grid *g, const nrr_relax_opts *o,
                                   double dt, double eta, double t_start,
                                   nrr_relax_result *res) {
  const Geo &geo = g->geo;
  TRY(ensure_state(g, 64));
  const int64_t inner = o->inner_steps > 0 ? o->inner_steps : o->check_every;
  double norm64 = 0.0;
  int64_t steps_total = 0;
  int64_t outer = 0;
  nrr_status status = NRR_ERR_NOT_CONVERGED;
  bool timed_out = false;
  if (g->device_loop) {
    // every whole outer iteration that max_iters and max_outer allow, with
    // the stop test on the device; the host loop below finishes a shorter
    // last one, if any
    int64_t max_chunks = o->max_iters / inner;
    if (o->max_outer > 0) max_chunks = std::min<int64_t>(max_chunks, o->max_outer);
    int64_t chunks = 0;
    TRY(relax_device_loop(g, NRR_FP32_DC, (int)inner, dt, eta, o->tol, o->r_int,
                          max_chunks, o->timeout_ms, t_start, &chunks, &norm64,
                          &timed_out));
    steps_total = chunks * inner;
    outer = chunks;
    if (timed_out) status = NRR_ERR_TIMEOUT;
  } else {
    launch_norm<double>(g, g->f64, g->c64, o->r_int, nullptr);
    TRY(sync_read_norm(g, &norm64));
  }
  FieldSet<float> dc = dc_fields(g);
  for (; !timed_out;) {
    if (!std::isfinite(norm64)) {
      status = NRR_ERR_DIVERGED;
      break;
    }
    if (norm64 < o->tol) {
      status = NRR_OK;
      break;
    }
    if ((o->max_outer > 0 && outer >= o->max_outer) || steps_total >= o->max_iters)
      break;
    if (o->timeout_ms > 0 && (now_s() - t_start) * 1e3 > (double)o->timeout_ms) {
      status = NRR_ERR_TIMEOUT;
      break;
    }
    int64_t m = inner;
    if (o->max_iters - steps_total < m) m = o->max_iters - steps_total;
    launch_dc_outer_prep(g, eta);
    if (m == inner) {
      cudaGraphExec_t exec;
      TRY(get_graph(g, NRR_FP32_DC, (int)m, dt, eta, o->r_int, &exec));
      CUDA_TRY(cudaGraphLaunch(exec, g->stream));
      g_launches += g->graph_kernels[GraphKey{NRR_FP32_DC, (int)m, dt, eta, o->r_int}];
    } else {
      launch_rk4_steps<float>(g, dc, g->c32, dt, eta, m);
      launch_dc_update(g->f64.y[0], g->f64.y[1], g->f32.y[0], g->f32.y[1],
                       geo.npts, g->stream);
      launch_norm<double>(g, g->f64, g->c64, o->r_int, nullptr);
      g_launches += 1;
    }
    CUDA_TRY(cudaGetLastError());
    TRY(sync_read_norm(g, &norm64));
    steps_total += m;
    outer++;
  }
  g->state_prec = 64;
  res->iters = steps_total;
  res->outer_iters = outer;
  res->final_norm = norm64;
  res->status = status;
  return NRR_OK;
}

}  // namespace

GridView nrr::grid_view(nrr_grid *g) {
  GridView v{};
  v.geo = g->geo;
  v.stream = g->stream;
  v.f64 = g->f64;
  v.c64 = g->c64;
  v.cart = g->cart;
  v.cfg64 = g->stage_cfg[0];
  v.res_cfg = g->res_cfg;
  v.jac = g->jac;
  v.rad = g->rad;
  v.scratch = g->res64;
  v.partials = g->partials;
  v.err = g->flag + 2;
  v.dsmin = g->dsmin_global;
  v.have_source = g->have_source;
  v.dc32 = dc_fields(g);
  v.c32 = g->c32;
  v.cfg32 = g->stage_cfg[1];
  return v;
}

void nrr::dc_outer_prep(nrr_grid *g, double eta, cudaStream_t st) {
  launch_dc_outer_prep(g, eta, st);
}

void nrr::dc_outer_update(nrr_grid *g, cudaStream_t st) {
  launch_dc_update(g->f64.y[0], g->f64.y[1], g->f32.y[0], g->f32.y[1], g->geo.npts, st);
  g_launches += 1;
}

// ------------------------------------------------------------------ C ABI

extern "C" {

const char *nrr_last_error(void) { return g_last_error.c_str(); }
int64_t nrr_kernel_launches(void) { return g_launches.load(); }
const char *nrr_version(void) {
  return NRR_DEBUG ? "nrr 0.1 (sm_103a, NRR_DEBUG address checks)" : "nrr 0.1 (sm_103a)";
}

nrr_status nrr_debug_check(int *enabled, unsigned long long *first_bad,
                           unsigned long long *refused) {
  unsigned long long bad = 0, cnt = 0;
  bool overflow = false;
  if (NRR_DEBUG) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess)
      return fail(NRR_ERR_CUDA, "cudaDeviceSynchronize: %s", cudaGetErrorString(e));
    DbgRegistry &r = dbg_registry();
    std::lock_guard<std::mutex> lock(r.mu);
    for (auto &u : r.units) u.second(&bad, &cnt);
    overflow = r.overflow;
    r.overflow = false;
  }
  if (enabled) *enabled = NRR_DEBUG ? 1 : 0;
  if (first_bad) *first_bad = bad;
  if (refused) *refused = cnt;
  if (overflow)
    return fail(NRR_ERR_STATE, "more than %d allocations were alive: the address "
                "check missed some", kDbgRanges);
  return NRR_OK;
}

nrr_status nrr_default_opts(nrr_relax_opts *o) {
  if (!o) return fail(NRR_ERR_INVALID_ARG, "null opts");
  memset(o, 0, sizeof *o);
  o->mode = NRR_FP64;
  o->tol = 1e-10;
  o->max_iters = 1000000;
  o->check_every = 50;
  o->cfl = 0.5;
  o->eta = 0.0;
  o->r_int = 100.0;
  o->initial = NRR_INIT_ZERO;
  o->u0 = nullptr;
  o->timeout_ms = 0;
  o->inner_steps = 0;
  o->max_outer = 0;
  return NRR_OK;
}

nrr_status nrr_image_map(const nrr_grid_desc *d, int32_t *out) {
  TRY(check_grid_desc(d));
  if (!out) return fail(NRR_ERR_INVALID_ARG, "null output");
  Geo g = grid_geo(d);
  if (g.npts > (int64_t)INT32_MAX)
    return fail(NRR_ERR_INVALID_ARG, "grid of %lld points: indices exceed int32",
                (long long)g.npts);
  for (int i2 = 0; i2 < g.s2; i2++)
    for (int i1 = 0; i1 < g.s1; i1++)
      for (int i0 = 0; i0 < g.s0; i0++) {
        int64_t p = flat(g, i0, i1, i2);
        int j0 = i0, j1 = i1, j2 = i2;
        if (g.coord != CARTESIAN) image_of(g, j0, j1, j2);
        out[p] = (int32_t)flat(g, j0, j1, j2);
      }
  return NRR_OK;
}

nrr_status nrr_create_grid(const nrr_grid_desc *d, void *stream,
                           nrr_grid **out) {
  if (!out) return fail(NRR_ERR_INVALID_ARG, "null output handle");
  *out = nullptr;
  TRY(check_grid_desc(d));
  Geo geo = grid_geo(d);
  if (geo.npts > (int64_t)1 << 31)
    return fail(NRR_ERR_INVALID_ARG, "grid of %lld points exceeds 2^31",
                (long long)geo.npts);
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  size_t need = footprint_bytes(geo), free_b = 0, total_b = 0;
  CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
  if (need + (size_t)(256u << 20) > free_b)
    return fail(NRR_ERR_OOM, "grid needs %zu bytes, %zu free", need, free_b);

  nrr_grid *g = new (std::nothrow) nrr_grid();
  if (!g) return fail(NRR_ERR_OOM, "host allocation failed");
  g->desc = *d;
  g->geo = geo;
  g->user_stream = static_cast<cudaStream_t>(stream);
  g->device = dev;
  nrr_status st = [&]() -> nrr_status {
    CUDA_TRY(cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking));
    CUDA_TRY(cudaEventCreateWithFlags(&g->order_ev, cudaEventDisableTiming));
    CUDA_TRY(cudaEventRecord(g->order_ev, g->user_stream));
    CUDA_TRY(cudaStreamWaitEvent(g->stream, g->order_ev, 0));
    const int64_t n = geo.npts;
    const int nc = geo.ncol, nco = ncoef(geo.ng);
    for (int c = 0; c < 2; c++) {
      TRY(dev_alloc(g, &g->f64.y[c], n));
      TRY(dev_alloc(g, &g->f64.s[c], n));
      TRY(dev_alloc(g, &g->f64.t[c], n));
      TRY(dev_alloc(g, &g->f64.a[c], n));
      TRY(dev_alloc(g, &g->f32.y[c], n));
      TRY(dev_alloc(g, &g->f32.s[c], n));
      TRY(dev_alloc(g, &g->f32.t[c], n));
      TRY(dev_alloc(g, &g->f32.a[c], n));
    }
    TRY(dev_alloc(g, &g->f64.alpha, n));
    TRY(dev_alloc(g, &g->f64.bc2, n));
    TRY(dev_alloc(g, &g->f32.alpha, n));
    TRY(dev_alloc(g, &g->f32.bc2, n));
    TRY(dev_alloc(g, &g->res64, n));
    TRY(dev_alloc(g, &g->u_save, n));
    TRY(dev_alloc(g, &g->acoef32, n));
    TRY(dev_alloc(g, &g->rhs32, n));
    TRY(dev_alloc(g, &g->fu32, n));
    TRY(dev_alloc(g, &g->h, 3 * (size_t)nc));
    TRY(dev_alloc(g, &g->gl, 2 * (size_t)nc));
    TRY(dev_alloc(g, &g->rad, nc));
    TRY(dev_alloc(g, &g->drdxx0, nc));
    TRY(dev_alloc(g, &g->jac, nc));
    TRY(dev_alloc(g, &g->dsmin, nc));
    TRY(dev_alloc(g, &g->c64.coef, (size_t)nco * nc));
    TRY(dev_alloc(g, &g->c64.somm, 4 * (size_t)nc));
    TRY(dev_alloc(g, &g->c64.c2inv, nc));
    TRY(dev_alloc(g, &g->c32.coef, (size_t)nco * nc));
    TRY(dev_alloc(g, &g->c32.somm, 4 * (size_t)nc));
    TRY(dev_alloc(g, &g->c32.c2inv, nc));
    TRY(dev_alloc(g, &g->scalars, 8));
    int nb = residual_blocks(geo, g->res_cfg);
    for (int k = 0; k < 2; k++) g->stage_cfg[k] = tuned_or_default(geo, k);
    TRY(dev_alloc(g, &g->partials, 2 * (size_t)nb + 64));
    TRY(dev_alloc(g, &g->flag, 4));
    CUDA_TRY(cudaMemsetAsync(g->flag, 0, 4 * sizeof(int), g->stream));
    CUDA_TRY(cudaMallocHost(&g->host_pinned, 8 * sizeof(double)));
    TRY(dev_alloc(g, reinterpret_cast<double **>(&g->ctl),
                  (sizeof(RelaxCtl) + 7) / 8));
    CUDA_TRY(cudaMallocHost(&g->ctl_host, sizeof(RelaxCtl)));
    // zero all state so unset regions are finite
    for (int c = 0; c < 2; c++) {
      double *f64s[4] = {g->f64.y[c], g->f64.s[c], g->f64.t[c], g->f64.a[c]};
      float *f32s[4] = {g->f32.y[c], g->f32.s[c], g->f32.t[c], g->f32.a[c]};
      for (int k = 0; k < 4; k++) {
        CUDA_TRY(cudaMemsetAsync(f64s[k], 0, n * sizeof(double), g->stream));
        CUDA_TRY(cudaMemsetAsync(f32s[k], 0, n * sizeof(float), g->stream));
      }
    }
    CUDA_TRY(cudaMemsetAsync(g->f64.alpha, 0, n * sizeof(double), g->stream));
    CUDA_TRY(cudaMemsetAsync(g->f64.bc2, 0, n * sizeof(double), g->stream));
    CUDA_TRY(cudaMemsetAsync(g->f32.alpha, 0, n * sizeof(float), g->stream));
    CUDA_TRY(cudaMemsetAsync(g->f32.bc2, 0, n * sizeof(float), g->stream));

    // FD weights, closed forms.
    int m = geo.ng;
    double w1[7] = {0}, w2[7] = {0};
    for (int k = 0; k <= m; k++) {
      w1[k] = k == 0 ? 0.0 : fd_first(m, k);
      w2[k] = fd_second(m, k);
    }
    if (geo.coord == CARTESIAN) {
      // Uniform spacing: dt from the smallest spacing, c = 1 when the
      // spacings agree (the wave speed follows the local spacing).
      double ds = fmin(geo.dxx[0], fmin(geo.dxx[1], geo.dxx[2]));
      g->dsmin_global = ds;
      CartCoef cc{};
      cc.cc = 0.0;
      cc.speed = 1.0;
      for (int dd = 0; dd < 3; dd++) {
        double inv = 1.0 / (geo.dxx[dd] * geo.dxx[dd]);
        cc.cc += w2[0] * inv;
        for (int k = 1; k <= m; k++) cc.a[dd][k - 1] = w2[k] * inv;
      }
      g->cart = cc;
      double host_s[1] = {ds};
      CUDA_TRY(cudaMemcpyAsync(g->scalars, host_s, sizeof(double),
                               cudaMemcpyHostToDevice, g->stream));
    } else {
      launch_column_geometry(geo, g->h, g->gl, g->rad, g->drdxx0, g->jac,
                             g->dsmin, g->stream);
      launch_min_interior(geo, g->dsmin, g->scalars, g->stream);
      launch_column_coefs(geo, g->h, g->gl, g->rad, g->drdxx0, g->dsmin,
                          g->scalars, w1, w2, g->c64, g->c32, g->stream);
      CUDA_TRY(cudaGetLastError());
      CUDA_TRY(cudaMemcpyAsync(g->host_pinned, g->scalars, sizeof(double),
                               cudaMemcpyDeviceToHost, g->stream));
      CUDA_TRY(cudaStreamSynchronize(g->stream));
      g->dsmin_global = g->host_pinned[0];
      if (!(g->dsmin_global > 0.0) || !std::isfinite(g->dsmin_global))
        return fail(NRR_ERR_INVALID_ARG, "degenerate grid spacing %g",
                    g->dsmin_global);
    }
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    return NRR_OK;
  }();
  if (st != NRR_OK) {
    std::string msg = g_last_error;
    nrr_destroy_grid(g);
    g_last_error = msg;
    return st;
  }
  *out = g;
  return NRR_OK;
}

nrr_status nrr_destroy_grid(nrr_grid *g) {
  if (!g) return NRR_OK;
  cudaSetDevice(g->device);
  if (g->stream) cudaStreamSynchronize(g->stream);
  for (auto &kv : g->graphs) cudaGraphExecDestroy(kv.second);
  for (void *p : g->allocs) {
    dbg_unregister(p);
    cudaFree(p);
  }
  if (g->host_pinned) cudaFreeHost(g->host_pinned);
  if (g->ctl_host) cudaFreeHost(g->ctl_host);
  if (g->order_ev) cudaEventDestroy(g->order_ev);
  if (g->stream) cudaStreamDestroy(g->stream);
  delete g;
  return NRR_OK;
}

nrr_status nrr_grid_dims(const nrr_grid *g, int s[3], int *ng,
                         int64_t *interior_points) {
  TRY(check_grid(g));
  if (s) {
    s[0] = g->geo.s0;
    s[1] = g->geo.s1;
    s[2] = g->geo.s2;
  }
  if (ng) *ng = g->geo.ng;
  if (interior_points)
    *interior_points = (int64_t)g->geo.n0 * g->geo.n1 * g->geo.n2;
  return NRR_OK;
}

nrr_status nrr_timestep(const nrr_grid *g, double cfl, double *dt,
                        double *eta_default) {
  TRY(check_grid(g));
  if (!(cfl > 0.0)) return fail(NRR_ERR_INVALID_ARG, "cfl must be positive");
  double d = cfl * g->dsmin_global;
  if (dt) *dt = d;
  if (eta_default) *eta_default = 2.0 * M_PI * cfl / (g->geo.n0 * d);
  return NRR_OK;
}

nrr_status nrr_set_punctures(nrr_grid *g, int n, const nrr_puncture *p) {
  TRY(check_grid(g));
  if (n < 1 || n > 8 || !p)
    return fail(NRR_ERR_INVALID_ARG, "need 1..8 punctures (got %d)", n);
  PunctureSet ps{};
  ps.n = n;
  for (int i = 0; i < n; i++) {
    if (!(p[i].m > 0.0) || !std::isfinite(p[i].m))
      return fail(NRR_ERR_INVALID_ARG, "puncture %d: mass must be positive", i);
    ps.p[i].m = p[i].m;
    for (int k = 0; k < 3; k++) {
      ps.p[i].x[k] = p[i].x[k];
      ps.p[i].P[k] = p[i].P[k];
      ps.p[i].S[k] = p[i].S[k];
      if (!std::isfinite(p[i].x[k]) || !std::isfinite(p[i].P[k]) ||
          !std::isfinite(p[i].S[k]))
        return fail(NRR_ERR_INVALID_ARG, "puncture %d: non-finite input", i);
    }
  }
  TRY(set_device(g));
  CUDA_TRY(cudaMemsetAsync(g->flag, 0, sizeof(int), g->stream));
  g_launches += 1;
  launch_source(g->geo, ps, g->dsmin, g->scalars, g->f64.alpha, g->f64.bc2,
                g->f32.alpha, g->f32.bc2, g->flag, g->stream);
  CUDA_TRY(cudaGetLastError());
  int bad = 0;
  CUDA_TRY(cudaMemcpyAsync(&bad, g->flag, sizeof(int), cudaMemcpyDeviceToHost,
                           g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  if (bad) {
    g->have_source = false;
    return fail(NRR_ERR_INVALID_ARG, "a puncture lies on a grid point");
  }
  g->have_source = true;
  g->punct = ps;
  return NRR_OK;
}

nrr_status nrr_set_speed_reference(nrr_grid *g, double ds_ref) {
  TRY(check_grid(g));
  if (!(ds_ref > 0.0) || !std::isfinite(ds_ref))
    return fail(NRR_ERR_INVALID_ARG, "ds_ref must be positive");
  TRY(set_device(g));
  const Geo &geo = g->geo;
  g->dsmin_global = ds_ref;
  CUDA_TRY(cudaMemcpyAsync(g->scalars, &g->dsmin_global, sizeof(double),
                           cudaMemcpyHostToDevice, g->stream));
  int m = geo.ng;
  double w1[7] = {0}, w2[7] = {0};
  for (int k = 0; k <= m; k++) {
    w1[k] = k == 0 ? 0.0 : fd_first(m, k);
    w2[k] = fd_second(m, k);
  }
  if (geo.coord == CARTESIAN) {
    const double ds = fmin(geo.dxx[0], fmin(geo.dxx[1], geo.dxx[2]));
    const double c = ds / ds_ref, c2 = c * c;
    CartCoef cc{};
    cc.speed = c;
    for (int dd = 0; dd < 3; dd++) {
      double inv = 1.0 / (geo.dxx[dd] * geo.dxx[dd]);
      cc.cc += c2 * w2[0] * inv;
      for (int k = 1; k <= m; k++) cc.a[dd][k - 1] = c2 * w2[k] * inv;
    }
    g->cart = cc;
  } else {
    launch_column_coefs(geo, g->h, g->gl, g->rad, g->drdxx0, g->dsmin,
                        g->scalars, w1, w2, g->c64, g->c32, g->stream);
    g_launches += 1;
  }
  if (g->have_source) {
    // c^2 beta with the new wave speed
    launch_source(geo, g->punct, g->dsmin, g->scalars, g->f64.alpha, g->f64.bc2,
                  g->f32.alpha, g->f32.bc2, g->flag, g->stream);
    g_launches += 1;
  }
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  // captured graphs hold the old coefficients (kernel parameters)
  for (auto &kv : g->graphs) cudaGraphExecDestroy(kv.second);
  g->graphs.clear();
  g->graph_kernels.clear();
  g->loop_kernels.clear();
  return NRR_OK;
}

nrr_status nrr_set_state(nrr_grid *g, const double *u, const double *v,
                         int on_device) {
  TRY(check_grid(g));
  if (!u) return fail(NRR_ERR_INVALID_ARG, "null u");
  TRY(set_device(g));
  size_t bytes = (size_t)g->geo.npts * sizeof(double);
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CUDA_TRY(cudaMemcpyAsync(g->f64.y[0], u, bytes, kind, g->stream));
  if (v)
    CUDA_TRY(cudaMemcpyAsync(g->f64.y[1], v, bytes, kind, g->stream));
  else
    CUDA_TRY(cudaMemsetAsync(g->f64.y[1], 0, bytes, g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  g->state_prec = 64;
  return NRR_OK;
}

nrr_status nrr_get_state(nrr_grid *g, double *u, double *v, int on_device) {
  TRY(check_grid(g));
  TRY(set_device(g));
  TRY(ensure_state(g, 64));
  size_t bytes = (size_t)g->geo.npts * sizeof(double);
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  for (int c = 0; c < 2; c++) launch_fill_ghosts<double>(g->geo, g->f64.y[c], g->stream);
  CUDA_TRY(cudaGetLastError());
  if (u) CUDA_TRY(cudaMemcpyAsync(u, g->f64.y[0], bytes, kind, g->stream));
  if (v) CUDA_TRY(cudaMemcpyAsync(v, g->f64.y[1], bytes, kind, g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  return NRR_OK;
}

nrr_status nrr_rhs(nrr_grid *g, int mode, double eta, const double *u,
                   const double *v, double *ku, double *kv) {
  TRY(check_grid(g));
  if (!u || !v || !ku || !kv) return fail(NRR_ERR_INVALID_ARG, "null pointer");
  if (!g->have_source) return fail(NRR_ERR_STATE, "punctures not set");
  if (mode != NRR_FP64 && mode != NRR_FP32)
    return fail(NRR_ERR_INVALID_ARG, "mode must be NRR_FP64 or NRR_FP32");
  TRY(set_device(g));
  int64_t n = g->geo.npts;
  if (mode == NRR_FP64) {
    StageArgs<double> a{};
    a.su = u; a.sv = v; a.ou = ku; a.ov = kv;
    a.alpha = g->f64.alpha; a.bc2 = g->f64.bc2; a.col = g->c64; a.cart = g->cart;
    a.eta = eta;
    CUDA_TRY(cudaMemsetAsync(ku, 0, n * sizeof(double), g->stream));
    CUDA_TRY(cudaMemsetAsync(kv, 0, n * sizeof(double), g->stream));
    launch_stage<double>(g->geo, STAGE_RAW, a, g->stage_cfg[0], g->stream);
  } else {
    // Round the inputs to FP32 in the grid's stage buffers, evaluate in
    // FP32, widen the result.
    TRY(ensure_state(g, 64));  // keep any FP32 state safe from the scratch use
    float *us = g->f32.s[0], *vs = g->f32.s[1], *ko = g->f32.t[0], *kw = g->f32.t[1];
    launch_convert(u, us, n, g->stream);
    launch_convert(v, vs, n, g->stream);
    CUDA_TRY(cudaMemsetAsync(ko, 0, n * sizeof(float), g->stream));
    CUDA_TRY(cudaMemsetAsync(kw, 0, n * sizeof(float), g->stream));
    StageArgs<float> a{};
    a.su = us; a.sv = vs; a.ou = ko; a.ov = kw;
    a.alpha = g->f32.alpha; a.bc2 = g->f32.bc2; a.col = g->c32; a.cart = g->cart;
    a.eta = (float)eta;
    launch_stage<float>(g->geo, STAGE_RAW, a, g->stage_cfg[1], g->stream);
    launch_convert(ko, ku, n, g->stream);
    launch_convert(kw, kv, n, g->stream);
  }
  launch_fill_ghosts<double>(g->geo, ku, g->stream);
  launch_fill_ghosts<double>(g->geo, kv, g->stream);
  CUDA_TRY(cudaGetLastError());
  return take_stage_error(g);
}

nrr_status nrr_step(nrr_grid *g, int mode, double dt, double eta,
                    int64_t steps) {
  TRY(check_grid(g));
  if (!g->have_source) return fail(NRR_ERR_STATE, "punctures not set");
  if (steps < 0 || !(dt > 0.0))
    return fail(NRR_ERR_INVALID_ARG, "need steps >= 0 and dt > 0");
  TRY(set_device(g));
  if (mode == NRR_FP32) {
    TRY(ensure_state(g, 32));
    launch_rk4_steps<float>(g, g->f32, g->c32, dt, eta, steps);
  } else if (mode == NRR_FP64) {
    TRY(ensure_state(g, 64));
    launch_rk4_steps<double>(g, g->f64, g->c64, dt, eta, steps);
  } else {
    return fail(NRR_ERR_INVALID_ARG, "mode must be NRR_FP64 or NRR_FP32");
  }
  CUDA_TRY(cudaGetLastError());
  return take_stage_error(g);
}

nrr_status nrr_profile_stages(nrr_grid *g, int mode, double dt, double eta,
                              int64_t steps, double *ms_per_launch) {
  TRY(check_grid(g));
  if (!g->have_source) return fail(NRR_ERR_STATE, "punctures not set");
  if (steps < 1 || !(dt > 0.0) || !ms_per_launch)
    return fail(NRR_ERR_INVALID_ARG, "need steps >= 1, dt > 0, output");
  if (mode != NRR_FP64 && mode != NRR_FP32)
    return fail(NRR_ERR_INVALID_ARG, "mode must be NRR_FP64 or NRR_FP32");
  TRY(set_device(g));
  TRY(ensure_state(g, mode == NRR_FP32 ? 32 : 64));
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  CUDA_TRY(cudaEventRecord(e0, g->stream));
  if (mode == NRR_FP32)
    launch_rk4_steps<float>(g, g->f32, g->c32, dt, eta, steps);
  else
    launch_rk4_steps<double>(g, g->f64, g->c64, dt, eta, steps);
  CUDA_TRY(cudaEventRecord(e1, g->stream));
  CUDA_TRY(cudaEventSynchronize(e1));
  float ms = 0.f;
  CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms_per_launch = (double)ms / (4.0 * (double)steps);
  CUDA_TRY(cudaGetLastError());
  return take_stage_error(g);
}

nrr_status nrr_set_launch(nrr_grid *g, int mode, int variant, int zc, int block) {
  TRY(check_grid(g));
  if (block != 0 && block != 32 && block != 64 && block != 128 && block != 256)
    return fail(NRR_ERR_INVALID_ARG, "block must be 0 (keep), 32, 64, 128 or 256");
  if (mode != NRR_FP64 && mode != NRR_FP32)
    return fail(NRR_ERR_INVALID_ARG, "mode must be NRR_FP64 or NRR_FP32");
  if (variant < 0 || variant > 6)
    return fail(NRR_ERR_INVALID_ARG,
                "variant must be 0 (column), 1 (tiled), 2 (persistent column), "
                "3 (tensor-copy tiled), 4 (multi-stage), 5 (multi-stage "
                "tensor-copy) or 6 (two stages per launch)");
  if ((variant == 0 && zc != 1 && zc != 2 && zc != 4) ||
      ((variant == 1 || variant == 3 || variant == 5) && zc != 2 && zc != 4 &&
       zc != 8 && zc != 16) ||
      ((variant == 2 || variant == 4 || variant == 6) && zc != 1))
    return fail(NRR_ERR_INVALID_ARG,
                "zc must be 1, 2 or 4 (column), 2, 4, 8 or 16 (tiled, tensor-copy), "
                "1 (persistent, multi-stage, two-stage)");
  if (variant == 6 && (mode != NRR_FP32 || !stage2_ok(g->geo)))
    return fail(NRR_ERR_INVALID_ARG,
                "variant 6 runs FP32 stages of SinhSymTP grids of FD order 8 with "
                "n0 %% 32 == 0, n1 %% 4 == 0 and n2 <= 16");
  if (g->geo.coord == SINHCYLINDRICAL && variant != 0)
    return fail(NRR_ERR_INVALID_ARG,
                "SinhCylindrical grids run the column kernel (variant 0) only");
  g->stage_cfg[mode == NRR_FP32].variant = variant;
  g->stage_cfg[mode == NRR_FP32].zc = zc;
  if (block) g->stage_cfg[mode == NRR_FP32].block = block;
  for (auto &kv : g->graphs) cudaGraphExecDestroy(kv.second);
  g->graphs.clear();
  g->graph_kernels.clear();
  g->loop_kernels.clear();
  return NRR_OK;
}

nrr_status nrr_get_launch(const nrr_grid *g, int mode, int *variant, int *zc,
                          int *block) {
  TRY(check_grid(g));
  if (mode != NRR_FP64 && mode != NRR_FP32)
    return fail(NRR_ERR_INVALID_ARG, "mode must be NRR_FP64 or NRR_FP32");
  const LaunchCfg &c = g->stage_cfg[mode == NRR_FP32];
  if (variant) *variant = c.variant;
  if (zc) *zc = c.zc;
  if (block) *block = c.block;
  return NRR_OK;
}

nrr_status nrr_set_pdl(nrr_grid *g, int on) {
  TRY(check_grid(g));
  if (on != 0 && on != 1) return fail(NRR_ERR_INVALID_ARG, "on must be 0 or 1");
  g->stage_cfg[0].pdl = on;
  g->stage_cfg[1].pdl = on;
  for (auto &kv : g->graphs) cudaGraphExecDestroy(kv.second);
  g->graphs.clear();
  g->graph_kernels.clear();
  g->loop_kernels.clear();
  return NRR_OK;
}

nrr_status nrr_set_device_loop(nrr_grid *g, int on) {
  TRY(check_grid(g));
  if (on != 0 && on != 1) return fail(NRR_ERR_INVALID_ARG, "on must be 0 or 1");
  g->device_loop = on;
  return NRR_OK;
}

nrr_status nrr_autotune_save(const char *path) {
  if (!path) return fail(NRR_ERR_INVALID_ARG, "null path");
  std::map<TuneKey, LaunchCfg> copy;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    copy = g_tuned;
  }
  FILE *f = fopen(path, "w");
  if (!f) return fail(NRR_ERR_STATE, "cannot write %s", path);
  fprintf(f, "{\"nrr_autotune\": 1, \"entries\": [");
  bool first = true;
  for (const auto &kv : copy) {
    const TuneKey &k = kv.first;
    const LaunchCfg &c = kv.second;
    fprintf(f,
            "%s\n  {\"coord\": %d, \"n\": [%d, %d, %d], \"ng\": %d, "
            "\"fp32\": %d, \"variant\": %d, \"zc\": %d, \"block\": %d, "
            "\"pdl\": %d}",
            first ? "" : ",", k.coord, k.n0, k.n1, k.n2, k.ng, k.prec, c.variant,
            c.zc, c.block, c.pdl);
    first = false;
  }
  fprintf(f, "\n]}\n");
  const bool ok = fclose(f) == 0;
  return ok ? NRR_OK : fail(NRR_ERR_STATE, "cannot write %s", path);
}

nrr_status nrr_autotune_load(const char *path) {
  if (!path) return fail(NRR_ERR_INVALID_ARG, "null path");
  FILE *f = fopen(path, "r");
  if (!f) return fail(NRR_ERR_INVALID_ARG, "cannot read %s", path);
  std::string text;
  char buf[4096];
  size_t got;
  while ((got = fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, got);
  fclose(f);
  if (text.find("\"nrr_autotune\"") == std::string::npos)
    return fail(NRR_ERR_INVALID_ARG, "%s is not an autotuner file", path);
  // entries are the objects after the "entries" key
  size_t pos = text.find("\"entries\"");
  if (pos == std::string::npos) return fail(NRR_ERR_INVALID_ARG, "no entries in %s", path);
  std::map<TuneKey, LaunchCfg> add;
  while ((pos = text.find('{', pos + 1)) != std::string::npos) {
    const size_t end = text.find('}', pos);
    if (end == std::string::npos) return fail(NRR_ERR_INVALID_ARG, "unterminated entry");
    const char *b = text.c_str() + pos, *e = text.c_str() + end;
    TuneKey k{};
    LaunchCfg c{};
    int n[3];
    if (!json_int(b, e, "coord", &k.coord) || !json_int3(b, e, "n", n) ||
        !json_int(b, e, "ng", &k.ng) || !json_int(b, e, "fp32", &k.prec) ||
        !json_int(b, e, "variant", &c.variant) || !json_int(b, e, "zc", &c.zc) ||
        !json_int(b, e, "block", &c.block) || !json_int(b, e, "pdl", &c.pdl))
      return fail(NRR_ERR_INVALID_ARG, "incomplete entry at byte %zu of %s", pos, path);
    k.n0 = n[0];
    k.n1 = n[1];
    k.n2 = n[2];
    if (k.coord < NRR_SINHSYMTP || k.coord > NRR_SINHSPHERICAL || k.ng < 1 ||
        k.ng > 6 || (k.prec != 0 && k.prec != 1) || k.n0 < 1 || k.n1 < 1 ||
        k.n2 < 1 || !valid_shape(c))
      return fail(NRR_ERR_INVALID_ARG, "invalid entry at byte %zu of %s", pos, path);
    add[k] = c;
    pos = end;
  }
  std::lock_guard<std::mutex> lock(g_tune_mu);
  for (const auto &kv : add) g_tuned[kv.first] = kv.second;
  return NRR_OK;
}

nrr_status nrr_autotune_clear(void) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tuned.clear();
  return NRR_OK;
}

nrr_status nrr_autotune(nrr_grid *g, int mode, int64_t trial_steps,
                        int *best_variant, int *best_zc,
                        double *best_ms_per_launch) {
  TRY(check_grid(g));
  if (!g->have_source) return fail(NRR_ERR_STATE, "punctures not set");
  if (mode != NRR_FP64 && mode != NRR_FP32)
    return fail(NRR_ERR_INVALID_ARG, "mode must be NRR_FP64 or NRR_FP32");
  if (trial_steps < 1) return fail(NRR_ERR_INVALID_ARG, "trial_steps >= 1");
  TRY(set_device(g));
  const int prec = mode == NRR_FP32 ? 32 : 64;
  // The state's own precision: trials in the other precision run on a
  // converted copy and leave the state's buffers untouched.
  const int prec0 = g->state_prec;
  TRY(ensure_state(g, prec));
  double dt = 0.0, eta = 0.0;
  TRY(nrr_timestep(g, 0.5, &dt, &eta));
  // Keep the state: trials run from it and it is restored afterwards.
  size_t bytes = (size_t)g->geo.npts * (prec == 32 ? sizeof(float) : sizeof(double));
  void *save_u = prec == 32 ? (void *)g->acoef32 : (void *)g->res64;
  void *save_v = prec == 32 ? (void *)g->rhs32 : (void *)g->u_save;
  void *yu = prec == 32 ? (void *)g->f32.y[0] : (void *)g->f64.y[0];
  void *yv = prec == 32 ? (void *)g->f32.y[1] : (void *)g->f64.y[1];
  CUDA_TRY(cudaMemcpyAsync(save_u, yu, bytes, cudaMemcpyDeviceToDevice, g->stream));
  CUDA_TRY(cudaMemcpyAsync(save_v, yv, bytes, cudaMemcpyDeviceToDevice, g->stream));
  LaunchCfg &cfg = g->stage_cfg[prec == 32];
  const LaunchCfg keep = cfg;
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  LaunchCfg best = keep;
  double best_ms = 1e30;
  // (variant 6, two stages per launch, measured 4-7x slower than these on
  // every eligible grid, is left to nrr_set_launch)
  const LaunchCfg cands[24] = {{128, 1, 0},  {32, 1, 0},   {64, 1, 0},   {256, 1, 0},  {128, 2, 0},
                               {64, 2, 0},   {128, 4, 0},  {128, 2, 1},  {128, 4, 1},
                               {128, 8, 1},  {128, 16, 1}, {128, 1, 2},  {128, 2, 3},
                               {128, 4, 3},  {128, 8, 3},  {128, 16, 3}, {256, 2, 3},
                               {256, 4, 3},  {256, 8, 3},  {256, 16, 3}, {128, 1, 4},
                               {128, 4, 5},  {128, 8, 5},  {128, 16, 5}};
  for (const LaunchCfg &cand0 : cands) {
    // SinhCylindrical grids have the column kernel only
    if (g->geo.coord == SINHCYLINDRICAL && cand0.variant != 0) continue;
    LaunchCfg cand = cand0;
    cand.pdl = keep.pdl;
    cfg = cand;
    for (int rep = 0; rep < 2; rep++) {  // first repetition warms up
      CUDA_TRY(cudaEventRecord(e0, g->stream));
      if (prec == 32)
        launch_rk4_steps<float>(g, g->f32, g->c32, dt, eta, trial_steps);
      else
        launch_rk4_steps<double>(g, g->f64, g->c64, dt, eta, trial_steps);
      // a shape this grid cannot launch is skipped, not chosen
      if (cudaGetLastError() != cudaSuccess) break;
      CUDA_TRY(cudaEventRecord(e1, g->stream));
      CUDA_TRY(cudaEventSynchronize(e1));
      float ms = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
      // a shape whose bounded waits expired is skipped (and the flag cleared)
      if (take_stage_error(g) != NRR_OK) break;
      double per = ms / (4.0 * (double)trial_steps);
      if (rep == 1 && per < best_ms) {
        best_ms = per;
        best = cand;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cfg = best;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned[tune_key(g->geo, prec == 32)] = cfg;
  }
  CUDA_TRY(cudaMemcpyAsync(yu, save_u, bytes, cudaMemcpyDeviceToDevice, g->stream));
  CUDA_TRY(cudaMemcpyAsync(yv, save_v, bytes, cudaMemcpyDeviceToDevice, g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  g->state_prec = prec0;
  // cached relaxation graphs hold the old shape
  for (auto &kv : g->graphs) cudaGraphExecDestroy(kv.second);
  g->graphs.clear();
  g->graph_kernels.clear();
  g->loop_kernels.clear();
  if (best_variant) *best_variant = best.variant;
  if (best_zc) *best_zc = best.zc;
  if (best_ms_per_launch) *best_ms_per_launch = best_ms;
  return NRR_OK;
}

nrr_status nrr_residual(nrr_grid *g, double r_int, double *norm_out,
                        double *h_out, int h_on_device) {
  TRY(check_grid(g));
  if (!g->have_source) return fail(NRR_ERR_STATE, "punctures not set");
  TRY(set_device(g));
  TRY(ensure_state(g, 64));
  double *hdev = nullptr;
  size_t bytes = (size_t)g->geo.npts * sizeof(double);
  if (h_out) {
    hdev = h_on_device ? h_out : g->res64;
    CUDA_TRY(cudaMemsetAsync(hdev, 0, bytes, g->stream));
  }
  launch_norm<double>(g, g->f64, g->c64, r_int, hdev);
  CUDA_TRY(cudaGetLastError());
  if (h_out && !h_on_device)
    CUDA_TRY(cudaMemcpyAsync(h_out, hdev, bytes, cudaMemcpyDeviceToHost, g->stream));
  double nrm = 0.0;
  TRY(sync_read_norm(g, &nrm));
  if (norm_out) *norm_out = nrm;
  return NRR_OK;
}

nrr_status nrr_relax(nrr_grid *g, const nrr_relax_opts *o,
                     nrr_relax_result *r) {
  double t_start = now_s();
  TRY(check_grid(g));
  if (!o) return fail(NRR_ERR_INVALID_ARG, "null opts");
  if (!g->have_source) return fail(NRR_ERR_STATE, "punctures not set");
  if (o->mode != NRR_FP64 && o->mode != NRR_FP32 && o->mode != NRR_FP32_DC)
    return fail(NRR_ERR_INVALID_ARG, "unknown mode %d", o->mode);
  if (!(o->tol > 0.0) || o->check_every < 1 || o->max_iters < 0 ||
      !(o->cfl > 0.0) || !(o->r_int > 0.0))
    return fail(NRR_ERR_INVALID_ARG, "invalid relax options");
  if (o->inner_steps < 0 || o->max_outer < 0)
    return fail(NRR_ERR_INVALID_ARG, "inner_steps and max_outer must be >= 0");
  TRY(set_device(g));
  double dt = 0.0, eta_def = 0.0;
  TRY(nrr_timestep(g, o->cfl, &dt, &eta_def));
  double eta = o->eta > 0.0 ? o->eta : eta_def;
  size_t bytes = (size_t)g->geo.npts * sizeof(double);
  switch (o->initial) {
    case NRR_INIT_ZERO:
      for (int c = 0; c < 2; c++)
        CUDA_TRY(cudaMemsetAsync(g->f64.y[c], 0, bytes, g->stream));
      g->state_prec = 64;
      break;
    case NRR_INIT_CURRENT:
      break;
    case NRR_INIT_HOST:
    case NRR_INIT_DEVICE:
      if (!o->u0) return fail(NRR_ERR_INVALID_ARG, "u0 required");
      CUDA_TRY(cudaMemcpyAsync(g->f64.y[0], o->u0, bytes,
                               o->initial == NRR_INIT_HOST ? cudaMemcpyHostToDevice
                                                           : cudaMemcpyDeviceToDevice,
                               g->stream));
      // v = eta u: the steady-state relation of the relaxation system.
      CUDA_TRY(cudaMemcpyAsync(g->f64.y[1], g->f64.y[0], bytes,
                               cudaMemcpyDeviceToDevice, g->stream));
      launch_scale(g->f64.y[1], eta, g->geo.npts, g->stream);
      g->state_prec = 64;
      break;
    default:
      return fail(NRR_ERR_INVALID_ARG, "unknown initial mode %d", o->initial);
  }
  nrr_relax_result res{};
  nrr_status status;
  double nrm = 0.0;
  int64_t it = 0;
  if (o->mode == NRR_FP32_DC) {
    TRY(relax_defect_correction(g, o, dt, eta, t_start, &res));
    status = (nrr_status)res.status;
    nrm = res.final_norm;
    it = res.iters;
  } else {
    int prec = o->mode == NRR_FP32 ? 32 : 64;
    TRY(ensure_state(g, prec));
    bool timed_out = false;
    int64_t it0 = 0;
    if (g->device_loop) {
      // whole chunks with the stop test on the device; relax_chunks below
      // finishes a shorter last chunk, if max_iters leaves one
      int64_t chunks = 0;
      TRY(relax_device_loop(g, o->mode, o->check_every, dt, eta, o->tol,
                            o->r_int, o->max_iters / o->check_every,
                            o->timeout_ms, t_start, &chunks, &nrm, &timed_out));
      it0 = chunks * o->check_every;
    } else {
      if (prec == 32)
        launch_norm<float>(g, g->f32, g->c32, o->r_int, nullptr);
      else
        launch_norm<double>(g, g->f64, g->c64, o->r_int, nullptr);
      CUDA_TRY(cudaGetLastError());
      TRY(sync_read_norm(g, &nrm));
    }
    if (timed_out) {
      status = NRR_ERR_TIMEOUT;
    } else {
      TRY(relax_chunks(g, o->mode, dt, eta, o->tol, o->r_int, o->check_every,
                       o->max_iters - it0, t_start, o->timeout_ms, &it, &nrm,
                       &status));
    }
    it += it0;
    res.iters = it;
    res.outer_iters = 0;
    res.final_norm = nrm;
    res.status = status;
  }

  res.seconds = now_s() - t_start;
  {
    // a stage kernel whose bounded wait for its tensor copies expired
    int stage_err = 0;
    CUDA_TRY(cudaMemcpyAsync(&stage_err, g->flag + 2, sizeof(int),
                             cudaMemcpyDeviceToHost, g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    if (stage_err) {
      CUDA_TRY(cudaMemsetAsync(g->flag + 2, 0, sizeof(int), g->stream));
      res.status = status = NRR_ERR_TIMEOUT;
    }
  }
  if (r) *r = res;
  if (status == NRR_ERR_NOT_CONVERGED)
    return fail(status, "not converged after %lld steps (norm %.3e)",
                (long long)it, nrm);
  if (status == NRR_ERR_DIVERGED)
    return fail(status, "residual norm not finite after %lld steps",
                (long long)it);
  if (status == NRR_ERR_TIMEOUT)
    return fail(status, "timeout after %lld steps (norm %.3e)", (long long)it,
                nrm);
  return NRR_OK;
}

}  // extern "C"
