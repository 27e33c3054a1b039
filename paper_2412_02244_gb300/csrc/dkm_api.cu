// dkm_api.cu -- the extern "C" boundary of libdkm (declared in include/dkm.h).
//
// Host code only: argument checks, the device arena of a context, the grid
// planner (the memory-tunable index of Section V-A), and the Lloyd loop of
// Algorithm 1 captured once per (context, max_iter) as a CUDA graph.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "dkm_host.h"

using namespace dkm;

namespace {

thread_local std::string g_last_error;

dkm_status fail(dkm_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

#define DKM_CK(call)                                                                     \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      return fail(e_ == cudaErrorMemoryAllocation ? DKM_ENOMEM : DKM_ECUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                    \
    }                                                                                    \
  } while (0)

#define DKM_TRY(expr)                  \
  do {                                 \
    dkm_status s_ = (expr);            \
    if (s_ != DKM_OK) return s_;       \
  } while (0)

constexpr size_t kDefaultBudget = size_t(64) << 20;
constexpr int64_t kMaxPoints = (int64_t(1) << 31) - kBlockPts;

// true for memory a kernel may dereference directly (device or managed)
bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

dkm_options resolve(const dkm_options* o) {
  dkm_options r;
  dkm_default_options(&r);
  if (o) {
    r = *o;
    if (r.mem_budget_bytes == 0) r.mem_budget_bytes = kDefaultBudget;
    if (!(r.cells_per_centroid > 0.f)) r.cells_per_centroid = 1.0f;
  }
  return r;
}

// bytes of the per-iteration centroid index for a grid of `cells`
size_t index_bytes_for(int64_t cells, int k, int cap) {
  return size_t(2) * cells * (sizeof(int) + size_t(cap) * sizeof(float4)) +
         size_t(2) * k * sizeof(float4) + 2 * sizeof(int);
}

// Plan the grid; *max_cells = the cell count any point set of this (n, k,
// budget) can need, which sizes the arena.
dkm_status plan_grid(int64_t n, int d, int k, const float* lo, const float* hi,
                     const dkm_options& o, dkm_plan_info* out, int64_t* max_cells) {
  const int cap = kBucketCap;
  const size_t per_cell = size_t(2) * (sizeof(int) + size_t(cap) * sizeof(float4));
  const size_t fixed = index_bytes_for(0, k, cap);
  if (o.mem_budget_bytes < fixed + per_cell)
    return fail(DKM_ENOMEM, "memory budget %zu B cannot hold the centroid index of k=%d (needs >= %zu B)",
                o.mem_budget_bytes, k, fixed + per_cell);
  int64_t budget_cells = (int64_t)((o.mem_budget_bytes - fixed) / per_cell);
  int64_t target = (int64_t)std::ceil((double)o.cells_per_centroid * (double)k);
  if (target < 1) target = 1;
  if (target > budget_cells) target = budget_cells;
  if (target > (int64_t(1) << 28)) target = int64_t(1) << 28;
  double E[3] = {0, 0, 0};
  int deff = 0;
  double vol = 1.0;
  for (int a = 0; a < d; ++a) {
    E[a] = std::max(0.0, (double)hi[a] - (double)lo[a]);
    if (E[a] > 0) {
      ++deff;
      vol *= E[a];
    }
  }
  double s = 1.0;
  int64_t dims[3] = {1, 1, 1};
  if (deff > 0) {
    s = std::pow(vol / (double)target, 1.0 / deff);
    if (!(s > 0)) s = 1e-30;
    for (int guard = 0; guard < 100000; ++guard) {
      int64_t cells = 1;
      for (int a = 0; a < d; ++a) {
        double q = std::ceil(E[a] / s);
        dims[a] = q < 1 ? 1 : (q > 1e6 ? (int64_t)1e6 : (int64_t)q);
        cells *= dims[a];
      }
      if (cells <= target) break;
      s *= 1.02;
    }
  }
  memset(out, 0, sizeof(*out));
  int64_t cells = 1;
  for (int a = 0; a < 3; ++a) {
    out->dims[a] = (int)dims[a];
    out->origin[a] = a < d ? lo[a] : 0.f;
    cells *= dims[a];
  }
  out->cell = (float)s;
  out->bucket_cap = cap;
  out->cells = cells;
  out->index_bytes = index_bytes_for(cells, k, cap);
  *max_cells = target;
  (void)n;
  return DKM_OK;
}

struct Layout {
  size_t off = 0;
  template <class T>
  size_t take(size_t count) {
    size_t o = off;
    off = align_up(off + count * sizeof(T), 256);
    return o;
  }
};

// Offsets of every buffer in the arena, shared by plan and create.
struct ArenaPlan {
  size_t xs, ys, zs, keys0, keys1, vals0, vals1, rs_counts, rs_totals, tbox, tiles, n_tiles, wcnt,
      wbase, level_hist, lab, cw, acc, slots, st, gcnt0, gcnt1, gbkt0, gbkt1, ovf0, ovf1, ovf_cnt,
      tlist, tcnt, cstage, cstage2, kstage, total;
};

int64_t windows_of(int64_t n) { return (n + kTilePts - 1) / kTilePts; }
// Cube cuts add at most one tile per cube, and the tiling level is chosen so
// that the cubes number at most an eighth of the windows.
int64_t tiles_max_of(int64_t n) { return windows_of(n) + windows_of(n) / 8 + 2; }

ArenaPlan arena_plan(int64_t n, int d, int k, int64_t max_cells, int cap) {
  ArenaPlan P;
  Layout L;
  const int64_t nb = (n + kBlockPts - 1) / kBlockPts;
  const int64_t n_pad = nb * kBlockPts;
  const int64_t nw = windows_of(n), tm = tiles_max_of(n);
  P.xs = L.take<float>(n_pad);
  P.ys = L.take<float>(n_pad);
  P.zs = L.take<float>(d == 3 ? n_pad : 1);
  P.keys0 = L.take<uint32_t>(n);
  P.keys1 = L.take<uint32_t>(n);
  P.vals0 = L.take<uint32_t>(n);
  P.vals1 = L.take<uint32_t>(n);
  P.rs_counts = L.take<uint32_t>(256 * radix_sort_nb(n));
  P.rs_totals = L.take<uint32_t>(256);
  P.tbox = L.take<float4>(2 * tm);
  P.tiles = L.take<int2>(tm);
  P.n_tiles = L.take<int>(1);
  P.wcnt = L.take<int>(nw);
  P.wbase = L.take<int>(nw);
  P.level_hist = L.take<unsigned long long>(kMaxLevels + 1);
  P.lab = L.take<int32_t>(n_pad);
  P.cw = L.take<float4>(k);
  P.acc = L.take<Acc>(k);
  P.slots = L.take<Slot>(kSlots);
  P.st = L.take<DevState>(1);
  P.gcnt0 = L.take<int>(max_cells);
  P.gcnt1 = L.take<int>(max_cells);
  P.gbkt0 = L.take<float4>(max_cells * cap);
  P.gbkt1 = L.take<float4>(max_cells * cap);
  P.ovf0 = L.take<float4>(k);
  P.ovf1 = L.take<float4>(k);
  P.ovf_cnt = L.take<int>(2);
  P.tlist = L.take<int>(tm * kTileCap);
  P.tcnt = L.take<int>(tm);
  P.cstage = L.take<float>((size_t)k * d);
  P.cstage2 = L.take<float>((size_t)k * d);
  P.kstage = L.take<int32_t>(k);
  P.total = L.off;
  return P;
}

IterArgs iter_args(const dkm_ctx* c, int track_changes, int early_stop) {
  IterArgs A;
  memset(&A, 0, sizeof(A));
  A.n = c->n;
  A.k = c->k;
  A.n_windows = c->n_windows;
  A.tiles_max = c->tiles_max;
  A.n_tiles = c->n_tiles_dev;
  A.tiles = c->tiles;
  A.xs = c->xs;
  A.ys = c->ys;
  A.zs = c->zs;
  A.tbox = c->tbox;
  A.lab = c->lab;
  A.cw = c->cw;
  A.acc = c->acc;
  A.slots = c->slots;
  A.st = c->st;
  A.grid = c->grid;
  for (int p = 0; p < 2; ++p) {
    A.gcnt[p] = c->gcnt[p];
    A.gbkt[p] = c->gbkt[p];
    A.ovf[p] = c->ovf[p];
  }
  A.ovf_cnt = c->ovf_cnt;
  A.tlist = c->tlist;
  A.tcnt = c->tcnt;
  A.sse_hist = c->sse_hist;
  A.chg_hist = c->chg_hist;
  A.track_changes = track_changes;
  A.early_stop = early_stop;
  A.row_filter_min = c->row_filter_min;
  return A;
}

// Tuning knob, read once per context: DKM_ROW_FILTER_MIN (default 48).
int env_int(const char* name, int def) {
  const char* v = getenv(name);
  if (!v || !*v) return def;
  char* end = nullptr;
  long x = strtol(v, &end, 10);
  return (end && *end == 0) ? (int)x : def;
}

dkm_status check_ctx(const dkm_ctx* c) {
  if (!c) return fail(DKM_EINVAL, "null context");
  if (!c->ready) return fail(DKM_EINVAL, "context has no valid point index (a dkm_setup failed)");
  return DKM_OK;
}

dkm_status read_state(dkm_ctx* c, DevState* h) {
  DKM_CK(cudaMemcpyAsync(h, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
  DKM_CK(cudaStreamSynchronize(c->stream));
  return DKM_OK;
}

// Copy a k x d centroid array (host or device) into the context's staging.
dkm_status stage_centroids(dkm_ctx* c, const float* C) {
  size_t bytes = (size_t)c->k * c->d * sizeof(float);
  DKM_CK(cudaMemcpyAsync(c->cstage, C, bytes,
                         is_device_ptr(C) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                         c->stream));
  return DKM_OK;
}

dkm_status ensure_lstage(dkm_ctx* c) {
  if (!c->lstage) DKM_CK(cudaMalloc(&c->lstage, (size_t)c->n * sizeof(int32_t)));
  return DKM_OK;
}

// centroid bbox of the staged centroids (for the fixed-point scale) + check
dkm_status centroid_box(dkm_ctx* c, bool check) {
  DKM_CK(launch_bbox(c->cstage, c->k, c->d, c->st, 1, c->d, c->stream));
  if (check) {
    DevState h;
    DKM_TRY(read_state(c, &h));
    if (h.bad) return fail(DKM_EINVAL, "centroids contain a non-finite or |x| > 1e18 coordinate");
  }
  return DKM_OK;
}

dkm_status zero_run_buffers(dkm_ctx* c, bool labels_to_minus_one) {
  DKM_CK(launch_reset_run(c->st, c->stream));
  DKM_CK(cudaMemsetAsync(c->acc, 0, (size_t)c->k * sizeof(Acc), c->stream));
  DKM_CK(cudaMemsetAsync(c->slots, 0, (size_t)kSlots * sizeof(Slot), c->stream));
  DKM_CK(cudaMemsetAsync(c->gcnt[0], 0, (size_t)c->max_cells * sizeof(int), c->stream));
  DKM_CK(cudaMemsetAsync(c->gcnt[1], 0, (size_t)c->max_cells * sizeof(int), c->stream));
  DKM_CK(cudaMemsetAsync(c->ovf_cnt, 0, 2 * sizeof(int), c->stream));
  if (labels_to_minus_one)
    DKM_CK(cudaMemsetAsync(c->lab, 0xff, (size_t)c->n_pad * sizeof(int32_t), c->stream));
  return DKM_OK;
}

dkm_status ensure_hist(dkm_ctx* c, int iters) {
  if (iters <= c->hist_cap) return DKM_OK;
  if (c->sse_hist) cudaFree(c->sse_hist);
  if (c->chg_hist) cudaFree(c->chg_hist);
  c->sse_hist = nullptr;
  c->chg_hist = nullptr;
  c->hist_cap = 0;
  int cap = iters < 64 ? 64 : iters;
  DKM_CK(cudaMalloc(&c->sse_hist, (size_t)cap * sizeof(double)));
  DKM_CK(cudaMalloc(&c->chg_hist, (size_t)cap * sizeof(unsigned long long)));
  c->hist_cap = cap;
  if (c->gexec) {   // the cached graph holds the old pointers
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    c->g_iters = -1;
  }
  return DKM_OK;
}

void destroy_graph(dkm_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
  c->g_iters = -1;
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  c->ev.clear();
}

float ev_ms(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
    cudaGetLastError();
    return 0.f;
  }
  return ms;
}

// One labelling pass against the staged centroids (used by dkm_assign and
// by dkm_run with max_iter = 0).  Leaves the sums in acc.
dkm_status one_pass(dkm_ctx* c, bool track_changes) {
  const int brute = c->opts.algo == DKM_ALGO_BRUTE;
  DKM_TRY(zero_run_buffers(c, false));
  IterArgs A = iter_args(c, track_changes ? 1 : 0, 0);
  DKM_CK(launch_centroids(A, 0, -1, c->d, c->cstage, !brute, 0, nullptr, c->stream));
  if (!brute) DKM_CK(launch_search(A, 0, c->d, c->stream));
  DKM_CK(launch_assign(A, c->d, brute, c->stream));
  DKM_CK(launch_collect(A, -1, c->stream));
  return DKM_OK;
}

// labels (sorted, device) -> caller array in original order
dkm_status export_labels(dkm_ctx* c, int32_t* labels, bool do_sse) {
  IterArgs A = iter_args(c, 0, 0);
  int32_t* dst = nullptr;
  bool host = labels && !is_device_ptr(labels);
  if (labels) {
    if (host) DKM_TRY(ensure_lstage(c));
    dst = host ? c->lstage : labels;
  }
  if (!dst && !do_sse) return DKM_OK;
  DKM_CK(launch_finalize(A, c->d, c->perm, dst, do_sse ? 1 : 0, c->stream));
  if (host)
    DKM_CK(cudaMemcpyAsync(labels, c->lstage, (size_t)c->n * sizeof(int32_t),
                           cudaMemcpyDeviceToHost, c->stream));
  return DKM_OK;
}

dkm_status export_centroids(dkm_ctx* c, float* out) {
  if (!out) return DKM_OK;
  bool host = !is_device_ptr(out);
  float* dst = host ? c->cstage2 : out;
  DKM_CK(launch_export(c->cw, c->k, c->d, dst, c->stream));
  if (host)
    DKM_CK(cudaMemcpyAsync(out, c->cstage2, (size_t)c->k * c->d * sizeof(float),
                           cudaMemcpyDeviceToHost, c->stream));
  return DKM_OK;
}

dkm_status check_state(const DevState& h) {
  if (h.err & kErrNoCentroid) return fail(DKM_EINTERNAL, "candidate search found no centroid");
  if (h.err & kErrEmptyList) return fail(DKM_EINTERNAL, "a tile received an empty candidate list");
  return DKM_OK;
}

dkm_status build_run_graph(dkm_ctx* c, int iters, int early, int profile) {
  destroy_graph(c);
  const int brute = c->opts.algo == DKM_ALGO_BRUTE;
  IterArgs A = iter_args(c, early, early);
  if (profile) {
    c->ev.resize((size_t)4 * iters);
    for (auto& e : c->ev) DKM_CK(cudaEventCreate(&e));
  }
  cudaGraph_t g = nullptr;
  DKM_CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  dkm_status st = DKM_OK;
  cudaError_t e = cudaSuccess;
  do {
    if ((st = zero_run_buffers(c, early != 0)) != DKM_OK) break;
    if ((e = launch_centroids(A, 0, -1, c->d, c->cstage, !brute, 0, nullptr, c->stream))) break;
    for (int t = 0; t < iters; ++t) {
      const int par = t & 1;
      if (profile && (e = cudaEventRecordWithFlags(c->ev[4 * t + 0], c->stream, cudaEventRecordExternal))) break;
      if (!brute && (e = launch_search(A, par, c->d, c->stream))) break;
      if (profile && (e = cudaEventRecordWithFlags(c->ev[4 * t + 1], c->stream, cudaEventRecordExternal))) break;
      if ((e = launch_assign(A, c->d, brute, c->stream))) break;
      if (profile && (e = cudaEventRecordWithFlags(c->ev[4 * t + 2], c->stream, cudaEventRecordExternal))) break;
      const int insert = !brute && t + 1 < iters;
      if ((e = launch_centroids(A, 1, t, c->d, nullptr, insert, par ^ 1, nullptr, c->stream))) break;
      if (profile && (e = cudaEventRecordWithFlags(c->ev[4 * t + 3], c->stream, cudaEventRecordExternal))) break;
    }
  } while (0);
  cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
  if (st != DKM_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return fail(DKM_ECUDA, "graph capture failed: %s",
                cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(&c->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    c->gexec = nullptr;
    return fail(DKM_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
  }
  c->g_iters = iters;
  c->g_algo = c->opts.algo;
  c->g_early = early;
  c->g_profile = profile;
  return DKM_OK;
}

dkm_status validate_sizes(int64_t n, int d, int k) {
  if (d != 2 && d != 3) return fail(DKM_EINVAL, "d must be 2 or 3 (got %d)", d);
  if (n < 1 || n > kMaxPoints) return fail(DKM_EINVAL, "n must be in [1, %lld] (got %lld)",
                                           (long long)kMaxPoints, (long long)n);
  if (k < 1) return fail(DKM_EINVAL, "k must be >= 1 (got %d)", k);
  if ((int64_t)k > n) return fail(DKM_EINVAL, "k (%d) must not exceed n (%lld)", k, (long long)n);
  return DKM_OK;
}

}  // namespace

void dkm::dkm_set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void dkm_default_options(dkm_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->mem_budget_bytes = kDefaultBudget;
  o->cells_per_centroid = 1.0f;
  o->algo = DKM_ALGO_INDEXED;
  o->early_stop = 1;
  o->profile = 0;
  o->stream = nullptr;
}

const char* dkm_status_string(dkm_status s) {
  switch (s) {
    case DKM_OK: return "DKM_OK";
    case DKM_EINVAL: return "DKM_EINVAL";
    case DKM_ENOMEM: return "DKM_ENOMEM";
    case DKM_ECUDA: return "DKM_ECUDA";
    case DKM_ETIMEOUT: return "DKM_ETIMEOUT";
    case DKM_EINTERNAL: return "DKM_EINTERNAL";
  }
  return "DKM_UNKNOWN";
}

const char* dkm_last_error(void) { return g_last_error.c_str(); }

dkm_status dkm_plan(int64_t n, int d, int k, const float* bbox_lo, const float* bbox_hi,
                    const dkm_options* opts, dkm_plan_info* out) {
  DKM_TRY(validate_sizes(n, d, k));
  if (!bbox_lo || !bbox_hi || !out) return fail(DKM_EINVAL, "null argument");
  for (int a = 0; a < d; ++a) {
    if (!std::isfinite(bbox_lo[a]) || !std::isfinite(bbox_hi[a]) || bbox_lo[a] > bbox_hi[a])
      return fail(DKM_EINVAL, "bad bounding box on axis %d", a);
  }
  dkm_options o = resolve(opts);
  int64_t max_cells = 0;
  DKM_TRY(plan_grid(n, d, k, bbox_lo, bbox_hi, o, out, &max_cells));
  out->scratch_bytes = arena_plan(n, d, k, max_cells, kBucketCap).total;
  return DKM_OK;
}

dkm_status dkm_setup(dkm_ctx* c, const float* points) {
  if (!c) return fail(DKM_EINVAL, "null context");
  if (!points) return fail(DKM_EINVAL, "null points");
  c->ready = false;
  c->acc_valid = false;
  const float* src = points;
  if (!is_device_ptr(points)) {
    if (!c->pstage) DKM_CK(cudaMalloc(&c->pstage, (size_t)c->n * c->d * sizeof(float)));
    DKM_CK(cudaMemcpyAsync(c->pstage, points, (size_t)c->n * c->d * sizeof(float),
                           cudaMemcpyHostToDevice, c->stream));
    src = c->pstage;
  }
  if (c->opts.profile) DKM_CK(cudaEventRecord(c->ev_a, c->stream));
  DKM_CK(launch_bbox(src, c->n, c->d, c->st, 0, c->d, c->stream));
  DevState h;
  DKM_TRY(read_state(c, &h));
  if (h.bad) return fail(DKM_EINVAL, "points contain a non-finite or |x| > 1e18 coordinate");
  for (int a = 0; a < 3; ++a) {
    c->pbox_lo[a] = a < c->d ? float_of(h.pbox[a]) : 0.f;
    c->pbox_hi[a] = a < c->d ? float_of(h.pbox[3 + a]) : 0.f;
  }
  int64_t max_cells = 0;
  dkm_plan_info plan;
  DKM_TRY(plan_grid(c->n, c->d, c->k, c->pbox_lo, c->pbox_hi, c->opts, &plan, &max_cells));
  if (plan.cells > c->max_cells) return fail(DKM_EINTERNAL, "grid plan exceeds the arena");
  plan.scratch_bytes = c->arena_bytes;
  c->plan = plan;
  Grid g{};
  for (int a = 0; a < 3; ++a) {
    g.g0[a] = plan.origin[a];
    g.dims[a] = plan.dims[a];
  }
  g.inv_s = 1.0f / plan.cell;
  g.cap = plan.bucket_cap;
  g.cells = plan.cells;
  // the grid geometry is baked into the cached graph: rebuild it only if it changed
  if (memcmp(&g, &c->grid, sizeof(Grid)) != 0 && c->gexec) destroy_graph(c);
  c->grid = g;

  // Morton keys on a cubic lattice over the bbox
  float emax = 0.f;
  for (int a = 0; a < c->d; ++a) emax = std::max(emax, c->pbox_hi[a] - c->pbox_lo[a]);
  const float qmax = c->d == 3 ? 1023.f : 32767.f;
  const float inv = emax > 0.f ? qmax / emax : 0.f;
  DKM_CK(launch_morton(src, c->n, c->d, c->pbox_lo, inv, c->keys[0], c->vals[0], c->stream));
  int fin = 0;
  DKM_CK(launch_radix_sort(c->keys, c->vals, c->n, 30, c->rs_counts, c->rs_totals, &fin,
                           c->stream));
  c->perm = c->vals[fin];
  DKM_CK(launch_gather(src, c->n, c->d, c->perm, c->xs, c->ys, c->zs, c->n_pad, c->stream));
  // Tiling level: the finest Morton level whose cubes cut the sorted order
  // into at most n_windows / 8 pieces (so the cuts add at most 1/8 tiles).
  DKM_CK(launch_levels(c->keys[fin], c->n, c->d, c->level_hist, c->stream));
  unsigned long long hist[kMaxLevels + 1];
  DKM_CK(cudaMemcpyAsync(hist, c->level_hist, sizeof(hist), cudaMemcpyDeviceToHost, c->stream));
  DKM_CK(cudaStreamSynchronize(c->stream));
  const int levels = c->d == 3 ? 10 : 15;
  const unsigned long long seg_cap = (unsigned long long)std::max(1, c->n_windows / 8);
  int level = 0;
  unsigned long long segs = 1;
  for (int l = 1; l <= levels; ++l) {
    segs += hist[l];
    if (segs > seg_cap) break;
    level = l;
  }
  c->tile_level = level;
  const int shift = c->d * (levels - level);
  DKM_CK(launch_tiles(c->keys[fin], c->n, shift, c->n_windows, c->wcnt, c->wbase, c->n_tiles_dev,
                      c->tiles, c->stream));
  DKM_CK(launch_tile_boxes(c->xs, c->ys, c->zs, c->d, c->tiles, c->n_tiles_dev, c->tiles_max,
                           c->tbox, c->stream));
  DKM_CK(cudaMemsetAsync(c->lab, 0xff, (size_t)c->n_pad * sizeof(int32_t), c->stream));
  if (c->opts.profile) {
    DKM_CK(cudaEventRecord(c->ev_b, c->stream));
    DKM_CK(cudaEventSynchronize(c->ev_b));
    c->timings.setup_ms = ev_ms(c->ev_a, c->ev_b);
  }
  c->ready = true;
  return DKM_OK;
}

dkm_status dkm_create(dkm_ctx** out, const float* points, int64_t n, int d, int k,
                      const dkm_options* opts) {
  if (!out) return fail(DKM_EINVAL, "null output pointer");
  *out = nullptr;
  DKM_TRY(validate_sizes(n, d, k));
  if (!points) return fail(DKM_EINVAL, "null points");
  dkm_ctx* c = new dkm_ctx();
  c->n = n;
  c->d = d;
  c->k = k;
  c->opts = resolve(opts);
  c->row_filter_min = env_int("DKM_ROW_FILTER_MIN", 48);
  auto bail = [&](dkm_status s) {
    dkm_destroy(c);
    return s;
  };
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(DKM_ECUDA, "no CUDA device available"));
  }
  if (c->opts.stream) {
    c->stream = (cudaStream_t)c->opts.stream;
  } else {
    if (cudaStreamCreate(&c->stream) != cudaSuccess)
      return bail(fail(DKM_ECUDA, "cudaStreamCreate failed"));
    c->own_stream = true;
  }
  c->n_blocks = (int)((n + kBlockPts - 1) / kBlockPts);
  c->n_windows = (int)windows_of(n);
  c->tiles_max = (int)tiles_max_of(n);
  c->n_pad = (int64_t)c->n_blocks * kBlockPts;
  // arena sized for the largest grid this (k, budget) can plan
  {
    float lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
    dkm_plan_info p;
    int64_t mc = 0;
    dkm_status s = plan_grid(n, d, k, lo, hi, c->opts, &p, &mc);
    if (s != DKM_OK) return bail(s);
    c->max_cells = mc;
  }
  ArenaPlan P = arena_plan(n, d, k, c->max_cells, kBucketCap);
  cudaError_t e = cudaMalloc(&c->arena, P.total);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->arena = nullptr;
    return bail(fail(DKM_ENOMEM, "cudaMalloc(%zu B) failed: %s", P.total, cudaGetErrorString(e)));
  }
  c->arena_bytes = P.total;
  c->index_bytes = index_bytes_for(c->max_cells, k, kBucketCap);
  char* base = (char*)c->arena;
  c->xs = (float*)(base + P.xs);
  c->ys = (float*)(base + P.ys);
  c->zs = d == 3 ? (float*)(base + P.zs) : nullptr;
  c->keys[0] = (uint32_t*)(base + P.keys0);
  c->keys[1] = (uint32_t*)(base + P.keys1);
  c->vals[0] = (uint32_t*)(base + P.vals0);
  c->vals[1] = (uint32_t*)(base + P.vals1);
  c->rs_counts = (uint32_t*)(base + P.rs_counts);
  c->rs_totals = (uint32_t*)(base + P.rs_totals);
  c->tbox = (float4*)(base + P.tbox);
  c->tiles = (int2*)(base + P.tiles);
  c->n_tiles_dev = (int*)(base + P.n_tiles);
  c->wcnt = (int*)(base + P.wcnt);
  c->wbase = (int*)(base + P.wbase);
  c->level_hist = (unsigned long long*)(base + P.level_hist);
  c->lab = (int32_t*)(base + P.lab);
  c->cw = (float4*)(base + P.cw);
  c->acc = (Acc*)(base + P.acc);
  c->slots = (Slot*)(base + P.slots);
  c->st = (DevState*)(base + P.st);
  c->gcnt[0] = (int*)(base + P.gcnt0);
  c->gcnt[1] = (int*)(base + P.gcnt1);
  c->gbkt[0] = (float4*)(base + P.gbkt0);
  c->gbkt[1] = (float4*)(base + P.gbkt1);
  c->ovf[0] = (float4*)(base + P.ovf0);
  c->ovf[1] = (float4*)(base + P.ovf1);
  c->ovf_cnt = (int*)(base + P.ovf_cnt);
  c->tlist = (int*)(base + P.tlist);
  c->tcnt = (int*)(base + P.tcnt);
  c->cstage = (float*)(base + P.cstage);
  c->cstage2 = (float*)(base + P.cstage2);
  c->kstage = (int32_t*)(base + P.kstage);
  if (cudaMemsetAsync(c->arena, 0, P.total, c->stream) != cudaSuccess ||
      cudaEventCreate(&c->ev_a) != cudaSuccess || cudaEventCreate(&c->ev_b) != cudaSuccess ||
      cudaEventCreate(&c->ev_c) != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(DKM_ECUDA, "context initialisation failed"));
  }
  dkm_status s = dkm_setup(c, points);
  if (s != DKM_OK) return bail(s);
  *out = c;
  return DKM_OK;
}

dkm_status dkm_assign(dkm_ctx* c, const float* centroids, int32_t* labels, double* sse_out,
                      int64_t* changed_out) {
  DKM_TRY(check_ctx(c));
  if (!centroids) return fail(DKM_EINVAL, "null centroids");
  c->acc_valid = false;
  DKM_TRY(stage_centroids(c, centroids));
  DKM_TRY(centroid_box(c, false));
  DKM_TRY(one_pass(c, true));
  DKM_TRY(export_labels(c, labels, false));
  DevState h;
  DKM_TRY(read_state(c, &h));
  if (h.bad) return fail(DKM_EINVAL, "centroids contain a non-finite or |x| > 1e18 coordinate");
  DKM_TRY(check_state(h));
  if (sse_out) *sse_out = h.last_sse;
  if (changed_out) *changed_out = (int64_t)h.last_changed;
  c->acc_valid = true;
  return DKM_OK;
}

dkm_status dkm_update(dkm_ctx* c, const int32_t* labels, float* centroids_inout, int32_t* counts) {
  DKM_TRY(check_ctx(c));
  if (!centroids_inout) return fail(DKM_EINVAL, "null centroids");
  IterArgs A = iter_args(c, 0, 0);
  if (!labels) {
    if (!c->acc_valid) return fail(DKM_EINVAL, "dkm_update(labels=NULL) needs a preceding dkm_assign");
  } else {
    DKM_TRY(stage_centroids(c, centroids_inout));
    DKM_TRY(centroid_box(c, true));
    const int32_t* ul = labels;
    if (!is_device_ptr(labels)) {
      DKM_TRY(ensure_lstage(c));
      DKM_CK(cudaMemcpyAsync(c->lstage, labels, (size_t)c->n * sizeof(int32_t),
                             cudaMemcpyHostToDevice, c->stream));
      ul = c->lstage;
    }
    DKM_TRY(zero_run_buffers(c, false));
    DKM_CK(launch_centroids(A, 0, -1, c->d, c->cstage, 0, 0, nullptr, c->stream));
    DKM_CK(launch_accum_labels(A, c->d, ul, c->perm, c->stream));
    DevState h;
    DKM_TRY(read_state(c, &h));
    if (h.label_err) {
      c->acc_valid = false;
      return fail(DKM_EINVAL, "a label is outside [0, k)");
    }
  }
  bool host_counts = counts && !is_device_ptr(counts);
  int32_t* cdst = counts ? (host_counts ? c->kstage : counts) : nullptr;
  DKM_CK(launch_centroids(A, 1, -1, c->d, nullptr, 0, 0, cdst, c->stream));
  c->acc_valid = false;
  DKM_TRY(export_centroids(c, centroids_inout));
  if (host_counts)
    DKM_CK(cudaMemcpyAsync(counts, c->kstage, (size_t)c->k * sizeof(int32_t),
                           cudaMemcpyDeviceToHost, c->stream));
  DKM_CK(cudaStreamSynchronize(c->stream));
  return DKM_OK;
}

dkm_status dkm_run(dkm_ctx* c, const float* init, int max_iter, float* centroids_out,
                   int32_t* labels_out, int* iterations_out, double* sse_out) {
  DKM_TRY(check_ctx(c));
  if (!init) return fail(DKM_EINVAL, "null init centroids");
  if (max_iter < 0 || max_iter > kMaxIterCap)
    return fail(DKM_EINVAL, "max_iter must be in [0, %d] (got %d)", kMaxIterCap, max_iter);
  c->acc_valid = false;
  DKM_TRY(stage_centroids(c, init));
  DKM_TRY(centroid_box(c, true));
  DevState h;
  if (max_iter == 0) {
    DKM_TRY(one_pass(c, false));
    DKM_TRY(export_labels(c, labels_out, false));
    DKM_TRY(export_centroids(c, centroids_out));
    DKM_TRY(read_state(c, &h));
    DKM_TRY(check_state(h));
    if (iterations_out) *iterations_out = 0;
    if (sse_out) *sse_out = h.last_sse;
    return DKM_OK;
  }
  DKM_TRY(ensure_hist(c, max_iter));
  const int early = c->opts.early_stop ? 1 : 0;
  const int profile = c->opts.profile ? 1 : 0;
  if (!c->gexec || c->g_iters != max_iter || c->g_algo != c->opts.algo || c->g_early != early ||
      c->g_profile != profile)
    DKM_TRY(build_run_graph(c, max_iter, early, profile));
  if (profile) DKM_CK(cudaEventRecord(c->ev_a, c->stream));
  DKM_CK(cudaGraphLaunch(c->gexec, c->stream));
  if (profile) DKM_CK(cudaEventRecord(c->ev_b, c->stream));
  // final labels in caller order + SSE of those labels against the final centroids
  IterArgs A = iter_args(c, 0, 0);
  DKM_TRY(export_labels(c, labels_out, true));
  DKM_CK(launch_collect(A, -2, c->stream));
  DKM_TRY(export_centroids(c, centroids_out));
  if (profile) DKM_CK(cudaEventRecord(c->ev_c, c->stream));
  DKM_TRY(read_state(c, &h));
  DKM_TRY(check_state(h));
  if (iterations_out) *iterations_out = h.passes;
  if (sse_out) *sse_out = h.final_sse;
  if (profile) {
    dkm_timings& T = c->timings;
    T.iterations_ms = ev_ms(c->ev_a, c->ev_b);
    T.finalize_ms = ev_ms(c->ev_b, c->ev_c);
    T.passes = h.passes;
    double s = 0, a = 0, u = 0;
    for (int t = 0; t < h.passes && t < max_iter; ++t) {
      s += ev_ms(c->ev[4 * t + 0], c->ev[4 * t + 1]);
      a += ev_ms(c->ev[4 * t + 1], c->ev[4 * t + 2]);
      u += ev_ms(c->ev[4 * t + 2], c->ev[4 * t + 3]);
    }
    int p = h.passes > 0 ? h.passes : 1;
    T.search_ms = (float)(s / p);
    T.assign_ms = (float)(a / p);
    T.update_ms = (float)(u / p);
  }
  return DKM_OK;
}

dkm_status dkm_fit(const float* points, int64_t n, int d, int k, const float* init, int max_iter,
                   float* centroids_out, int32_t* labels_out, int* iterations_out,
                   double* sse_out, const dkm_options* opts) {
  dkm_ctx* c = nullptr;
  DKM_TRY(dkm_create(&c, points, n, d, k, opts));
  dkm_status s = dkm_run(c, init, max_iter, centroids_out, labels_out, iterations_out, sse_out);
  std::string keep = g_last_error;
  dkm_destroy(c);
  g_last_error = keep;
  return s;
}

dkm_status dkm_query_memory(const dkm_ctx* c, size_t* device_bytes, size_t* index_bytes) {
  if (!c) return fail(DKM_EINVAL, "null context");
  size_t extra = (c->pstage ? (size_t)c->n * c->d * sizeof(float) : 0) +
                 (c->lstage ? (size_t)c->n * sizeof(int32_t) : 0) +
                 (size_t)c->hist_cap * (sizeof(double) + sizeof(unsigned long long));
  if (device_bytes) *device_bytes = c->arena_bytes + extra;
  if (index_bytes) *index_bytes = c->plan.index_bytes;
  return DKM_OK;
}

dkm_status dkm_get_plan(const dkm_ctx* c, dkm_plan_info* out) {
  if (!c || !out) return fail(DKM_EINVAL, "null argument");
  *out = c->plan;
  return DKM_OK;
}

dkm_status dkm_last_timings(const dkm_ctx* c, dkm_timings* out) {
  if (!c || !out) return fail(DKM_EINVAL, "null argument");
  *out = c->timings;
  return DKM_OK;
}

dkm_status dkm_last_stats(dkm_ctx* c, dkm_stats* out) {
  if (!c || !out) return fail(DKM_EINVAL, "null argument");
  DevState h;
  DKM_TRY(read_state(c, &h));
  out->evals_per_point = (double)h.last_evals / (double)c->n;
  out->candidates_per_tile = h.last_tiles ? (double)h.last_cands / (double)h.last_tiles : 0.0;
  out->tiles = (int64_t)h.last_tiles;
  out->tile_level = c->tile_level;
  out->fallback_tiles = (int64_t)h.last_fallback;
  out->grid_overflow = (int64_t)h.grid_ovf;
  out->passes = h.passes;
  return DKM_OK;
}

void dkm_destroy(dkm_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  destroy_graph(c);
  if (c->ev_a) cudaEventDestroy(c->ev_a);
  if (c->ev_b) cudaEventDestroy(c->ev_b);
  if (c->ev_c) cudaEventDestroy(c->ev_c);
  if (c->arena) cudaFree(c->arena);
  if (c->pstage) cudaFree(c->pstage);
  if (c->lstage) cudaFree(c->lstage);
  if (c->sse_hist) cudaFree(c->sse_hist);
  if (c->chg_hist) cudaFree(c->chg_hist);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  cudaGetLastError();
  delete c;
}

}  // extern "C"
