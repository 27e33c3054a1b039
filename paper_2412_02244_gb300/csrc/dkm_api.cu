// dkm_api.cu -- the extern "C" boundary of libdkm (declared in include/dkm.h).
//
// Host code only: argument checks, the device arena of a context, the grid
// planner (the memory-tunable index of Section V-A), and the Lloyd loop of
// Algorithm 1 captured once per (context, max_iter) as a CUDA graph.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

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
constexpr int kMaxClouds = 65535;        // grid.y limit of the per-cloud box kernel
constexpr float kTuneMaxCpc = 4.0f;      // densest grid the arena is sized for
constexpr int kMinCutDiv = 1;            // most tile cuts the arena is sized for

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

size_t per_cell_bytes(int cap) { return size_t(2) * (sizeof(int) + size_t(cap) * sizeof(float4)); }

// bytes of the per-iteration centroid index for grids of `cells` in all
size_t index_bytes_for(int64_t cells, int64_t k, int cap) {
  return size_t(cells) * per_cell_bytes(cap) + size_t(2) * k * sizeof(float4) + 2 * sizeof(int);
}

// Cells per cloud under the memory budget (the memory-tunable index of
// Section V-A): ceil(cpc * k_b) each, scaled down together until the grids
// of all clouds fit the budget (at least one cell per cloud).
dkm_status cell_targets(const std::vector<int>& ks, float cpc, size_t budget,
                        std::vector<int64_t>* tgt, int64_t* total) {
  const int cap = kBucketCap;
  const int64_t B = (int64_t)ks.size();
  int64_t K = 0;
  for (int kb : ks) K += kb;
  const size_t fixed = index_bytes_for(0, K, cap);
  const size_t need = fixed + size_t(B) * per_cell_bytes(cap);
  if (budget < need)
    return fail(DKM_ENOMEM, "memory budget %zu B cannot hold the centroid index of k=%lld (needs >= %zu B)",
                budget, (long long)K, need);
  const int64_t budget_cells = (int64_t)((budget - fixed) / per_cell_bytes(cap));
  tgt->assign(B, 1);
  int64_t sum = 0;
  for (int64_t b = 0; b < B; ++b) {
    int64_t t = (int64_t)std::ceil((double)cpc * (double)ks[b]);
    t = std::min<int64_t>(std::max<int64_t>(t, 1), int64_t(1) << 28);
    (*tgt)[b] = t;
    sum += t;
  }
  if (sum > budget_cells) {
    // t' = 1 + floor((t - 1) f) with f = (budget_cells - B) / (sum - B):
    // sum t' <= budget_cells and t' >= 1
    const double f = (double)(budget_cells - B) / (double)(sum - B);
    sum = 0;
    for (int64_t b = 0; b < B; ++b) {
      (*tgt)[b] = 1 + (int64_t)std::floor((double)((*tgt)[b] - 1) * f);
      sum += (*tgt)[b];
    }
  }
  *total = sum;
  return DKM_OK;
}

// Uniform grid over [lo, hi] with at most `target` cells: cell edge s,
// cells per axis dims.
void grid_geometry(int d, const float* lo, const float* hi, int64_t target, int64_t dims[3],
                   double* s_out) {
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
  dims[0] = dims[1] = dims[2] = 1;
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
  *s_out = s;
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
  size_t xs, ys, zs, keys0, keys1, vals0, vals1, rs_scratch, tbox, tiles,
      tcloud, tfirst, kcloud, ubox, ucloud, ufirst, tunit, cb2, drift, tlab, tl_scratch, level_hist, doff, dcoff, clouds, crun, cacc, lab, cw, acc, slots,
      st, gcnt0, gcnt1, gbkt0, gbkt1, ovf0, ovf1, ovf_cnt0, ovf_cnt1, tlist, tcnt, tref, cstage, cstage2,
      kstage, total;
};

int64_t windows_of(int64_t n) { return (n + kTilePts - 1) / kTilePts; }
// Tiles of B clouds: every window, plus at most B - 1 cloud cuts, plus the
// cube cuts, which the tiling level keeps to max(1, windows_b / cut_div)
// per cloud (windows_b summing to at most windows + B).
int64_t tiles_cap_of(int64_t n, int64_t B) {
  return windows_of(n) + windows_of(n) / kMinCutDiv + 3 * B + 2;
}

ArenaPlan arena_plan(int64_t n, int d, int64_t k, int64_t B, int64_t max_cells, int cap) {
  ArenaPlan P;
  Layout L;
  const int64_t nb = (n + kBlockPts - 1) / kBlockPts;
  const int64_t n_pad = nb * kBlockPts;
  const int64_t nw = windows_of(n), tm = tiles_cap_of(n, B);
  P.xs = L.take<float>(n_pad);
  P.ys = L.take<float>(n_pad);
  P.zs = L.take<float>(d == 3 ? n_pad : 1);
  P.keys0 = L.take<uint32_t>(n);
  P.keys1 = L.take<uint32_t>(n);
  P.vals0 = L.take<uint32_t>(n);
  P.vals1 = L.take<uint32_t>(n);
  P.rs_scratch = L.take<unsigned char>(rs_scratch_bytes(n));
  P.tbox = L.take<float4>(2 * tm);
  P.tiles = L.take<int2>(tm);
  P.tcloud = L.take<int>(tm);
  P.tfirst = L.take<int>(B);
  P.kcloud = L.take<int>(k);
  P.ubox = L.take<float4>(2 * tm);
  P.ucloud = L.take<int>(tm);
  P.ufirst = L.take<int>(tm + 1);
  P.tunit = L.take<int>(tm);
  P.cb2 = L.take<float>(k);
  P.drift = L.take<float>(k);
  P.tlab = L.take<int>(tm);
  P.tl_scratch = L.take<unsigned>(tiles_scratch_words((int)nw));
  P.level_hist = L.take<unsigned long long>(B * (kMaxLevels + 1));
  P.doff = L.take<int64_t>(B + 1);
  P.dcoff = L.take<int64_t>(B + 1);
  P.clouds = L.take<Cloud>(B);
  P.crun = L.take<CloudRun>(B);
  P.cacc = L.take<CloudAcc>(B);
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
  P.ovf_cnt0 = L.take<int>(B);
  P.ovf_cnt1 = L.take<int>(B);
  P.tlist = L.take<float4>(tm * kTileCap);
  P.tcnt = L.take<int>(tm);
  P.tref = L.take<int>(tm);
  P.cstage = L.take<float>((size_t)k * d);
  P.cstage2 = L.take<float>((size_t)k * d);
  P.kstage = L.take<int32_t>(k);
  P.total = L.off;
  return P;
}

// grid cells the arena holds: the budget-capped targets of the densest
// grid the context may use (the tuner tries up to kTuneMaxCpc)
dkm_status cell_capacity(const std::vector<int>& ks, const dkm_options& o, int64_t* cap) {
  std::vector<int64_t> tgt;
  return cell_targets(ks, std::max(o.cells_per_centroid, kTuneMaxCpc), o.mem_budget_bytes, &tgt,
                      cap);
}

IterArgs iter_args(const dkm_ctx* c, int track_changes, int early_stop) {
  IterArgs A;
  memset(&A, 0, sizeof(A));
  A.n = c->n;
  A.k = c->k;
  A.B = c->B;
  A.n_windows = c->n_windows;
  A.n_tiles = c->n_tiles;
  A.tiles = c->tiles;
  A.tcloud = c->tcloud;
  A.tfirst = c->tfirst;
  A.kcloud = c->kcloud;
  A.unit_g = c->unit_g;
  A.n_units = c->n_units;
  A.ubox = c->unit_g > 1 ? c->ubox : c->tbox;
  A.ucloud = c->unit_g > 1 ? c->ucloud : c->tcloud;
  A.tunit = c->tunit;
  A.clouds = c->clouds;
  A.cl0 = c->h_clouds[0];
  A.crun = c->crun;
  A.cacc = c->cacc;
  A.xs = c->xs;
  A.ys = c->ys;
  A.zs = c->zs;
  A.tbox = c->tbox;
  A.lab = c->lab;
  A.cw = c->cw;
  A.acc = c->acc;
  A.slots = c->slots;
  A.st = c->st;
  A.total_cells = c->total_cells;
  for (int p = 0; p < 2; ++p) {
    A.gcnt[p] = c->gcnt[p];
    A.gbkt[p] = c->gbkt[p];
    A.ovf[p] = c->ovf[p];
    A.ovf_cnt[p] = c->ovf_cnt[p];
  }
  A.tlist = c->tlist;
  A.tcnt = c->tcnt;
  A.tref = c->tref;
  A.sse_hist = c->sse_hist;
  A.chg_hist = c->chg_hist;
  A.track_changes = track_changes;
  A.early_stop = early_stop;
  A.want_sse = 1;
  A.want_stats = 1;
  A.row_filter_min = c->row_filter_min;
  A.sort_max = c->sort_max;
  A.stay = (c->unit_g == 1 && c->opts.algo != DKM_ALGO_BRUTE) ? c->stay : 0;
  A.cb2 = c->cb2;
  A.tlab = c->tlab;
  A.drift = c->drift;
  A.slot_keys = c->k < (1 << 24) ? 1 : 0;
  return A;
}

dkm_status check_ctx(const dkm_ctx* c) {
  if (!c) return fail(DKM_EINVAL, "null context");
  if (!c->ready) return fail(DKM_EINVAL, "context has no valid point index (a dkm_setup failed)");
  return DKM_OK;
}

// Pinned staging block of a context: DevState, then B CloudRun, then B
// Cloud (copies from and to it are truly asynchronous).
size_t pin_bytes(int B) {
  return align_up(sizeof(DevState), 256) + align_up(sizeof(CloudRun) * B, 256) +
         sizeof(Cloud) * B;
}
DevState* pin_state(dkm_ctx* c) { return (DevState*)c->hpin; }
CloudRun* pin_crun(dkm_ctx* c) {
  return (CloudRun*)((char*)c->hpin + align_up(sizeof(DevState), 256));
}
Cloud* pin_clouds(dkm_ctx* c) {
  return (Cloud*)((char*)pin_crun(c) + align_up(sizeof(CloudRun) * c->B, 256));
}

dkm_status read_state(dkm_ctx* c, DevState* h) {
  DKM_CK(cudaMemcpyAsync(pin_state(c), c->st, sizeof(DevState), cudaMemcpyDeviceToHost,
                         c->stream));
  DKM_CK(cudaStreamSynchronize(c->stream));
  *h = *pin_state(c);
  return DKM_OK;
}

// run state and every cloud's state with one synchronisation
dkm_status read_state_clouds(dkm_ctx* c, DevState* h, std::vector<CloudRun>* hr) {
  DKM_CK(cudaMemcpyAsync(pin_state(c), c->st, sizeof(DevState), cudaMemcpyDeviceToHost,
                         c->stream));
  DKM_CK(cudaMemcpyAsync(pin_crun(c), c->crun, sizeof(CloudRun) * c->B, cudaMemcpyDeviceToHost,
                         c->stream));
  DKM_CK(cudaStreamSynchronize(c->stream));
  if (h) *h = *pin_state(c);
  hr->assign(pin_crun(c), pin_crun(c) + c->B);
  return DKM_OK;
}

dkm_status read_clouds(dkm_ctx* c, std::vector<CloudRun>* hr) {
  return read_state_clouds(c, nullptr, hr);
}

// Stream-ordered upload of the host cloud table.  The staging block may be
// rewritten before an earlier copy has run; that copy then carries newer
// values, and the last copy, issued after the last host change, lands
// before any later kernel.
dkm_status upload_clouds(dkm_ctx* c) {
  memcpy(pin_clouds(c), c->h_clouds.data(), sizeof(Cloud) * c->B);
  DKM_CK(cudaMemcpyAsync(c->clouds, pin_clouds(c), sizeof(Cloud) * c->B, cudaMemcpyHostToDevice,
                         c->stream));
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

// per-cloud bbox of the staged centroids, then the fixed-point exponents
// of every cloud; optional non-finite check
dkm_status centroid_box(dkm_ctx* c, bool check) {
  DKM_CK(launch_bbox(c->cstage, c->d, c->dcoff, c->B, c->max_k_b, c->crun, c->st, 1, c->d,
                     c->stream));
  DKM_CK(launch_exponents(c->clouds, c->crun, c->B, c->stream));
  if (check) {
    DevState h;
    DKM_TRY(read_state(c, &h));
    if (h.bad) return fail(DKM_EINVAL, "centroids contain a non-finite or |x| > 1e18 coordinate");
  }
  return DKM_OK;
}

dkm_status zero_run_buffers(dkm_ctx* c, bool labels_to_minus_one) {
  IterArgs A = iter_args(c, 0, 0);
  DKM_CK(launch_reset_run(A, c->stream));
  DKM_CK(cudaMemsetAsync(c->acc, 0, (size_t)c->k * sizeof(Acc), c->stream));
  DKM_CK(cudaMemsetAsync(c->slots, 0, (size_t)kSlots * sizeof(Slot), c->stream));
  DKM_CK(cudaMemsetAsync(c->gcnt[0], 0, (size_t)c->total_cells * sizeof(int), c->stream));
  DKM_CK(cudaMemsetAsync(c->gcnt[1], 0, (size_t)c->total_cells * sizeof(int), c->stream));
  DKM_CK(cudaMemsetAsync(c->ovf_cnt[0], 0, (size_t)c->B * sizeof(int), c->stream));
  DKM_CK(cudaMemsetAsync(c->ovf_cnt[1], 0, (size_t)c->B * sizeof(int), c->stream));
  if (labels_to_minus_one)
    DKM_CK(cudaMemsetAsync(c->lab, 0xff, (size_t)c->n_pad * sizeof(int32_t), c->stream));
  return DKM_OK;
}

void destroy_graph(dkm_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
  c->g_iters = -1;
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  c->ev.clear();
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
  destroy_graph(c);   // the cached graph holds the old pointers
  return DKM_OK;
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
  if (A.stay) DKM_CK(launch_cbound(A, 0, c->d, 0, c->stream));
  if (!brute) DKM_CK(launch_seed_refs(A, 0, c->d, c->stream));
  if (!brute) DKM_CK(launch_search(A, 0, c->d, c->stream));
  DKM_CK(launch_assign(A, c->d, brute, c->stream));
  DKM_CK(launch_collect(A, -1, c->stream));
  return DKM_OK;
}

// labels (sorted, device) -> caller array in original order (cloud-local
// indices); with do_sse the per-cloud SSE of those labels is left in the
// pass counters for a t = -2 collect
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

// The cached graph can be relaunched: same loop shape, and every kernel
// argument it captured (tile and unit counts, grids, cloud 0's table,
// settings) equal to the current ones.
bool graph_current(const dkm_ctx* c, int iters, int early, int profile) {
  if (!c->gexec || c->g_iters != iters || c->g_algo != c->opts.algo || c->g_early != early ||
      c->g_profile != profile)
    return false;
  const IterArgs now = iter_args(c, early, early);
  return memcmp(&now, &c->g_args, sizeof(IterArgs)) == 0;
}

// Passes whose kernels are bracketed by CUDA events: one in each `period`
// (the middle one of each period), the middle pass of a run shorter than
// the period, and with the default period 5 every pass of a run of up to
// five.  Every event node costs the graph some launch overlap, so long
// periods keep a timed run close to an unprofiled one.
int profile_period(const dkm_ctx* c) { return c->opts.profile == 1 ? 5 : c->opts.profile; }
bool profiled_pass(int t, int iters, int period) {
  if (period <= 5 && iters <= 5) return true;
  if (iters < period) return t == (iters - 1) / 2;
  return t % period == (period - 1) / 2;
}

// The kernels of a run (prep, then per pass search, assignment, update),
// enqueued on the context's stream: captured into the run graph, or
// launched directly by a one-shot fit.  Returns the first launch error in
// *e (a status other than DKM_OK comes from clearing the run buffers).
dkm_status enqueue_run(dkm_ctx* c, const IterArgs& A0, int iters, int early, int profile,
                       bool capturing, cudaError_t* e_out) {
  // inside a capture the profiling events become external event nodes
  const unsigned evf = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  const int brute = c->opts.algo == DKM_ALGO_BRUTE;
  dkm_status st = DKM_OK;
  cudaError_t e = cudaSuccess;
  do {
    if ((st = zero_run_buffers(c, early != 0)) != DKM_OK) break;
    if ((e = launch_centroids(A0, 0, -1, c->d, c->cstage, !brute, 0, nullptr, c->stream))) break;
    if (A0.stay && (e = launch_cbound(A0, 0, c->d, 0, c->stream))) break;
    if (!brute && (e = launch_seed_refs(A0, 0, c->d, c->stream))) break;
    for (int t = 0; t < iters; ++t) {
      const int par = t & 1;
      // a run returns the SSE of its final labels (computed after the
      // loop) and the pruning counters of its last pass
      IterArgs A = A0;
      A.want_sse = 0;
      // (an early-stopping run may end on any pass: it counts every pass)
      A.want_stats = (early || t + 1 == iters) ? 1 : 0;
      const bool pe = profile && profiled_pass(t, iters, profile);
      if (pe && (e = cudaEventRecordWithFlags(c->ev[4 * t + 0], c->stream, evf))) break;
      if (!brute && (e = launch_search(A, par, c->d, c->stream))) break;
      if (pe && (e = cudaEventRecordWithFlags(c->ev[4 * t + 1], c->stream, evf))) break;
      if ((e = launch_assign(A, c->d, brute, c->stream))) break;
      if (pe && (e = cudaEventRecordWithFlags(c->ev[4 * t + 2], c->stream, evf))) break;
      const int insert = !brute && t + 1 < iters;
      if ((e = launch_centroids(A, 1, t, c->d, nullptr, insert, par ^ 1, nullptr, c->stream))) break;
      if (A.stay && insert && (e = launch_cbound(A, par ^ 1, c->d, 1, c->stream))) break;
      if (pe && (e = cudaEventRecordWithFlags(c->ev[4 * t + 3], c->stream, evf))) break;
    }
  } while (0);
  *e_out = e;
  return st;
}

// per-pass profiling events of a run (created once per graph or fit)
dkm_status make_run_events(dkm_ctx* c, int iters, int profile) {
  if (!profile) return DKM_OK;
  c->ev.resize((size_t)4 * iters);
  for (auto& e : c->ev) DKM_CK(cudaEventCreate(&e));
  return DKM_OK;
}

dkm_status build_run_graph(dkm_ctx* c, int iters, int early, int profile) {
  destroy_graph(c);
  const IterArgs A0 = iter_args(c, early, early);
  DKM_TRY(make_run_events(c, iters, profile));
  cudaGraph_t g = nullptr;
  DKM_CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  const dkm_status st = enqueue_run(c, A0, iters, early, profile, true, &e);
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
  c->g_args = A0;
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

dkm_status validate_batch(const std::vector<int64_t>& off, const std::vector<int>& ks, int d) {
  const int B = (int)ks.size();
  if (d != 2 && d != 3) return fail(DKM_EINVAL, "d must be 2 or 3 (got %d)", d);
  if (B < 1 || B > kMaxClouds) return fail(DKM_EINVAL, "B must be in [1, %d] (got %d)", kMaxClouds, B);
  if (off[0] != 0) return fail(DKM_EINVAL, "offsets[0] must be 0");
  int64_t K = 0;
  for (int b = 0; b < B; ++b) {
    const int64_t nb = off[b + 1] - off[b];
    if (nb < 1) return fail(DKM_EINVAL, "cloud %d is empty (offsets must increase)", b);
    if (ks[b] < 1) return fail(DKM_EINVAL, "k of cloud %d must be >= 1 (got %d)", b, ks[b]);
    if ((int64_t)ks[b] > nb)
      return fail(DKM_EINVAL, "k of cloud %d (%d) exceeds its %lld points", b, ks[b], (long long)nb);
    K += ks[b];
  }
  if (off[B] > kMaxPoints) return fail(DKM_EINVAL, "at most %lld points in all (got %lld)",
                                       (long long)kMaxPoints, (long long)off[B]);
  if (K > kMaxPoints) return fail(DKM_EINVAL, "too many centroids in all (%lld)", (long long)K);
  return DKM_OK;
}

// Grid geometry of every cloud from its point box at the context's cells
// per centroid, under the memory budget; fills the cloud table (host copy)
// and the plan summary.
dkm_status plan_clouds(dkm_ctx* c, const std::vector<float>& blo, const std::vector<float>& bhi) {
  std::vector<int64_t> tgt;
  int64_t tot = 0;
  DKM_TRY(cell_targets(c->ks, c->cpc, c->opts.mem_budget_bytes, &tgt, &tot));
  int64_t cell0 = 0;
  for (int b = 0; b < c->B; ++b) {
    int64_t dims[3];
    double sz;
    grid_geometry(c->d, &blo[3 * b], &bhi[3 * b], tgt[b], dims, &sz);
    Grid g{};
    int64_t cells = 1;
    for (int a = 0; a < 3; ++a) {
      g.g0[a] = a < c->d ? blo[3 * b + a] : 0.f;
      g.dims[a] = (int)dims[a];
      cells *= dims[a];
    }
    g.inv_s = 1.0f / (float)sz;
    g.cap = kBucketCap;
    g.cells = cells;
    c->h_clouds[b].grid = g;
    c->h_clouds[b].cell0 = cell0;
    cell0 += cells;
    if (b == 0) {
      for (int a = 0; a < 3; ++a) {
        c->plan.dims[a] = (int)dims[a];
        c->plan.origin[a] = g.g0[a];
      }
      c->plan.cell = (float)sz;
    }
  }
  if (cell0 > c->max_cells) return fail(DKM_EINTERNAL, "grid plan exceeds the arena");
  c->total_cells = cell0;
  c->plan.bucket_cap = kBucketCap;
  c->plan.cells = cell0;
  c->plan.index_bytes = index_bytes_for(cell0, c->k, kBucketCap);
  c->plan.scratch_bytes = c->arena_bytes;
  return DKM_OK;
}

dkm_status apply_units(dkm_ctx* c, bool reset_lists);

// Tiles from the level histogram (device work only, no synchronisation):
// per cloud the cube level the tiles are cut at (k_choose_levels), then tile
// ranges, boxes, the tile -> cloud map and the tile count (DevState.tiles).
dkm_status launch_tiling(dkm_ctx* c) {
  DKM_CK(launch_tiles(c->skeys, c->n, c->clouds, c->d, c->mb, c->B, c->cut_div, c->level_hist,
                      c->n_windows, c->xs, c->ys, c->zs, c->tl_scratch, c->tiles_cap, c->tiles,
                      c->tbox, c->tcloud, c->tfirst, &c->st->tiles, c->stream));
  return DKM_OK;
}

// Host side of a tiling, from the synchronised DevState and cloud table
// (pinned copies): the cut shifts and the tile count.
dkm_status finish_tiling(dkm_ctx* c, const DevState& h, const Cloud* dev_clouds) {
  if (h.sort_err) return fail(DKM_ETIMEOUT, "index build: a radix-sort look-back wait timed out");
  for (int b = 0; b < c->B; ++b) c->h_clouds[b].shift = dev_clouds[b].shift;
  c->tile_level = c->mb - c->h_clouds[0].shift / c->d;
  const int nt = h.tiles;
  if (nt < 1 || nt > c->tiles_cap) return fail(DKM_EINTERNAL, "tile count %d out of range", nt);
  c->n_tiles = nt;
  return DKM_OK;
}

// Re-cut the tiles of the current point index (a new tile_cut_div).
dkm_status apply_tiling(dkm_ctx* c) {
  DKM_TRY(launch_tiling(c));
  DKM_CK(cudaMemcpyAsync(pin_state(c), c->st, sizeof(DevState), cudaMemcpyDeviceToHost,
                         c->stream));
  DKM_CK(cudaMemcpyAsync(pin_clouds(c), c->clouds, sizeof(Cloud) * c->B, cudaMemcpyDeviceToHost,
                         c->stream));
  DKM_CK(cudaStreamSynchronize(c->stream));
  DKM_TRY(finish_tiling(c, *pin_state(c), pin_clouds(c)));
  return apply_units(c, true);
}

// Search units (hierarchical tiles): groups of unit_g consecutive tiles of
// one cloud share one grid search over the union of their boxes, and each
// tile narrows the unit's list with its own box in k_assign.  unit_g = 1:
// every tile is its own unit.
// Candidate lists only seed the next search's bound (k_search ignores ids
// outside the tile's cloud), so they survive a rebuild of the same tiling
// (dkm_setup) and are cleared when the tiles or units are re-cut
// (reset_lists).  The stay test's single labels always are.
dkm_status apply_units(dkm_ctx* c, bool reset_lists) {
  if (reset_lists) {
    DKM_CK(cudaMemsetAsync(c->tcnt, 0, sizeof(int) * c->tiles_cap, c->stream));
    DKM_CK(cudaMemsetAsync(c->tref, 0xff, sizeof(int) * c->tiles_cap, c->stream));
  }
  DKM_CK(cudaMemsetAsync(c->tlab, 0xff, sizeof(int) * c->tiles_cap, c->stream));
  if (c->unit_g <= 1) {
    c->n_units = c->n_tiles;
    return DKM_OK;
  }
  std::vector<int> tf(c->B);
  DKM_CK(cudaMemcpyAsync(tf.data(), c->tfirst, sizeof(int) * c->B, cudaMemcpyDeviceToHost,
                         c->stream));
  DKM_CK(cudaStreamSynchronize(c->stream));
  std::vector<int> uf;
  uf.reserve((size_t)c->n_tiles / c->unit_g + c->B + 1);
  for (int b = 0; b < c->B; ++b) {
    const int t_begin = tf[b];
    const int t_end = b + 1 < c->B ? tf[b + 1] : c->n_tiles;
    for (int t = t_begin; t < t_end; t += c->unit_g) uf.push_back(t);
  }
  uf.push_back(c->n_tiles);
  c->n_units = (int)uf.size() - 1;
  DKM_CK(cudaMemcpyAsync(c->ufirst, uf.data(), sizeof(int) * uf.size(), cudaMemcpyHostToDevice,
                         c->stream));
  DKM_CK(launch_unit_boxes(c->tbox, c->tcloud, c->ufirst, c->n_units, c->ubox, c->ucloud,
                           c->tunit, c->stream));
  DKM_CK(cudaStreamSynchronize(c->stream));
  return DKM_OK;
}

// the point boxes of the last dkm_setup, per cloud (3 floats each)
void cloud_boxes(dkm_ctx* c, const std::vector<CloudRun>& hr, std::vector<float>* lo,
                 std::vector<float>* hi) {
  lo->assign(3 * c->B, 0.f);
  hi->assign(3 * c->B, 0.f);
  for (int b = 0; b < c->B; ++b)
    for (int a = 0; a < c->d; ++a) {
      (*lo)[3 * b + a] = float_of(hr[b].pbox[a]);
      (*hi)[3 * b + a] = float_of(hr[b].pbox[3 + a]);
    }
}

// The cached run graph stays valid across a setup when the kernel arguments
// it was captured with come out the same (run_impl compares them).
dkm_status setup_impl(dkm_ctx* c, const float* points) {
  c->ready = false;
  c->acc_valid = false;
  const float* src = points;
  if (!is_device_ptr(points)) {
    if (!c->pstage) DKM_CK(cudaMalloc(&c->pstage, (size_t)c->n * c->d * sizeof(float)));
    DKM_CK(cudaMemcpyAsync(c->pstage, points, (size_t)c->n * c->d * sizeof(float),
                           cudaMemcpyHostToDevice, c->stream));
    src = c->pstage;
  }
  if (c->opts.profile) DKM_CK(cudaEventRecord(c->ev_s0, c->stream));
  // Everything up to the tiles runs on the device without a host round
  // trip (the Morton lattice and the cut levels are computed there); one
  // synchronisation at the end brings back the boxes, the cloud table, the
  // tile count and the error flags.  Non-finite input is rejected then: the
  // kernels before clamp every key into range, so they stay in bounds.
  // the device cloud table must hold every cloud's point range before the
  // lattice and level kernels fill in their fields
  DKM_TRY(upload_clouds(c));
  DKM_CK(launch_bbox(src, c->d, c->doff, c->B, c->max_n_b, c->crun, c->st, 0, c->d, c->stream));
  DKM_CK(launch_lattice(c->clouds, c->crun, c->B, c->d, c->mb, c->stream));
  int fin = 0;
  // The top 24 key bits are sorted: the lower ones only order points inside
  // the finest Morton cells, far below the cube level tiles are cut at, and
  // every order is a valid index (tiles are cut wherever the compared key
  // bits change, and boxes are taken from the points themselves).
  const int bits_lo = c->key_bits > 24 ? c->key_bits - 24 : 0;
  DKM_CK(launch_morton(src, c->n, c->d, c->doff, c->B, c->clouds, c->mb, c->keys[0], bits_lo,
                       c->key_bits, c->rs_scratch, c->stream));
  DKM_CK(launch_radix_sort(c->keys, c->vals, c->n, bits_lo, c->key_bits, c->rs_scratch, c->st,
                           &fin, c->stream));
  c->perm = c->vals[fin];
  c->skeys = c->keys[fin];
  DKM_CK(launch_gather(src, c->n, c->d, c->perm, c->xs, c->ys, c->zs, c->n_pad, c->stream));
  DKM_CK(launch_levels(c->skeys, c->n, c->d, c->mb, c->B, c->level_hist, c->stream));
  DKM_TRY(launch_tiling(c));
  DKM_CK(cudaMemsetAsync(c->lab, 0xff, (size_t)c->n_pad * sizeof(int32_t), c->stream));
  DKM_CK(cudaMemcpyAsync(pin_clouds(c), c->clouds, sizeof(Cloud) * c->B, cudaMemcpyDeviceToHost,
                         c->stream));
  DevState h;
  std::vector<CloudRun> hr;
  DKM_TRY(read_state_clouds(c, &h, &hr));
  if (h.bad) return fail(DKM_EINVAL, "points contain a non-finite or |x| > 1e18 coordinate");
  cloud_boxes(c, hr, &c->h_blo, &c->h_bhi);
  for (int b = 0; b < c->B; ++b) {
    const Cloud& dc = pin_clouds(c)[b];
    for (int a = 0; a < 3; ++a) c->h_clouds[b].mlo[a] = dc.mlo[a];
    c->h_clouds[b].minv = dc.minv;
  }
  DKM_TRY(finish_tiling(c, h, pin_clouds(c)));
  DKM_TRY(plan_clouds(c, c->h_blo, c->h_bhi));
  DKM_TRY(upload_clouds(c));
  DKM_TRY(apply_units(c, !c->lists_seeded));   // lists of an earlier setup stay as seeds
  c->lists_seeded = true;
  if (c->opts.profile) {   // read out lazily (dkm_last_timings), no synchronisation here
    DKM_CK(cudaEventRecord(c->ev_s, c->stream));
    c->setup_pending = true;
  }
  c->ready = true;
  return DKM_OK;
}

dkm_status create_impl(dkm_ctx** out, const float* points, const std::vector<int64_t>& off,
                       const std::vector<int>& ks, int d, const dkm_options* opts) {
  *out = nullptr;
  DKM_TRY(validate_batch(off, ks, d));
  dkm_ctx* c = new dkm_ctx();
  auto bail = [&](dkm_status s) {
    dkm_destroy(c);
    return s;
  };
  c->B = (int)ks.size();
  c->n = off[c->B];
  c->d = d;
  c->offsets = off;
  c->ks = ks;
  c->coffs.assign(c->B + 1, 0);
  for (int b = 0; b < c->B; ++b) {
    c->coffs[b + 1] = c->coffs[b] + ks[b];
    c->max_n_b = std::max<int64_t>(c->max_n_b, off[b + 1] - off[b]);
    c->max_k_b = std::max<int64_t>(c->max_k_b, ks[b]);
  }
  c->k = (int)c->coffs[c->B];
  c->opts = resolve(opts);
  c->cpc = c->opts.cells_per_centroid;
  c->row_filter_min = 48;   // default tuning (dkm_set_tuning changes it)
  // sort key: cloud index in the top cb bits, mb Morton bits per axis below
  int cb = 0;
  while ((1 << cb) < c->B) ++cb;
  const int lmax = d == 3 ? 10 : 15;
  c->mb = std::min(lmax, (32 - cb) / d);
  c->key_bits = d * c->mb + cb;
  c->h_clouds.assign(c->B, Cloud{});
  for (int b = 0; b < c->B; ++b) {
    c->h_clouds[b].p0 = off[b];
    c->h_clouds[b].n = off[b + 1] - off[b];
    c->h_clouds[b].c0 = (int)c->coffs[b];
    c->h_clouds[b].k = ks[b];
  }
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
  c->n_blocks = (int)((c->n + kBlockPts - 1) / kBlockPts);
  c->n_windows = (int)windows_of(c->n);
  c->tiles_cap = (int)tiles_cap_of(c->n, c->B);
  c->n_pad = (int64_t)c->n_blocks * kBlockPts;
  {
    dkm_status s = cell_capacity(ks, c->opts, &c->max_cells);
    if (s != DKM_OK) return bail(s);
  }
  ArenaPlan P = arena_plan(c->n, d, c->k, c->B, c->max_cells, kBucketCap);
  cudaError_t e = cudaMalloc(&c->arena, P.total);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->arena = nullptr;
    return bail(fail(DKM_ENOMEM, "cudaMalloc(%zu B) failed: %s", P.total, cudaGetErrorString(e)));
  }
  c->arena_bytes = P.total;
  char* base = (char*)c->arena;
  c->xs = (float*)(base + P.xs);
  c->ys = (float*)(base + P.ys);
  c->zs = d == 3 ? (float*)(base + P.zs) : nullptr;
  c->keys[0] = (uint32_t*)(base + P.keys0);
  c->keys[1] = (uint32_t*)(base + P.keys1);
  c->vals[0] = (uint32_t*)(base + P.vals0);
  c->vals[1] = (uint32_t*)(base + P.vals1);
  c->rs_scratch = (void*)(base + P.rs_scratch);
  c->tbox = (float4*)(base + P.tbox);
  c->tiles = (int2*)(base + P.tiles);
  c->tcloud = (int*)(base + P.tcloud);
  c->tfirst = (int*)(base + P.tfirst);
  c->kcloud = (int*)(base + P.kcloud);
  c->ubox = (float4*)(base + P.ubox);
  c->ucloud = (int*)(base + P.ucloud);
  c->ufirst = (int*)(base + P.ufirst);
  c->tunit = (int*)(base + P.tunit);
  c->cb2 = (float*)(base + P.cb2);
  c->drift = (float*)(base + P.drift);
  c->tlab = (int*)(base + P.tlab);
  c->tl_scratch = (unsigned*)(base + P.tl_scratch);
  c->level_hist = (unsigned long long*)(base + P.level_hist);
  c->doff = (int64_t*)(base + P.doff);
  c->dcoff = (int64_t*)(base + P.dcoff);
  c->clouds = (Cloud*)(base + P.clouds);
  c->crun = (CloudRun*)(base + P.crun);
  c->cacc = (CloudAcc*)(base + P.cacc);
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
  c->ovf_cnt[0] = (int*)(base + P.ovf_cnt0);
  c->ovf_cnt[1] = (int*)(base + P.ovf_cnt1);
  c->tlist = (float4*)(base + P.tlist);
  c->tcnt = (int*)(base + P.tcnt);
  c->tref = (int*)(base + P.tref);
  c->cstage = (float*)(base + P.cstage);
  c->cstage2 = (float*)(base + P.cstage2);
  c->kstage = (int32_t*)(base + P.kstage);
  std::vector<int> kc(c->k);
  for (int b = 0; b < c->B; ++b)
    for (int64_t j = c->coffs[b]; j < c->coffs[b + 1]; ++j) kc[j] = b;
  if (cudaMemsetAsync(c->arena, 0, P.total, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(c->doff, off.data(), sizeof(int64_t) * (c->B + 1), cudaMemcpyHostToDevice,
                      c->stream) != cudaSuccess ||
      cudaMemcpyAsync(c->dcoff, c->coffs.data(), sizeof(int64_t) * (c->B + 1),
                      cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(c->kcloud, kc.data(), sizeof(int) * c->k, cudaMemcpyHostToDevice,
                      c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess ||
      cudaEventCreate(&c->ev_a) != cudaSuccess || cudaEventCreate(&c->ev_b) != cudaSuccess ||
      cudaEventCreate(&c->ev_c) != cudaSuccess || cudaEventCreate(&c->ev_s0) != cudaSuccess ||
      cudaEventCreate(&c->ev_s) != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(DKM_ECUDA, "context initialisation failed"));
  }
  if (cudaMallocHost(&c->hpin, pin_bytes(c->B)) != cudaSuccess) {
    cudaGetLastError();
    c->hpin = nullptr;
    return bail(fail(DKM_ENOMEM, "pinned host staging allocation failed"));
  }
  dkm_status s = setup_impl(c, points);
  if (s != DKM_OK) return bail(s);
  *out = c;
  return DKM_OK;
}

// Host copy of a small int64 / int32 array given as a host or device pointer.
template <class T>
dkm_status host_copy(const T* p, size_t count, std::vector<T>* out) {
  out->resize(count);
  if (is_device_ptr(p)) {
    DKM_CK(cudaMemcpy(out->data(), p, sizeof(T) * count, cudaMemcpyDeviceToHost));
  } else {
    memcpy(out->data(), p, sizeof(T) * count);
  }
  return DKM_OK;
}

template <class T>
dkm_status put_small(T* dst, const T* src, size_t count) {
  if (!dst) return DKM_OK;
  if (is_device_ptr(dst)) {
    DKM_CK(cudaMemcpy(dst, src, sizeof(T) * count, cudaMemcpyHostToDevice));
  } else {
    memcpy(dst, src, sizeof(T) * count);
  }
  return DKM_OK;
}

// Lloyd's loop on every cloud of the context; leaves the run state on the
// device and in *h.
dkm_status run_impl(dkm_ctx* c, const float* init, int max_iter, float* centroids_out,
                    int32_t* labels_out, DevState* h) {
  DKM_TRY(check_ctx(c));
  if (!init) return fail(DKM_EINVAL, "null init centroids");
  if (max_iter < 0 || max_iter > kMaxIterCap)
    return fail(DKM_EINVAL, "max_iter must be in [0, %d] (got %d)", kMaxIterCap, max_iter);
  c->acc_valid = false;
  DKM_TRY(stage_centroids(c, init));
  // The non-finite check of the initial centroids is read with the run's
  // final state instead of a synchronisation here; a run on bad centroids
  // stays in bounds (NaN maps to cell 0) and its outputs are then discarded.
  DKM_TRY(centroid_box(c, false));
  if (max_iter == 0) {
    DKM_TRY(one_pass(c, false));
    DKM_TRY(export_labels(c, labels_out, false));
    DKM_TRY(export_centroids(c, centroids_out));
    DKM_TRY(read_state(c, h));
    if (h->bad) return fail(DKM_EINVAL, "centroids contain a non-finite or |x| > 1e18 coordinate");
    DKM_TRY(check_state(*h));
    return DKM_OK;
  }
  DKM_TRY(ensure_hist(c, max_iter));
  const int early = c->opts.early_stop ? 1 : 0;
  const int profile = c->opts.profile > 0 ? profile_period(c) : 0;   // 0 or the period
  if (c->one_shot) {
    // a fit that destroys its context afterwards: capturing and
    // instantiating a graph for a single launch would cost more host time
    // than it saves, so the same kernels are launched directly
    destroy_graph(c);
    DKM_TRY(make_run_events(c, max_iter, profile));
    if (profile) DKM_CK(cudaEventRecord(c->ev_a, c->stream));
    cudaError_t e = cudaSuccess;
    DKM_TRY(enqueue_run(c, iter_args(c, early, early), max_iter, early, profile, false, &e));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(DKM_ECUDA, "run launch failed: %s", cudaGetErrorString(e));
    }
  } else {
    if (!graph_current(c, max_iter, early, profile))
      DKM_TRY(build_run_graph(c, max_iter, early, profile));
    if (profile) DKM_CK(cudaEventRecord(c->ev_a, c->stream));
    DKM_CK(cudaGraphLaunch(c->gexec, c->stream));
  }
  if (profile) DKM_CK(cudaEventRecord(c->ev_b, c->stream));
  // final labels in caller order + SSE of those labels against the final centroids
  IterArgs A = iter_args(c, 0, 0);
  DKM_TRY(export_labels(c, labels_out, true));
  DKM_CK(launch_collect(A, -2, c->stream));
  DKM_TRY(export_centroids(c, centroids_out));
  if (profile) DKM_CK(cudaEventRecord(c->ev_c, c->stream));
  DKM_TRY(read_state(c, h));
  if (h->bad) return fail(DKM_EINVAL, "centroids contain a non-finite or |x| > 1e18 coordinate");
  DKM_TRY(check_state(*h));
  if (profile) {
    dkm_timings& T = c->timings;
    T.iterations_ms = ev_ms(c->ev_a, c->ev_b);
    T.finalize_ms = ev_ms(c->ev_b, c->ev_c);
    double s = 0, a = 0, u = 0;
    int p = 0;
    for (int t = 0; t < h->passes && t < max_iter; ++t) {
      if (!profiled_pass(t, max_iter, profile)) continue;
      s += ev_ms(c->ev[4 * t + 0], c->ev[4 * t + 1]);
      a += ev_ms(c->ev[4 * t + 1], c->ev[4 * t + 2]);
      u += ev_ms(c->ev[4 * t + 2], c->ev[4 * t + 3]);
      ++p;
    }
    T.passes = p;
    p = p > 0 ? p : 1;
    T.search_ms = (float)(s / p);
    T.assign_ms = (float)(a / p);
    T.update_ms = (float)(u / p);
  }
  return DKM_OK;
}

// ---------------------------------------------------------------------------
// Index tuning
// ---------------------------------------------------------------------------
dkm_status tuning_check(const dkm_ctx* c, const dkm_tuning& t) {
  const float cmax = std::max(c->opts.cells_per_centroid, kTuneMaxCpc);
  if (!(t.cells_per_centroid > 0.f) || t.cells_per_centroid > cmax)
    return fail(DKM_EINVAL, "cells_per_centroid must be in (0, %g] (got %g)", cmax,
                t.cells_per_centroid);
  if (t.tile_cut_div < kMinCutDiv || t.tile_cut_div > 1024)
    return fail(DKM_EINVAL, "tile_cut_div must be in [%d, 1024] (got %d)", kMinCutDiv,
                t.tile_cut_div);
  if (t.row_filter_min < 0) return fail(DKM_EINVAL, "row_filter_min must be >= 0");
  if (t.sort_max < 0 || t.sort_max > 32)
    return fail(DKM_EINVAL, "sort_max must be in [0, 32] (got %d)", t.sort_max);
  if (t.tile_group < 1 || t.tile_group > 32)
    return fail(DKM_EINVAL, "tile_group must be in [1, 32] (got %d)", t.tile_group);
  if (t.stay_test < 0 || t.stay_test > 2)
    return fail(DKM_EINVAL, "stay_test must be 0, 1 or 2 (got %d)", t.stay_test);
  return DKM_OK;
}

dkm_status apply_tuning(dkm_ctx* c, const dkm_tuning& t) {
  DKM_TRY(tuning_check(c, t));
  bool changed = false;
  if (t.cells_per_centroid != c->cpc) {
    const float old = c->cpc;
    c->cpc = t.cells_per_centroid;
    dkm_status r = plan_clouds(c, c->h_blo, c->h_bhi);
    if (r != DKM_OK) {   // keep the context on its previous, valid grids
      const std::string msg = dkm_last_error();
      c->cpc = old;
      plan_clouds(c, c->h_blo, c->h_bhi);
      dkm_set_last_error(msg.c_str());
      return r;
    }
    DKM_TRY(upload_clouds(c));
    changed = true;
  }
  if (t.tile_cut_div != c->cut_div) {
    c->cut_div = t.tile_cut_div;
    dkm_status r = apply_tiling(c);
    if (r != DKM_OK) {
      c->ready = false;   // the point index is half re-cut: a dkm_setup must rebuild it
      return r;
    }
    changed = true;
  }
  if (t.row_filter_min != c->row_filter_min) {
    c->row_filter_min = t.row_filter_min;
    changed = true;
  }
  if (t.sort_max != c->sort_max) {
    c->sort_max = t.sort_max;
    changed = true;
  }
  if (t.stay_test != c->stay) {
    c->stay = t.stay_test;
    changed = true;
  }
  if (t.tile_group != c->unit_g) {
    c->unit_g = t.tile_group;
    DKM_TRY(apply_units(c, true));
    changed = true;
  }
  if (changed) {
    destroy_graph(c);
    c->acc_valid = false;
  }
  return DKM_OK;
}

dkm_tuning current_tuning(const dkm_ctx* c) {
  dkm_tuning t;
  memset(&t, 0, sizeof(t));
  t.cells_per_centroid = c->cpc;
  t.tile_cut_div = c->cut_div;
  t.row_filter_min = c->row_filter_min;
  t.sort_max = c->sort_max;
  t.tile_group = c->unit_g;
  t.stay_test = c->stay;
  return t;
}

// Mean ms per pass of `passes` Lloyd passes from the staged centroids
// (graph launch, no early stop), best of two timed launches after one
// warm-up launch.
dkm_status time_passes(dkm_ctx* c, int passes, float* ms) {
  DKM_TRY(ensure_hist(c, passes));
  if (!graph_current(c, passes, 0, 0))
    DKM_TRY(build_run_graph(c, passes, 0, 0));
  DKM_CK(cudaGraphLaunch(c->gexec, c->stream));
  float best = INFINITY;
  for (int r = 0; r < 2; ++r) {
    DKM_CK(cudaEventRecord(c->ev_a, c->stream));
    DKM_CK(cudaGraphLaunch(c->gexec, c->stream));
    DKM_CK(cudaEventRecord(c->ev_b, c->stream));
    DKM_CK(cudaEventSynchronize(c->ev_b));
    best = std::min(best, ev_ms(c->ev_a, c->ev_b));
  }
  DevState h;
  DKM_TRY(read_state(c, &h));
  DKM_TRY(check_state(h));
  *ms = best / (float)passes;
  return DKM_OK;
}

// workload shape -> tuning, shared by every context of the process
using TuneKey = std::tuple<int, int, int, int, int, int>;
std::mutex g_tune_mu;
std::map<TuneKey, dkm_tuning> g_tune_cache;

TuneKey tune_key(const dkm_ctx* c) {
  const double mn = (double)c->n / c->B, mk = (double)c->k / c->B;
  int bb = 0;
  while ((1 << bb) < c->B) ++bb;
  return TuneKey(c->d, bb, (int)std::lround(std::log2(mn)), (int)std::lround(std::log2(mk)),
                 c->opts.algo, (int)(c->opts.mem_budget_bytes >> 20));
}

dkm_status autotune_impl(dkm_ctx* c, const float* init, int passes, int use_cache,
                         dkm_tuning* out) {
  DKM_TRY(check_ctx(c));
  if (!init) return fail(DKM_EINVAL, "null init centroids");
  if (passes < 1 || passes > 64) return fail(DKM_EINVAL, "passes must be in [1, 64] (got %d)", passes);
  const TuneKey key = tune_key(c);
  if (use_cache) {
    dkm_tuning hit;
    bool found = false;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) {
        hit = it->second;
        found = true;
      }
    }
    if (found) {
      DKM_TRY(apply_tuning(c, hit));
      if (out) {
        *out = current_tuning(c);
        out->from_cache = 1;
      }
      return DKM_OK;
    }
  }
  DKM_TRY(stage_centroids(c, init));
  DKM_TRY(centroid_box(c, true));
  dkm_tuning best = current_tuning(c);
  float best_ms = 0.f;
  DKM_TRY(time_passes(c, passes, &best_ms));
  const float before_ms = best_ms;
  int trials = 1;
  auto trial = [&](dkm_tuning t) -> dkm_status {
    DKM_TRY(apply_tuning(c, t));
    float ms = 0.f;
    DKM_TRY(time_passes(c, passes, &ms));
    ++trials;
    if (ms < best_ms) {
      best_ms = ms;
      best = t;
    }
    return DKM_OK;
  };
  for (float v : {0.5f, 1.0f, 2.0f, 4.0f}) {
    if (v == best.cells_per_centroid) continue;
    dkm_tuning t = best;
    t.cells_per_centroid = v;
    DKM_TRY(trial(t));
  }
  for (int v : {1, 2, 4, 8, 16, 32}) {
    if (v == best.tile_cut_div) continue;
    dkm_tuning t = best;
    t.tile_cut_div = v;
    DKM_TRY(trial(t));
  }
  for (int v : {16, 32, 48, 96, 256}) {
    if (v == best.row_filter_min) continue;
    dkm_tuning t = best;
    t.row_filter_min = v;
    DKM_TRY(trial(t));
  }
  for (int v : {0, 16, 32}) {
    if (v == best.sort_max) continue;
    dkm_tuning t = best;
    t.sort_max = v;
    DKM_TRY(trial(t));
  }
  for (int v : {1, 2, 4, 8, 16}) {
    if (v == best.tile_group) continue;
    dkm_tuning t = best;
    t.tile_group = v;
    DKM_TRY(trial(t));
  }
  if (best.tile_group == 1) {
    for (int v : {0, 1, 2}) {
      if (v == best.stay_test) continue;
      dkm_tuning t = best;
      t.stay_test = v;
      DKM_TRY(trial(t));
    }
  }
  DKM_TRY(apply_tuning(c, best));
  destroy_graph(c);   // the next dkm_run captures with the caller's flags
  c->acc_valid = false;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
  }
  if (out) {
    *out = best;
    out->ms_per_pass = best_ms;
    out->ms_per_pass_before = before_ms;
    out->trials = trials;
    out->from_cache = 0;
  }
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

dkm_status dkm_selftest_wait(double* seconds_out) {
  const int64_t n = 8192;
  void* buf = nullptr;
  const size_t key_bytes = sizeof(uint32_t) * n;
  const size_t scratch = rs_scratch_bytes(n);
  // after the pass: the n x 3 points the gather reads and its SoA output
  const size_t pts_bytes = sizeof(float) * 3 * n;
  const size_t soa_bytes = sizeof(float) * 3 * n;
  const size_t total = 4 * key_bytes + scratch + sizeof(DevState) + pts_bytes + soa_bytes;
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
    return fail(DKM_ECUDA, "cudaStreamCreate failed");
  if (cudaMalloc(&buf, total) != cudaSuccess) {
    cudaStreamDestroy(s);
    return fail(DKM_ECUDA, "cudaMalloc failed");
  }
  char* base = (char*)buf;
  uint32_t* keys[2] = {(uint32_t*)base, (uint32_t*)(base + key_bytes)};
  uint32_t* vals[2] = {(uint32_t*)(base + 2 * key_bytes), (uint32_t*)(base + 3 * key_bytes)};
  void* scr = base + 4 * key_bytes;
  DevState* st = (DevState*)(base + 4 * key_bytes + scratch);   // scratch is a multiple of 8
  float* pts = (float*)(base + 4 * key_bytes + scratch + sizeof(DevState));
  float* soa = pts + 3 * n;
  dkm_status r = DKM_OK;
  const auto t0 = std::chrono::steady_clock::now();
  cudaError_t e = cudaMemsetAsync(buf, 0, total, s);
  // the pass's value output starts as out-of-range indices, so every slot
  // the interrupted pass leaves unwritten is a stale entry
  if (e == cudaSuccess) e = cudaMemsetAsync(vals[1], 0xff, key_bytes, s);
  if (e == cudaSuccess) e = launch_sort_wait_selftest(keys, vals, n, scr, st, s);
  const double sec =
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  // dkm_setup gathers the points by the sort's order before it reads the
  // error flag: that gather must stay inside the point array too
  if (e == cudaSuccess) e = launch_gather(pts, n, 3, vals[1], soa, soa + n, soa + 2 * n, n, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  int flag = 0;
  if (e == cudaSuccess)
    e = cudaMemcpy(&flag, &st->sort_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) r = fail(DKM_ECUDA, "self-test: %s", cudaGetErrorString(e));
  else if (!flag) r = fail(DKM_EINTERNAL, "self-test: the wait ended without reporting");
  if (seconds_out) *seconds_out = sec;
  cudaFree(buf);
  cudaStreamDestroy(s);
  return r;
}

dkm_status dkm_plan(int64_t n, int d, int k, const float* bbox_lo, const float* bbox_hi,
                    const dkm_options* opts, dkm_plan_info* out) {
  DKM_TRY(validate_sizes(n, d, k));
  if (!bbox_lo || !bbox_hi || !out) return fail(DKM_EINVAL, "null argument");
  for (int a = 0; a < d; ++a) {
    if (!std::isfinite(bbox_lo[a]) || !std::isfinite(bbox_hi[a]) || bbox_lo[a] > bbox_hi[a])
      return fail(DKM_EINVAL, "bad bounding box on axis %d", a);
  }
  dkm_options o = resolve(opts);
  const std::vector<int> ks(1, k);
  std::vector<int64_t> tgt;
  int64_t tot = 0, cap_cells = 0;
  DKM_TRY(cell_targets(ks, o.cells_per_centroid, o.mem_budget_bytes, &tgt, &tot));
  DKM_TRY(cell_capacity(ks, o, &cap_cells));
  int64_t dims[3];
  double sz;
  grid_geometry(d, bbox_lo, bbox_hi, tgt[0], dims, &sz);
  memset(out, 0, sizeof(*out));
  int64_t cells = 1;
  for (int a = 0; a < 3; ++a) {
    out->dims[a] = (int)dims[a];
    out->origin[a] = a < d ? bbox_lo[a] : 0.f;
    cells *= dims[a];
  }
  out->cell = (float)sz;
  out->bucket_cap = kBucketCap;
  out->cells = cells;
  out->index_bytes = index_bytes_for(cells, k, kBucketCap);
  out->scratch_bytes = arena_plan(n, d, k, 1, cap_cells, kBucketCap).total;
  return DKM_OK;
}

dkm_status dkm_setup(dkm_ctx* c, const float* points) {
  if (!c) return fail(DKM_EINVAL, "null context");
  if (!points) return fail(DKM_EINVAL, "null points");
  return setup_impl(c, points);
}

dkm_status dkm_create(dkm_ctx** out, const float* points, int64_t n, int d, int k,
                      const dkm_options* opts) {
  if (!out) return fail(DKM_EINVAL, "null output pointer");
  *out = nullptr;
  DKM_TRY(validate_sizes(n, d, k));
  if (!points) return fail(DKM_EINVAL, "null points");
  return create_impl(out, points, std::vector<int64_t>{0, n}, std::vector<int>{k}, d, opts);
}

dkm_status dkm_create_batched(dkm_ctx** out, const float* points, const int64_t* offsets, int B,
                              int d, const int32_t* ks, const dkm_options* opts) {
  if (!out) return fail(DKM_EINVAL, "null output pointer");
  *out = nullptr;
  if (!points || !offsets || !ks) return fail(DKM_EINVAL, "null argument");
  if (B < 1 || B > kMaxClouds) return fail(DKM_EINVAL, "B must be in [1, %d] (got %d)", kMaxClouds, B);
  std::vector<int64_t> off;
  std::vector<int32_t> kv;
  DKM_TRY(host_copy(offsets, (size_t)B + 1, &off));
  DKM_TRY(host_copy(ks, (size_t)B, &kv));
  return create_impl(out, points, off, std::vector<int>(kv.begin(), kv.end()), d, opts);
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
  DevState h;
  DKM_TRY(run_impl(c, init, max_iter, centroids_out, labels_out, &h));
  if (iterations_out) *iterations_out = max_iter == 0 ? 0 : h.passes;
  if (sse_out) *sse_out = max_iter == 0 ? h.last_sse : h.final_sse;
  return DKM_OK;
}

dkm_status dkm_run_batched(dkm_ctx* c, const float* init, int max_iter, float* centroids_out,
                           int32_t* labels_out, int32_t* iterations_out, double* sse_out) {
  DevState h;
  DKM_TRY(run_impl(c, init, max_iter, centroids_out, labels_out, &h));
  if (!iterations_out && !sse_out) return DKM_OK;
  std::vector<CloudRun> hr;
  DKM_TRY(read_clouds(c, &hr));
  std::vector<int32_t> it(c->B);
  std::vector<double> ss(c->B);
  for (int b = 0; b < c->B; ++b) {
    it[b] = max_iter == 0 ? 0 : hr[b].passes;
    ss[b] = max_iter == 0 ? hr[b].last_sse : hr[b].final_sse;
  }
  DKM_TRY(put_small(iterations_out, it.data(), it.size()));
  DKM_TRY(put_small(sse_out, ss.data(), ss.size()));
  return DKM_OK;
}

dkm_status dkm_fit(const float* points, int64_t n, int d, int k, const float* init, int max_iter,
                   float* centroids_out, int32_t* labels_out, int* iterations_out,
                   double* sse_out, const dkm_options* opts) {
  dkm_ctx* c = nullptr;
  DKM_TRY(dkm_create(&c, points, n, d, k, opts));
  c->one_shot = true;
  dkm_status s = dkm_run(c, init, max_iter, centroids_out, labels_out, iterations_out, sse_out);
  std::string keep = g_last_error;
  dkm_destroy(c);
  g_last_error = keep;
  return s;
}

dkm_status dkm_fit_batched(const float* points, const int64_t* offsets, int B, int d,
                           const int32_t* ks, const float* init, int max_iter,
                           float* centroids_out, int32_t* labels_out, int32_t* iterations_out,
                           double* sse_out, const dkm_options* opts) {
  dkm_ctx* c = nullptr;
  DKM_TRY(dkm_create_batched(&c, points, offsets, B, d, ks, opts));
  c->one_shot = true;
  dkm_status s =
      dkm_run_batched(c, init, max_iter, centroids_out, labels_out, iterations_out, sse_out);
  std::string keep = g_last_error;
  dkm_destroy(c);
  g_last_error = keep;
  return s;
}

dkm_status dkm_get_tuning(const dkm_ctx* c, dkm_tuning* out) {
  if (!c || !out) return fail(DKM_EINVAL, "null argument");
  *out = current_tuning(c);
  return DKM_OK;
}

dkm_status dkm_set_tuning(dkm_ctx* c, const dkm_tuning* t) {
  DKM_TRY(check_ctx(c));
  if (!t) return fail(DKM_EINVAL, "null tuning");
  return apply_tuning(c, *t);
}

dkm_status dkm_autotune(dkm_ctx* c, const float* init, int passes, int use_cache,
                        dkm_tuning* out) {
  return autotune_impl(c, init, passes, use_cache, out);
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

dkm_status dkm_last_timings(dkm_ctx* c, dkm_timings* out) {
  if (!c || !out) return fail(DKM_EINVAL, "null argument");
  if (c->setup_pending) {
    DKM_CK(cudaEventSynchronize(c->ev_s));
    c->timings.setup_ms = ev_ms(c->ev_s0, c->ev_s);
    c->setup_pending = false;
  }
  *out = c->timings;
  return DKM_OK;
}

dkm_status dkm_last_stats(dkm_ctx* c, dkm_stats* out) {
  if (!c || !out) return fail(DKM_EINVAL, "null argument");
  DevState h;
  DKM_TRY(read_state(c, &h));
  out->evals_per_point = (double)h.last_evals / (double)c->n;
  out->candidates_per_tile = h.last_tiles ? (double)h.last_cands / (double)h.last_tiles : 0.0;
  out->tiles = (int64_t)c->n_tiles;
  out->tile_level = c->tile_level;
  out->fallback_tiles = (int64_t)h.last_fallback;
  out->stayed_tiles = (int64_t)h.last_stays;
  out->stayed_points = (int64_t)h.last_pstays;
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
  if (c->ev_s0) cudaEventDestroy(c->ev_s0);
  if (c->ev_s) cudaEventDestroy(c->ev_s);
  if (c->arena) cudaFree(c->arena);
  if (c->pstage) cudaFree(c->pstage);
  if (c->lstage) cudaFree(c->lstage);
  if (c->sse_hist) cudaFree(c->sse_hist);
  if (c->chg_hist) cudaFree(c->chg_hist);
  if (c->hpin) cudaFreeHost(c->hpin);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  cudaGetLastError();
  delete c;
}

}  // extern "C"
