// dkm_device.cuh -- layouts, constants and exact arithmetic helpers shared by
// the libdkm kernels (sm_103a).  Nothing here is visible through the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dkm {

// ---------------------------------------------------------------------------
// Work decomposition of the Morton-sorted points.
//   row    = 64 consecutive points handled by one warp, two per lane, so the
//            distance arithmetic runs on packed f32x2 pairs;
//   window = 4 rows = 256 aligned sorted positions;
//   tile   = the points of one window that lie in one Morton cube of the
//            chosen level (a window is cut where the cube changes); one
//            warp per tile; it owns a static AABB and one candidate list per
//            pass (the batch of Section IV-A).
// ---------------------------------------------------------------------------
constexpr int kRowPts = 64;
constexpr int kRowsPerWarp = 4;
constexpr int kTilePts = kRowPts * kRowsPerWarp;          // 256
constexpr int kWarpsPerBlock = 8;
constexpr int kBlockThreads = 32 * kWarpsPerBlock;        // 256
constexpr int kBlockPts = kTilePts * kWarpsPerBlock;      // 2048 (padding unit of the arrays)
constexpr int kTileCap = 256;      // candidate-list capacity of one tile
constexpr int kSlots = 256;        // spread counters (SSE, changed, evals)
constexpr int kBucketCap = 8;      // centroid slots per grid cell
constexpr int kMaxIterCap = 1 << 16;
constexpr int kMaxLevels = 16;     // Morton levels (10 in 3D, 15 in 2D) + "never differs"

// Keep a centroid as a candidate if mind^2(box, c) <= U^2 * kKeep.  The
// factor covers the FP32 rounding of d^2, mind^2 and maxd^2 (each within
// about 5 ulp relative); 1 + 2^-16 leaves a 12x margin.
constexpr float kKeep = 1.0000152587890625f;

// Per-slot pruning counters, 64 bytes so two slots never share a 32-byte
// sector.
struct Slot {
  unsigned long long evals;     // point x candidate distance evaluations
  unsigned long long cands;     // sum of tile candidate-list lengths
  unsigned long long fallback;  // tiles whose candidate list overflowed
  unsigned long long stays;     // tiles that passed the stay test (no search)
  unsigned long long pstays;    // points that passed the point stay test
  unsigned long long pad[3];
};

// Device-resident run state (whole context).
struct DevState {
  unsigned pbox[6];      // ordered-uint bbox (used by the allocation-free step)
  unsigned cbox[6];
  int bad;               // non-finite or out-of-range coordinate seen
  int n_done;            // clouds that reached their early stop
  int passes;            // max over clouds of the passes of the current run
  int err;               // internal error bits (kErr*)
  int label_err;         // dkm_update: a label outside [0, k_b)
  int sort_err;          // dkm_setup: a radix-sort look-back gave up waiting
  int tiles;             // dkm_setup: tiles of the new point index
  int pad0;
  unsigned long long last_evals, last_cands, last_fallback, last_changed, last_tiles, last_stays;
  unsigned long long last_pstays;
  unsigned long long grid_ovf;   // centroids put in an overflow list, last rebuild
  double last_sse;               // total SSE of the last pass (against its input centroids)
  double final_sse;              // total SSE of the final labels against the final centroids
};

constexpr int kErrEmptyList = 1;     // a tile found no candidate (cannot happen for k >= 1)
constexpr int kErrNoCentroid = 2;    // the search found no centroid at all

// Accumulator per centroid: sum of residuals (p - c_old) per axis in fixed
// point (two's complement in u64, unit 2^-s_glob of its cloud) and the count.
struct Acc { unsigned long long s[3]; unsigned long long cnt; };

// Centroid grid geometry of one cloud (uniform cells; border cells are
// open-ended).
struct Grid {
  float g0[3];
  float inv_s;
  int dims[3];
  int cap;
  long long cells;
};

// One point cloud of a context (a context holds B >= 1 independent
// k-means problems).  Points of cloud b occupy sorted positions
// [p0, p0 + n) -- the same range as in the caller's concatenated input,
// because the cloud index is the most significant part of the sort key --
// and its centroids are [c0, c0 + k) of the context's centroid arrays.
struct Cloud {
  int64_t p0, n;
  int c0, k;
  long long cell0;       // first cell of its grid in the shared cell arrays
  Grid grid;
  float mlo[3];          // Morton lattice: origin and 1 / step
  float minv;
  int shift;             // tiles are cut where (key >> shift) changes
  int pad;
};

// Per-cloud run state.
struct CloudRun {
  unsigned pbox[6];      // ordered-uint point bbox: lo[3], hi[3]
  unsigned cbox[6];      // ordered-uint bbox of the run's initial centroids
  int s_glob, s_sse;     // fixed-point exponents of the run (fixed_exponents)
  int done;              // early stop reached
  int passes;            // assignment passes executed in the current run
  // max centroid drift of the cloud in the update of pass t, in slot t & 1
  // (ordered bits of a non-negative float; the other slot is cleared then)
  unsigned dmax[2];
  unsigned long long last_changed;
  double last_sse;
  double final_sse;
};

// Per-cloud pass counters, spread over kCloudSlots addresses.
constexpr int kCloudSlots = 8;
struct CloudAcc {
  unsigned long long sse[kCloudSlots];      // fixed point, unit 2^-s_sse of the cloud
  unsigned long long changed[kCloudSlots];
};

// Everything an iteration kernel needs (passed by value).
struct IterArgs {
  int64_t n;                 // total points
  int k;                     // total centroids
  int B;                     // clouds
  int n_windows;             // ceil(n / 256)
  int n_tiles;               // tiles of the point index (launch size)
  const int2* tiles;         // per tile: [start, end) in sorted order
  const int* tcloud;         // per tile: its cloud
  const int* tfirst;         // per cloud: its first tile
  // Search units: tile_group consecutive tiles of one cloud share one grid
  // search (unit_g = 1: every tile is its own unit, ubox = tbox).
  int unit_g;
  int n_units;
  const float4* ubox;        // per unit: lo, hi
  const int* ucloud;         // per unit: its cloud
  const int* tunit;          // per tile: its unit (unit_g > 1)
  const int* kcloud;         // per centroid: its cloud
  const Cloud* clouds;
  Cloud cl0;                 // copy of clouds[0] (kernel-parameter space)
  CloudRun* crun;
  CloudAcc* cacc;
  const float* xs; const float* ys; const float* zs;   // sorted SoA points
  const float4* tbox;        // per tile: lo, hi (2 x float4)
  int32_t* lab;              // sorted labels (context-wide centroid index)
  float4* cw;                // working centroids (x, y, z, id bits)
  Acc* acc;                  // per centroid
  Slot* slots;
  DevState* st;
  long long total_cells;     // cells of all clouds' grids
  int* gcnt[2];              // per cell fill counter, two parities
  float4* gbkt[2];           // cells * cap entries
  float4* ovf[2];            // overflow lists: cloud b uses [c0, c0 + k)
  int* ovf_cnt[2];           // per cloud overflow count, two parities
  float4* tlist;             // per unit kTileCap candidates (x, y, z, id bits; unordered)
  int* tcnt;                 // per unit list length (> kTileCap = overflow)
  int* tref;                 // per unit: id of the last search's bound-defining centroid (-1: none)
  double* sse_hist;
  unsigned long long* chg_hist;
  int track_changes;         // read previous labels and count changes
  int early_stop;
  int want_sse;              // sum the pass SSE (dkm_assign; a run computes its final SSE apart)
  int want_stats;            // add the pruning counters and fold the pass counters
  int row_filter_min;        // tile lists longer than this are filtered again per row
  int sort_max;              // lists up to this length (<= 32) are sorted, early exit
  // Stay test (the bound layer): cb2[j] = squared distance from centroid j
  // to the nearest other centroid of its cloud; tlab[t] = the single label
  // of tile t in its last pass (-1: mixed or unknown).  stay = 1: the tile
  // test before the search; 2: also the point test in the assignment.
  int stay;
  float* cb2;
  int* tlab;
  float* drift;              // per centroid: distance moved by the last update
  // Total centroids below 2^24: k_assign keys its staged candidates as
  // (id << 8 | list position) and reads the winners' centroids from shared
  // memory for the update sums.
  int slot_keys;
};

// A tile whose box lies within cb[a]/2 of centroid a (maxd^2 <= kStay *
// cb[a]^2) has a as the unique nearest centroid of every point in it: for
// any other c_j, |p - c_j| >= cb[a] - |p - c_a| > |p - c_a|.  kStay =
// 1/4 (1 - 2^-9) keeps the relative gap of the squared distances above
// 2^-9, far above FP32 rounding.
constexpr float kStay = 0.25f * (1.0f - 1.0f / 512.0f);

// ---------------------------------------------------------------------------
// exact helpers
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ unsigned ord_of(float f) {
#ifdef __CUDA_ARCH__
  unsigned b = __float_as_uint(f);
#else
  unsigned b; memcpy(&b, &f, 4);
#endif
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__host__ __device__ __forceinline__ float float_of(unsigned u) {
  unsigned b = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float f; memcpy(&f, &b, 4); return f;
#endif
}

// An e with |x| < 2^e for finite x: the smallest one for normal x, -125 for
// 0 and denormals.
__device__ __forceinline__ int exp_bound(float m) {
  int eb = (int)((__float_as_uint(m) >> 23) & 0xffu);
  return (eb == 0 ? 1 : eb) - 126;
}

// 2^s as a float, s clamped to the normal range.
__device__ __forceinline__ float pow2f(int s) {
  s = s < -126 ? -126 : (s > 127 ? 127 : s);
  return __uint_as_float((unsigned)(s + 127) << 23);
}

// Rescale an integer sum in unit 2^-s_from to unit 2^-s_to (rounding to
// nearest on a right shift).  The callers guarantee the result fits.
__device__ __forceinline__ long long rescale(long long v, int s_from, int s_to) {
  int sh = s_to - s_from;
  if (sh >= 0) return sh >= 63 ? 0 : (v << sh);
  int r = -sh;
  if (r >= 62) return 0;
  return (v + (1ll << (r - 1))) >> r;
}

// Fixed-point exponents of a run, identical in every kernel:
//   s_glob: unit 2^-s_glob for per-centroid residual sums, so that
//           n * (2 * extent) * 2^s_glob <= 2^62;
//   s_sse : unit for the SSE, so that n * 4 * extent^2 * 2^s_sse <= 2^62.
// extent = the largest axis extent of the union of the point and the
// initial-centroid boxes (every later centroid is a mean of points, so it
// stays inside).
__device__ __forceinline__ void fixed_exponents_box(const unsigned* pbox, const unsigned* cbox,
                                                    int64_t n, int* s_glob, int* s_sse) {
  float E = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float lo = fminf(float_of(pbox[a]), float_of(cbox[a]));
    float hi = fmaxf(float_of(pbox[3 + a]), float_of(cbox[3 + a]));
    float e = hi - lo;
    E = fmaxf(E, e == e ? e : 0.f);
  }
  int eE = exp_bound(E) + 1;   // 2 * extent < 2^eE
  int en = 64 - __clzll((unsigned long long)n);  // n < 2^en
  *s_glob = 62 - en - eE;
  *s_sse = 60 - en - 2 * eE;
}

// One coordinate of the refine step's new centroid, c + s 2^-s_glob / cnt
// (s: the fixed-point residual sum of the cluster, cnt > 0: its size), in
// FP32: the sum and the count converted once (relative error 2^-24 each),
// one correctly rounded division, an exact power-of-two scaling and the
// final addition.  The result lies within a few ulp of the exactly rounded
// mean, and no FP64 arithmetic is needed (its rate on this GPU is a small
// fraction of FP32's).
__device__ __forceinline__ float refine_coord(float c, long long s, long long cnt, int s_glob) {
  const float m = __fdiv_rn(__ll2float_rn(s), __ll2float_rn(cnt));
  return __fadd_rn(c, ldexpf(m, -s_glob));
}

__device__ __forceinline__ void fixed_exponents(const DevState* st, int64_t n, int* s_glob,
                                                int* s_sse) {
  fixed_exponents_box(st->pbox, st->cbox, n, s_glob, s_sse);
}

__device__ __forceinline__ float mind2(const float4& lo, const float4& hi, float cx, float cy,
                                       float cz, int d) {
  float tx = fmaxf(fmaxf(lo.x - cx, cx - hi.x), 0.f);
  float ty = fmaxf(fmaxf(lo.y - cy, cy - hi.y), 0.f);
  float s = __fmul_rn(tx, tx);
  s = __fmaf_rn(ty, ty, s);
  if (d == 3) {
    float tz = fmaxf(fmaxf(lo.z - cz, cz - hi.z), 0.f);
    s = __fmaf_rn(tz, tz, s);
  }
  return s;
}

__device__ __forceinline__ float maxd2(const float4& lo, const float4& hi, float cx, float cy,
                                       float cz, int d) {
  float tx = fmaxf(fabsf(cx - lo.x), fabsf(cx - hi.x));
  float ty = fmaxf(fabsf(cy - lo.y), fabsf(cy - hi.y));
  float s = __fmul_rn(tx, tx);
  s = __fmaf_rn(ty, ty, s);
  if (d == 3) {
    float tz = fmaxf(fabsf(cz - lo.z), fabsf(cz - hi.z));
    s = __fmaf_rn(tz, tz, s);
  }
  return s;
}

// Dominance over a box (the filtering test of kd-tree k-means): c cannot be
// the nearest centroid of any point of the box [lo, hi] when every point of
// the box is closer to r.  d^2(p, r) - d^2(p, c) is linear in p, so its
// maximum over the box sits at the vertex that takes, per axis, the face
// toward c; c is dominated when d^2(v, c) - d^2(v, r) exceeds the margin
// kDom * (maxd^2(box, r) + maxd^2(box, c)).  That margin covers the FP32
// rounding of the distances compared here and of the assignment's own d^2
// (about 5 ulp relative each; 2^-17 leaves a 10x margin), so a tie that
// the lowest index could decide for c is never pruned.  `slack` is the
// margin or any upper bound of it (dom_slack).
constexpr float kDom = 7.62939453125e-06f;   // 2^-17

__device__ __forceinline__ bool dominated(const float4& lo, const float4& hi, const float4& r,
                                          float slack, float cx, float cy, float cz, int d) {
  const float vx = cx > r.x ? hi.x : lo.x;
  const float vy = cy > r.y ? hi.y : lo.y;
  const float ax = __fsub_rn(vx, r.x), ay = __fsub_rn(vy, r.y);
  const float bx = __fsub_rn(vx, cx), by = __fsub_rn(vy, cy);
  float dr = __fmaf_rn(ay, ay, __fmul_rn(ax, ax));
  float dc = __fmaf_rn(by, by, __fmul_rn(bx, bx));
  if (d == 3) {
    const float vz = cz > r.z ? hi.z : lo.z;
    const float az = __fsub_rn(vz, r.z), bz = __fsub_rn(vz, cz);
    dr = __fmaf_rn(az, az, dr);
    dc = __fmaf_rn(bz, bz, dc);
  }
  return __fsub_rn(dc, dr) > slack;
}

// A margin bound for every candidate c of a box with mind^2(box, c) <= u2k,
// against a reference with maxd^2(box, r) = r_maxd2: maxd(box, c) <=
// mind(box, c) + diam(box), so maxd^2(box, c) <= 2 u2k + 2 diam^2.
__device__ __forceinline__ float dom_slack(const float4& lo, const float4& hi, float r_maxd2,
                                           float u2k, int d) {
  const float ex = hi.x - lo.x, ey = hi.y - lo.y, ez = d == 3 ? hi.z - lo.z : 0.f;
  const float diam2 = ex * ex + ey * ey + ez * ez;
  return 1.0001f * kDom * (r_maxd2 + 2.f * u2k + 2.f * diam2);
}

// Cell coordinate of x along one axis (monotone in x; clamped).
// A NaN maps to cell 0, so a bad centroid can never index out of the grid.
__device__ __forceinline__ int cell_coord(float x, float g0, float inv_s, int dim) {
  float t = __fmul_rn(__fsub_rn(x, g0), inv_s);
  return t >= (float)dim ? dim - 1 : (t >= 0.f ? (int)t : 0);
}

}  // namespace dkm
