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

// Per-slot counters, 64 bytes so two slots never share a 32-byte sector.
struct Slot {
  unsigned long long sse;       // fixed point, unit 2^-s_sse
  unsigned long long changed;   // labels that differ from the previous pass
  unsigned long long evals;     // point x candidate distance evaluations
  unsigned long long cands;     // sum of block candidate-list lengths
  unsigned long long fallback;  // blocks whose candidate list overflowed
  unsigned long long pad[3];
};

// Device-resident run state.
struct DevState {
  unsigned pbox[6];      // ordered-uint point bbox: lo[3], hi[3]
  unsigned cbox[6];      // ordered-uint centroid bbox of the current run
  int bad;               // non-finite or out-of-range coordinate seen
  int done;              // early stop reached
  int passes;            // assignment passes executed in the current run
  int err;               // internal error bits (kErr*)
  int label_err;         // dkm_update: a label outside [0, k)
  int pad0;
  unsigned long long last_evals, last_cands, last_fallback, last_changed, last_tiles;
  unsigned long long grid_ovf;   // centroids put in the overflow list, last rebuild
  double last_sse;               // SSE of the last pass (against its input centroids)
  double final_sse;              // SSE of the final labels against the final centroids
};

constexpr int kErrEmptyList = 1;     // a tile found no candidate (cannot happen for k >= 1)
constexpr int kErrNoCentroid = 2;    // the search found no centroid at all

// Accumulator per centroid: sum of residuals (p - c_old) per axis in fixed
// point (two's complement in u64, unit 2^-s_glob) and the count.
struct Acc { unsigned long long s[3]; unsigned long long cnt; };

// Centroid grid geometry (uniform cells; border cells are open-ended).
struct Grid {
  float g0[3];
  float inv_s;
  int dims[3];
  int cap;
  long long cells;
};

// Everything an iteration kernel needs (passed by value).
struct IterArgs {
  int64_t n;
  int k;
  int n_windows;             // ceil(n / 256)
  int tiles_max;             // launch bound on the tile count
  const int* n_tiles;        // actual tile count (device)
  const int2* tiles;         // per tile: [start, end) in sorted order
  const float* xs; const float* ys; const float* zs;   // sorted SoA points
  const float4* tbox;        // per tile: lo, hi (2 x float4)
  int32_t* lab;              // sorted labels
  float4* cw;                // working centroids (x, y, z, id bits)
  Acc* acc;                  // per centroid
  Slot* slots;
  DevState* st;
  Grid grid;
  int* gcnt[2];              // per cell fill counter, two parities
  float4* gbkt[2];           // cells * cap entries
  float4* ovf[2];            // overflow list (k entries)
  int* ovf_cnt;              // [2]
  int* tlist;                // tiles_max * kTileCap candidate ids (unordered)
  int* tcnt;                 // per tile list length (> kTileCap = overflow)
  double* sse_hist;
  unsigned long long* chg_hist;
  int track_changes;         // read previous labels and count changes
  int early_stop;
  int row_filter_min;        // tile lists longer than this are filtered again per row
};

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
__device__ __forceinline__ void fixed_exponents(const DevState* st, int64_t n, int* s_glob,
                                                int* s_sse) {
  float E = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float lo = fminf(float_of(st->pbox[a]), float_of(st->cbox[a]));
    float hi = fmaxf(float_of(st->pbox[3 + a]), float_of(st->cbox[3 + a]));
    float e = hi - lo;
    E = fmaxf(E, e == e ? e : 0.f);
  }
  int eE = exp_bound(E) + 1;   // 2 * extent < 2^eE
  int en = 64 - __clzll((unsigned long long)n);  // n < 2^en
  *s_glob = 62 - en - eE;
  *s_sse = 60 - en - 2 * eE;
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

// Cell coordinate of x along one axis (monotone in x; clamped).
// A NaN maps to cell 0, so a bad centroid can never index out of the grid.
__device__ __forceinline__ int cell_coord(float x, float g0, float inv_s, int dim) {
  float t = __fmul_rn(__fsub_rn(x, g0), inv_s);
  return t >= (float)dim ? dim - 1 : (t >= 0.f ? (int)t : 0);
}

}  // namespace dkm
