// dkm_setup.cu -- one-time point index of a context (sm_103a).
//
// The paper builds a Ball-tree over the points once and keeps it for every
// iteration (Section IV-A, "Indexes on Spatial Vectors and Centroids";
// Algorithm 1, first step).  The GPU analog here: sort the points along a
// Morton (Z-order) curve so that consecutive points are spatially close,
// then cut the sorted order into tiles of at most 256 points that never
// leave one Morton cube of a chosen level (the cube bounds a tile's extent
// the way a node's radius bounds a ball), and store one static
// axis-aligned bounding box per tile.  Points never move, so the boxes stay
// valid for the whole run.
//
//   k_bbox         per-cloud bounding boxes (+ non-finite / range check)
//   k_morton       32-bit key per point: cloud index above a Morton code of
//                  mb bits per axis on the cloud's own box (mb = 10 in 3D
//                  and 15 in 2D for a single cloud, fewer when the cloud
//                  index needs the top bits)
//   k_rs_onesweep  stable LSD radix sort of (key, index), 8-bit digits,
//                  one kernel per digit
//   k_gather       sorted structure-of-arrays copy of the points
//   k_levels       per cloud, how many Morton cubes each level would cut
//                  the order into
//   k_choose_levels  per cloud, the cube level the tiles are cut at
//   k_tiles_*      tiles (256-point windows split at cube boundaries) and
//                  their AABBs
#include "dkm_host.h"

namespace dkm {

constexpr int kRsThreads = 256;
constexpr int kRsItems = 16;
constexpr int kRsTile = kRsThreads * kRsItems;   // 4096 keys per CTA of the sort
constexpr int kRsMaxPasses = 4;                  // 8-bit digits of a 32-bit key
#ifndef DKM_RS_MIN_BLOCKS
#define DKM_RS_MIN_BLOCKS 3   // resident sort CTAs per SM (80 registers)
#endif
constexpr float kMaxAbsCoord = 1.0e18f;          // larger coordinates are rejected

// ---------------------------------------------------------------------------
// Cloud of row i: the b with seg[b] <= i < seg[b + 1] (seg has B + 1
// ascending entries, seg[0] = 0).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int seg_of(const int64_t* __restrict__ seg, int B, int64_t i) {
  int lo = 0, hi = B;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (seg[mid] <= i) lo = mid; else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Per-cloud bounding boxes of an n x d row-major array cut into B segments
// (seg, B + 1 entries): blockIdx.y = cloud, blockIdx.x strides over its
// rows.  which = 0 -> CloudRun.pbox, 1 -> CloudRun.cbox.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void bbox_add(float v, int a, float (&lo)[3], float (&hi)[3], int& bad) {
  if (!(fabsf(v) <= kMaxAbsCoord)) {   // also catches NaN
    bad = 1;
  } else {
    lo[a] = fminf(lo[a], v);
    hi[a] = fmaxf(hi[a], v);
  }
}

// Rows are read in aligned groups of G = 4 (3D) or 2 (2D) rows, 16-byte
// loads of 12 or 4 floats, when the array is 16-byte aligned; the rows
// before the first and after the last whole group are read one by one.
__global__ void __launch_bounds__(256) k_bbox(const float* __restrict__ p, int d,
                                              const int64_t* __restrict__ seg, CloudRun* crun,
                                              DevState* st, int which) {
  const int b = blockIdx.y;
  const int64_t r0 = seg[b], r1 = seg[b + 1];
  float lo[3] = {INFINITY, INFINITY, INFINITY};
  float hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  int bad = 0;
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int G = d == 3 ? 4 : 2;
  int64_t ra = r0, rb = r0;   // whole groups cover [ra, rb)
#ifndef DKM_SCALAR_SETUP
  if ((reinterpret_cast<uintptr_t>(p) & 15) == 0) {
    ra = min(r1, (r0 + G - 1) / G * G);
    rb = ra + (r1 - ra) / G * G;
  }
#endif
  for (int64_t i = r0 + gt; i < r1; i += stride) {   // the rows outside the groups
    if (i >= ra && i < rb) continue;
    bbox_add(p[i * d], 0, lo, hi, bad);
    bbox_add(p[i * d + 1], 1, lo, hi, bad);
    if (d == 3) bbox_add(p[i * d + 2], 2, lo, hi, bad);
  }
  const float4* __restrict__ p4 = reinterpret_cast<const float4*>(p);
  for (int64_t q = ra / G + gt; q < rb / G; q += stride) {
    if (d == 3) {
      const float4 u = p4[3 * q], v = p4[3 * q + 1], w = p4[3 * q + 2];
      const float f[12] = {u.x, u.y, u.z, u.w, v.x, v.y, v.z, v.w, w.x, w.y, w.z, w.w};
#pragma unroll
      for (int e = 0; e < 12; ++e) bbox_add(f[e], e % 3, lo, hi, bad);
    } else {
      const float4 u = p4[q];
      bbox_add(u.x, 0, lo, hi, bad);
      bbox_add(u.y, 1, lo, hi, bad);
      bbox_add(u.z, 0, lo, hi, bad);
      bbox_add(u.w, 1, lo, hi, bad);
    }
  }
  for (int a = 0; a < 3; ++a) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
      hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
    }
  }
  bad = __reduce_or_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0) {
    unsigned* box = which == 0 ? crun[b].pbox : crun[b].cbox;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a < d && lo[a] <= hi[a]) {
        atomicMin(&box[a], ord_of(lo[a]));
        atomicMax(&box[3 + a], ord_of(hi[a]));
      }
    }
    if (bad) atomicOr(&st->bad, 1);
  }
}

// reset the selected boxes of every cloud to the empty box (2D contexts pin
// the z range to [0, 0]) and clear the bad-input flag
__global__ void k_reset_boxes(CloudRun* crun, int B, DevState* st, int d, int which_mask) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b == 0) {
    st->bad = 0;
    if (which_mask & 1) st->sort_err = 0;
  }
  if (b >= B) return;
  for (int w = 0; w < 2; ++w) {
    if (!(which_mask & (1 << w))) continue;
    unsigned* box = w == 0 ? crun[b].pbox : crun[b].cbox;
    for (int t = 0; t < 3; ++t) {
      box[t] = t < d ? 0xffffffffu : ord_of(0.f);
      box[3 + t] = t < d ? 0u : ord_of(0.f);
    }
  }
}

// fixed-point exponents of every cloud for the current run
__global__ void k_exponents(const Cloud* __restrict__ clouds, CloudRun* crun, int B) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  int sg, ss;
  fixed_exponents_box(crun[b].pbox, crun[b].cbox, clouds[b].n, &sg, &ss);
  crun[b].s_glob = sg;
  crun[b].s_sse = ss;
}

// ---------------------------------------------------------------------------
// Morton keys
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t spread3(uint32_t v) {   // 10 bits -> every 3rd bit
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

__device__ __forceinline__ uint32_t spread2(uint32_t v) {   // 15 bits -> every 2nd bit
  v &= 0x7fffu;
  v = (v | (v << 8)) & 0x00ff00ffu;
  v = (v | (v << 4)) & 0x0f0f0f0fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v;
}

// Key of a point of cloud b: b in the bits above d * mb, then the Morton
// code of its mb-bit-per-axis lattice coordinates on the cloud's own box.
__device__ __forceinline__ uint32_t morton_key(float x, float y, float z, int d, int b, int B,
                                               const Cloud& c, int mb) {
  const float qmax = (float)((1u << mb) - 1u);
  const float inv = c.minv;
  const float q0 = fminf(fmaxf((x - c.mlo[0]) * inv, 0.f), qmax);
  const float q1 = fminf(fmaxf((y - c.mlo[1]) * inv, 0.f), qmax);
  uint32_t key;
  if (d == 3) {
    const float q2 = fminf(fmaxf((z - c.mlo[2]) * inv, 0.f), qmax);
    key = spread3((uint32_t)q0) | (spread3((uint32_t)q1) << 1) | (spread3((uint32_t)q2) << 2);
  } else {
    key = spread2((uint32_t)q0) | (spread2((uint32_t)q1) << 1);
  }
  if (B > 1) key |= (uint32_t)b << (d * mb);
  return key;
}

// The keys of all points.  A thread takes G consecutive rows (4 in 3D, 2 in
// 2D: 16-byte loads of 12 or 4 floats and one 16- or 8-byte key store) when
// the array is 16-byte aligned, else one row.  The CTA also counts, for
// each of the npass sort passes, how many keys have each 8-bit digit
// (key >> (shift0 + 8 q)) & 255 (hist, npass x 256, zeroed beforehand).  A
// warp whose 32 keys share a digit adds 32 once, which keeps spatially
// coherent input free of shared-memory contention.
__global__ void __launch_bounds__(256) k_morton(const float* __restrict__ p, int64_t n, int d,
                                                const int64_t* __restrict__ seg, int B,
                                                const Cloud* __restrict__ clouds, int mb,
                                                uint32_t* __restrict__ keys, int shift0, int npass,
                                                uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[kRsMaxPasses][256];
  for (int t = threadIdx.x; t < kRsMaxPasses * 256; t += blockDim.x) (&h[0][0])[t] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  int G = 1;
#ifndef DKM_SCALAR_SETUP
  if ((reinterpret_cast<uintptr_t>(p) & 15) == 0) G = d == 3 ? 4 : 2;
#endif
  const int64_t ng = (n + G - 1) / G;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // the loop bound is uniform over the CTA: every lane takes part in the votes
  for (int64_t q0 = (int64_t)blockIdx.x * blockDim.x; q0 < ng; q0 += stride) {
    const int64_t q = q0 + threadIdx.x;
    uint32_t key[4] = {0u, 0u, 0u, 0u};
    bool v[4] = {false, false, false, false};
    if (G > 1 && (q + 1) * G <= n) {   // a whole aligned group
      const float4* __restrict__ p4 = reinterpret_cast<const float4*>(p);
      float f[12];
      if (d == 3) {
        const float4 u = p4[3 * q], w1 = p4[3 * q + 1], w2 = p4[3 * q + 2];
        f[0] = u.x; f[1] = u.y; f[2] = u.z; f[3] = u.w; f[4] = w1.x; f[5] = w1.y;
        f[6] = w1.z; f[7] = w1.w; f[8] = w2.x; f[9] = w2.y; f[10] = w2.z; f[11] = w2.w;
      } else {
        const float4 u = p4[q];
        f[0] = u.x; f[1] = u.y; f[2] = u.z; f[3] = u.w;
      }
      if (d == 3) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int64_t i = q * 4 + r;
          const int b = B > 1 ? seg_of(seg, B, i) : 0;
          key[r] = morton_key(f[3 * r], f[3 * r + 1], f[3 * r + 2], 3, b, B, clouds[b], mb);
          v[r] = true;
        }
      } else {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const int64_t i = q * 2 + r;
          const int b = B > 1 ? seg_of(seg, B, i) : 0;
          key[r] = morton_key(f[2 * r], f[2 * r + 1], 0.f, 2, b, B, clouds[b], mb);
          v[r] = true;
        }
      }
      if (d == 3) {
        reinterpret_cast<uint4*>(keys)[q] = make_uint4(key[0], key[1], key[2], key[3]);
      } else {
        reinterpret_cast<uint2*>(keys)[q] = make_uint2(key[0], key[1]);
      }
    } else {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int64_t i = q * G + r;
        if (r < G && i < n) {
          const int b = B > 1 ? seg_of(seg, B, i) : 0;
          key[r] = morton_key(p[i * d], p[i * d + 1], d == 3 ? p[i * d + 2] : 0.f, d, b, B,
                              clouds[b], mb);
          v[r] = true;
          keys[i] = key[r];
        }
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      if (r >= G) break;   // G is uniform
      for (int pq = 0; pq < npass; ++pq) {
        const uint32_t dig = (key[r] >> (shift0 + 8 * pq)) & 0xffu;
        const uint32_t d0 = __shfl_sync(0xffffffffu, dig, 0);
        if (__all_sync(0xffffffffu, v[r] && dig == d0)) {
          if (lane == 0) atomicAdd(&h[pq][d0], 32u);
        } else if (v[r]) {
          atomicAdd(&h[pq][dig], 1u);
        }
      }
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < npass * 256; t += blockDim.x) {
    const uint32_t c = (&h[0][0])[t];
    if (c) atomicAdd(&hist[t], c);
  }
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of (key, index) pairs, 8-bit digits, one kernel per
// digit (single-pass "onesweep" scheme).  k_morton has already counted every
// digit of every pass over the whole array; each CTA of k_rs_onesweep takes
// the next 4096-key tile in input order (a ticket, so every lower tile is
// already running), ranks its keys stably, publishes its per-digit counts,
// sums the counts of the lower tiles by decoupled look-back, and scatters.
//
// Look-back words, one per (tile, digit): tag in the high 32 bits (2p + 1:
// the tile's own count for pass p, 2p + 2: the inclusive prefix up to and
// including the tile), the count in the low 32 bits.  The buffer is zeroed
// once per sort; a word left by an earlier pass carries an older tag and
// reads as "not yet published".  Every wait is bounded: a look-back that
// has waited kRsWaitNs (or polled kRsSpinLimit times) sets DevState.sort_err
// and stops; the scatter then only writes inside the array.
// ---------------------------------------------------------------------------
constexpr int kRsSpinLimit = 1 << 24;                     // polls (second bound)
constexpr unsigned long long kRsWaitNs = 1000000000ull;   // 1 s of waiting

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
constexpr int kRsWindow = 16;   // look-back words a sort thread loads per round trip

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// exclusive scan of one value per thread across a 256-thread CTA
__device__ __forceinline__ uint32_t block_exclusive_scan256(uint32_t v, uint32_t* s_warp,
                                                            uint32_t* total) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t s = lane < 8 ? s_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < 8) s_warp[8 + lane] = s;   // inclusive warp totals
  }
  __syncthreads();
  uint32_t before = w > 0 ? s_warp[8 + w - 1] : 0u;
  if (total) *total = s_warp[8 + 7];
  return before + x - v;
}

// One pass: digit (key >> shift) & 255 of pass `pass`.  vin == nullptr
// stands for the identity (vals[i] = i) on the first pass.  The CTA's keys
// are ranked per warp (warp match + per-warp counters: stable in warp,
// item, lane order, which is the input order), placed in shared memory
// grouped by digit, then written out digit run by digit run so that
// consecutive threads store to consecutive addresses.
__global__ void __launch_bounds__(kRsThreads, DKM_RS_MIN_BLOCKS) k_rs_onesweep(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    uint32_t* __restrict__ vout, int64_t n, int shift, int pass,
    const uint32_t* __restrict__ hist, unsigned long long* status, uint32_t* ticket,
    DevState* st) {
  __shared__ uint32_t whist[8][256];
  __shared__ uint32_t goff[256];
  __shared__ uint32_t lbase[256];
  __shared__ uint32_t s_warp[16];
  __shared__ uint32_t skey[kRsTile];
  __shared__ uint32_t sval[kRsTile];
  __shared__ int s_tile;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_tile = (int)atomicAdd(ticket + pass, 1u);
  for (int t = threadIdx.x; t < 8 * 256; t += kRsThreads) (&whist[0][0])[t] = 0;
  __syncthreads();
  const int tile = s_tile;
  const int64_t cta0 = (int64_t)tile * kRsTile;
  const int64_t base = cta0 + (int64_t)w * (32 * kRsItems);
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t key[kRsItems], val[kRsItems], rank[kRsItems];
#pragma unroll
  for (int j = 0; j < kRsItems; ++j) {
    const int64_t i = base + j * 32 + lane;
    const bool v = i < n;
    key[j] = v ? kin[i] : 0u;
    val[j] = v ? (vin ? vin[i] : (uint32_t)i) : 0u;
  }
#pragma unroll
  for (int j = 0; j < kRsItems; ++j) {
    const int64_t i = base + j * 32 + lane;
    const bool v = i < n;
    const uint32_t dig = v ? ((key[j] >> shift) & 0xffu) : 0x100u;
    const uint32_t peers = __match_any_sync(0xffffffffu, dig);
    const int leader = 31 - __clz(peers);
    const uint32_t b = v ? whist[w][dig] : 0u;
    __syncwarp();
    if (v && lane == leader) whist[w][dig] = b + (uint32_t)__popc(peers);
    __syncwarp();
    rank[j] = b + (uint32_t)__popc(peers & lt);
  }
  __syncthreads();
  const int d = threadIdx.x;   // this thread's digit from here on
  uint32_t run = 0;
  for (int ww = 0; ww < 8; ++ww) {   // per digit: exclusive prefix over warps
    const uint32_t c = whist[ww][d];
    whist[ww][d] = run;
    run += c;
  }
  const unsigned long long tag_own = 2ull * pass + 1ull, tag_incl = 2ull * pass + 2ull;
  unsigned long long* my = status + (int64_t)tile * 256 + d;
  st_relaxed_u64(my, ((tile == 0 ? tag_incl : tag_own) << 32) | run);
  lbase[d] = block_exclusive_scan256(run, s_warp, nullptr);
  const uint32_t dstart = block_exclusive_scan256(hist[pass * 256 + d], s_warp, nullptr);
  // lbase and the warp prefixes are visible (barriers in the scan): group
  // the keys by digit in shared memory now, so that the look-back below runs
  // with the key registers free
#pragma unroll
  for (int j = 0; j < kRsItems; ++j) {
    const int64_t i = base + j * 32 + lane;
    if (i < n) {
      const uint32_t dig = (key[j] >> shift) & 0xffu;
      const uint32_t loc = lbase[dig] + whist[w][dig] + rank[j];
      skey[loc] = key[j];
      sval[loc] = val[j];
    }
  }
  uint32_t excl = 0;
  if (tile > 0) {
    // kRsWindow predecessors per round trip: their words are loaded
    // together, then consumed nearest first up to an inclusive prefix or
    // the first word not yet published
    int64_t tt = tile - 1;
    int polls = 0;
    unsigned long long t0 = 0;
    bool done = false;
    while (!done) {
      unsigned long long v[kRsWindow];
#pragma unroll
      for (int j = 0; j < kRsWindow; ++j)
        v[j] = tt - j >= 0 ? ld_relaxed_u64(status + (tt - j) * 256 + d) : (tag_incl << 32);
      int used = 0;
#pragma unroll
      for (int j = 0; j < kRsWindow; ++j) {
        if (done || used < j) break;   // stopped at a word not yet published
        const unsigned long long tag = v[j] >> 32;
        if (tag == tag_incl || tag == tag_own) {
          excl += (uint32_t)v[j];
          done = tag == tag_incl;
          used = j + 1;
        }
      }
      tt -= used;
      if (!done && used == 0) {
        if (polls == 0) t0 = global_ns();
        if (++polls > kRsSpinLimit || global_ns() - t0 > kRsWaitNs) {
          atomicOr(&st->sort_err, 1);
          break;
        }
        if (polls > 8) __nanosleep(64);
      }
    }
    st_relaxed_u64(my, (tag_incl << 32) | (excl + run));
  }
  goff[d] = dstart + excl;
  __syncthreads();
  const int cnt = (int)min((int64_t)kRsTile, n - cta0);
  for (int i = threadIdx.x; i < cnt; i += kRsThreads) {
    const uint32_t k = skey[i];
    const uint32_t dig = (k >> shift) & 0xffu;
    const uint32_t pos = goff[dig] + ((uint32_t)i - lbase[dig]);
    if ((int64_t)pos < n) {   // always, unless a look-back gave up (sort_err)
      kout[pos] = k;
      vout[pos] = sval[i];
    }
  }
}

// ---------------------------------------------------------------------------
// gather into sorted structure-of-arrays
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_gather(const float* __restrict__ p, int64_t n, int d,
                                                const uint32_t* __restrict__ order,
                                                float* __restrict__ xs, float* __restrict__ ys,
                                                float* __restrict__ zs, int64_t n_pad) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_pad) return;
  // padding slots (i >= n) repeat the last sorted point; they are never labelled.
  // A sort whose look-back gave up (sort_err) can leave stale entries in
  // `order`; the clamp keeps every read inside the point array (the setup
  // then reports DKM_ETIMEOUT).
  const uint32_t o = order[i < n ? i : n - 1];
  const int64_t src = (int64_t)o < n ? (int64_t)o : n - 1;
  xs[i] = p[src * d + 0];
  ys[i] = p[src * d + 1];
  if (d == 3) zs[i] = p[src * d + 2];
}

// ---------------------------------------------------------------------------
// Tiling.  Level l of a cloud's Morton code splits its box into 2^(d*l)
// cubes; a cube's points are contiguous in the sorted order.  k_levels
// counts, per cloud and level, how many sorted neighbours first differ at
// that level (a cube boundary of that level and every finer one); level 0
// is a cloud boundary.  k_choose_levels then picks, per cloud, the finest
// level whose cube count keeps the cloud's extra tiles within a set
// fraction.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int first_diff_level(uint32_t a, uint32_t b, int d, int mb) {
  const uint32_t x = a ^ b;
  if (x == 0) return kMaxLevels;          // same cube at every level
  const int p = 31 - __clz(x);            // highest differing bit
  if (p >= d * mb) return 0;              // different clouds
  return mb - p / d;                       // 1 = the coarsest level
}

// (clamped: keys left stale by a sort that gave up still index in bounds)
__device__ __forceinline__ int cloud_of_key(uint32_t key, int d, int mb, int B) {
  return B > 1 ? min((int)(key >> (d * mb)), B - 1) : 0;
}

// hist: B x (kMaxLevels + 1) counters.  With smem_hist the CTA first
// counts in shared memory (B * (kMaxLevels + 1) words, dynamic).
__global__ void __launch_bounds__(256) k_levels(const uint32_t* __restrict__ keys, int64_t n,
                                                int d, int mb, int B, int smem_hist,
                                                unsigned long long* __restrict__ hist) {
  extern __shared__ unsigned int h[];
  const int nh = B * (kMaxLevels + 1);
  if (smem_hist) {
    for (int q = threadIdx.x; q < nh; q += blockDim.x) h[q] = 0;
    __syncthreads();
  }
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x + 1; i < n; i += stride) {
    const uint32_t kb = keys[i];
    const int q = cloud_of_key(kb, d, mb, B) * (kMaxLevels + 1) + first_diff_level(keys[i - 1], kb, d, mb);
    if (smem_hist) atomicAdd(&h[q], 1u);
    else atomicAdd(&hist[q], 1ull);
  }
  if (smem_hist) {
    __syncthreads();
    for (int q = threadIdx.x; q < nh; q += blockDim.x)
      if (h[q]) atomicAdd(&hist[q], (unsigned long long)h[q]);
  }
}

// a sorted position starts a tile if it starts a 256-window or its key
// differs from its predecessor's above the cloud's cut shift (a cloud
// boundary always differs there)
__device__ __forceinline__ bool tile_starts(const uint32_t* __restrict__ keys, int64_t i,
                                            const Cloud* __restrict__ clouds, int d, int mb,
                                            int B) {
  if ((i & (kTilePts - 1)) == 0) return true;
  const uint32_t k1 = keys[i];
  const int shift = clouds[cloud_of_key(k1, d, mb, B)].shift;
  return (k1 >> shift) != (keys[i - 1] >> shift);
}

// Morton lattice of each cloud from its point box (k_bbox): a cube of
// 2^mb - 1 steps per axis over the box's longest side.
__global__ void k_lattice(Cloud* __restrict__ clouds, const CloudRun* __restrict__ crun, int B,
                          int d, int mb) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const float qmax = (float)((1u << mb) - 1u);
  float emax = 0.f;
  for (int a = 0; a < 3; ++a) {
    const float lo = a < d ? float_of(crun[b].pbox[a]) : 0.f;
    const float hi = a < d ? float_of(crun[b].pbox[3 + a]) : 0.f;
    if (a < d) emax = fmaxf(emax, hi - lo);
    clouds[b].mlo[a] = lo;
  }
  clouds[b].minv = emax > 0.f ? qmax / emax : 0.f;
}

// Per cloud the finest Morton level whose cubes cut its sorted run into at
// most max(1, windows_b / cut_div) pieces, so that cube cuts add few tiles;
// the tiles of cloud b are cut where keys differ above bit shift.
__global__ void k_choose_levels(const unsigned long long* __restrict__ hist,
                                Cloud* __restrict__ clouds, int B, int d, int mb, int cut_div) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const long long nw_b = (clouds[b].n + kTilePts - 1) / kTilePts;
  const unsigned long long seg_cap = (unsigned long long)max(1ll, nw_b / cut_div);
  const unsigned long long* h = hist + (size_t)b * (kMaxLevels + 1);
  int level = 0;
  unsigned long long segs = 1;
  for (int l = 1; l <= mb; ++l) {
    segs += h[l];
    if (segs > seg_cap) break;
    level = l;
  }
  clouds[b].shift = d * (mb - level);
}

// Tiles, in three kernels without any inter-CTA wait.  Every window start
// and every cut position (tile_starts) opens a tile, so a tile never leaves
// its 256-window.  One warp per window, 8 windows per CTA.
//   k_tiles_count: per window the 8 ballot masks of its tile starts (mask,
//     8 words per window) and its tile count (wcnt); per CTA the total (csum).
//   k_tiles_scan:  exclusive prefix of csum in place (one CTA); the total
//     tile count.
//   k_tiles_write: per window its tile ranges from the masks, their AABBs
//     (exact min / max of their points), clouds, and each cloud's first tile.
constexpr int kTlWindows = 8;

__global__ void __launch_bounds__(256) k_tiles_count(const uint32_t* __restrict__ keys, int64_t n,
                                                     const Cloud* __restrict__ clouds, int d,
                                                     int mb, int B, int n_windows,
                                                     unsigned* __restrict__ mask,
                                                     int* __restrict__ wcnt,
                                                     int* __restrict__ csum) {
  __shared__ int s_c[kTlWindows];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int64_t w = (int64_t)blockIdx.x * kTlWindows + wl;
  int c = 0;
  if (w < n_windows) {   // warp-uniform
    bool f[kTilePts / 32];
#pragma unroll
    for (int j = 0; j < kTilePts / 32; ++j) {
      const int64_t i = w * kTilePts + j * 32 + lane;
      f[j] = i < n && tile_starts(keys, i, clouds, d, mb, B);
    }
#pragma unroll
    for (int j = 0; j < kTilePts / 32; ++j) {
      const unsigned bal = __ballot_sync(0xffffffffu, f[j]);
      if (lane == j) mask[w * (kTilePts / 32) + j] = bal;
      c += __popc(bal);
    }
    if (lane == 0) wcnt[w] = c;
  }
  if (lane == 0) s_c[wl] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int q = 0; q < kTlWindows; ++q) t += s_c[q];
    csum[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(1024) k_tiles_scan(int* __restrict__ csum, int g,
                                                     int* __restrict__ n_tiles) {
  __shared__ int s_w[32];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  int carry = 0;
  for (int q0 = 0; q0 < g; q0 += 1024) {
    const int q = q0 + threadIdx.x;
    const int v = q < g ? csum[q] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[wl] = x;
    __syncthreads();
    if (wl == 0) {
      int t = s_w[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      s_w[lane] = t;   // inclusive warp totals
    }
    __syncthreads();
    const int before = wl > 0 ? s_w[wl - 1] : 0;
    if (q < g) csum[q] = carry + before + x - v;
    carry += s_w[31];
    __syncthreads();   // s_w is rewritten by the next chunk
  }
  if (threadIdx.x == 0) *n_tiles = carry;
}

__global__ void __launch_bounds__(256) k_tiles_write(
    const uint32_t* __restrict__ keys, int64_t n, int d, int mb, int B, int n_windows,
    const float* __restrict__ xs, const float* __restrict__ ys, const float* __restrict__ zs,
    const unsigned* __restrict__ mask, const int* __restrict__ wcnt, const int* __restrict__ cbase,
    int tiles_cap, int2* __restrict__ tiles, float4* __restrict__ tbox, int* __restrict__ tcloud,
    int* __restrict__ tfirst) {
  __shared__ int s_pos[kTlWindows][kTilePts + 1];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int64_t w0 = (int64_t)blockIdx.x * kTlWindows;
  const int64_t w = w0 + wl;
  if (w >= n_windows) return;   // warp-level exit, no CTA barrier below
  constexpr int kPer = kTilePts / 32;
  float x[kPer], y[kPer], z[kPer];
#pragma unroll
  for (int q = 0; q < kPer; ++q) {   // padded arrays: the whole window is addressable
    const int64_t i = w * kTilePts + q * 32 + lane;
    x[q] = xs[i];
    y[q] = ys[i];
    z[q] = d == 3 ? zs[i] : 0.f;
  }
  // the tiles of the CTA's earlier windows (lanes 0..7 hold one window each)
  const int cw = lane < wl && w0 + lane < n_windows ? wcnt[w0 + lane] : 0;
  const int base = cbase[blockIdx.x] + __reduce_add_sync(0xffffffffu, cw);
  const unsigned my_mask = lane < kPer ? mask[w * kPer + lane] : 0u;
  const unsigned lt = (1u << lane) - 1u;
  int c = 0;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const unsigned bal = __shfl_sync(0xffffffffu, my_mask, j);
    if (bal & (1u << lane)) s_pos[wl][c + __popc(bal & lt)] = (int)(w * kTilePts + j * 32 + lane);
    c += __popc(bal);
  }
  if (lane == 0) s_pos[wl][c] = (int)min((int64_t)(w + 1) * kTilePts, n);
  __syncwarp();
  for (int j = 0; j < c; ++j) {
    const int s0 = s_pos[wl][j], e0 = s_pos[wl][j + 1];
    unsigned lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0u, 0u, 0u};
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int64_t i = w * kTilePts + q * 32 + lane;
      if (i >= s0 && i < e0) {
        lo[0] = min(lo[0], ord_of(x[q])); hi[0] = max(hi[0], ord_of(x[q]));
        lo[1] = min(lo[1], ord_of(y[q])); hi[1] = max(hi[1], ord_of(y[q]));
        lo[2] = min(lo[2], ord_of(z[q])); hi[2] = max(hi[2], ord_of(z[q]));
      }
    }
    for (int a = 0; a < 3; ++a) {
      lo[a] = __reduce_min_sync(0xffffffffu, lo[a]);
      hi[a] = __reduce_max_sync(0xffffffffu, hi[a]);
    }
    const int t = base + j;
    if (lane == 0 && t < tiles_cap) {
      tiles[t] = make_int2(s0, e0);
      tbox[2 * t] = make_float4(float_of(lo[0]), float_of(lo[1]), float_of(lo[2]), 0.f);
      tbox[2 * t + 1] = make_float4(float_of(hi[0]), float_of(hi[1]), float_of(hi[2]), 0.f);
      const int b = cloud_of_key(keys[s0], d, mb, B);
      tcloud[t] = b;
      if (s0 == 0 || cloud_of_key(keys[s0 - 1], d, mb, B) != b) tfirst[b] = t;
    }
  }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static int grid_for(int64_t n, int threads, int cap) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  return (int)(g > cap ? cap : g);
}

cudaError_t launch_bbox(const float* p, int d, const int64_t* seg, int B, int64_t max_rows,
                        CloudRun* crun, DevState* st, int which, int d_ctx, cudaStream_t s) {
  k_reset_boxes<<<(B + 255) / 256, 256, 0, s>>>(crun, B, st, d_ctx, which == 0 ? 1 : 2);
  dim3 g(grid_for(max_rows, 256 * 4, 152 * 8), B);
  k_bbox<<<g, 256, 0, s>>>(p, d, seg, crun, st, which);
  return cudaGetLastError();
}

cudaError_t launch_exponents(const Cloud* clouds, CloudRun* crun, int B, cudaStream_t s) {
  k_exponents<<<(B + 255) / 256, 256, 0, s>>>(clouds, crun, B);
  return cudaGetLastError();
}

// Scratch of the sort (rs_scratch_bytes): npass x 256 digit counts, the
// passes' tickets, then one look-back word per (tile, digit).
constexpr size_t kRsHistWords = kRsMaxPasses * 256 + 64;

size_t rs_scratch_bytes(int64_t n) {
  return kRsHistWords * sizeof(uint32_t) +
         (size_t)((n + kRsTile - 1) / kRsTile) * 256 * sizeof(unsigned long long);
}

int rs_passes(int bits_lo, int bits_hi) { return (bits_hi - bits_lo + 7) / 8; }

cudaError_t launch_morton(const float* p, int64_t n, int d, const int64_t* seg, int B,
                          const Cloud* clouds, int mb, uint32_t* keys, int bits_lo, int bits_hi,
                          void* scratch, cudaStream_t s) {
  const int npass = rs_passes(bits_lo, bits_hi);
  if (npass < 1 || npass > kRsMaxPasses) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(scratch, 0, rs_scratch_bytes(n), s);
  if (e != cudaSuccess) return e;
  k_morton<<<grid_for(n, 256, 152 * 8), 256, 0, s>>>(p, n, d, seg, B, clouds, mb, keys, bits_lo,
                                                     npass, (uint32_t*)scratch);
  return cudaGetLastError();
}

// Sorts keys[0] (and the identity permutation) on bits [bits_lo, bits_hi);
// *final_buf: the buffer pair holding the result.  Expects launch_morton's
// digit counts and zeroed look-back words in scratch.
cudaError_t launch_radix_sort(uint32_t* keys[2], uint32_t* vals[2], int64_t n, int bits_lo,
                              int bits_hi, void* scratch, DevState* st, int* final_buf,
                              cudaStream_t s) {
  const int npass = rs_passes(bits_lo, bits_hi);
  if (npass < 1 || npass > kRsMaxPasses) return cudaErrorInvalidValue;
  uint32_t* hist = (uint32_t*)scratch;
  uint32_t* ticket = hist + kRsMaxPasses * 256;
  unsigned long long* status = (unsigned long long*)(hist + kRsHistWords);
  const int nt = (int)((n + kRsTile - 1) / kRsTile);
  int cur = 0;
  for (int q = 0; q < npass; ++q) {
    k_rs_onesweep<<<nt, kRsThreads, 0, s>>>(keys[cur], q == 0 ? nullptr : vals[cur],
                                            keys[cur ^ 1], vals[cur ^ 1], n, bits_lo + 8 * q, q,
                                            hist, status, ticket, st);
    cur ^= 1;
  }
  *final_buf = cur;
  return cudaGetLastError();
}

// Self-test of the bounded wait: one radix pass over n keys whose only CTA
// is handed tile 1 (the ticket starts at 1), so it waits for tile 0, which
// never runs; the wait must end by itself and set DevState.sort_err.
cudaError_t launch_sort_wait_selftest(uint32_t* keys[2], uint32_t* vals[2], int64_t n,
                                      void* scratch, DevState* st, cudaStream_t s) {
  if (n < 2 * (int64_t)kRsTile) return cudaErrorInvalidValue;
  uint32_t* hist = (uint32_t*)scratch;
  uint32_t* ticket = hist + kRsMaxPasses * 256;
  unsigned long long* status = (unsigned long long*)(hist + kRsHistWords);
  cudaError_t e = cudaMemsetAsync(scratch, 0, rs_scratch_bytes(n), s);
  if (e != cudaSuccess) return e;
  const uint32_t one = 1;
  e = cudaMemcpyAsync(ticket, &one, sizeof(one), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  k_rs_onesweep<<<1, kRsThreads, 0, s>>>(keys[0], nullptr, keys[1], vals[1], n, 0, 0, hist,
                                         status, ticket, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);   // `one` lives on this stack frame
}

cudaError_t launch_gather(const float* p, int64_t n, int d, const uint32_t* order, float* xs,
                          float* ys, float* zs, int64_t n_pad, cudaStream_t s) {
  k_gather<<<grid_for(n_pad, 256, 1 << 30), 256, 0, s>>>(p, n, d, order, xs, ys, zs, n_pad);
  return cudaGetLastError();
}

constexpr int kLevelSmemMax = 48 * 1024;

cudaError_t launch_levels(const uint32_t* keys, int64_t n, int d, int mb, int B,
                          unsigned long long* hist, cudaStream_t s) {
  const size_t nh = (size_t)B * (kMaxLevels + 1);
  cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * nh, s);
  if (e != cudaSuccess) return e;
  const size_t smem = nh * sizeof(unsigned int);
  const int use_smem = smem <= (size_t)kLevelSmemMax;
  // shared histograms pay a flush per CTA: fewer CTAs when they are large
  const int cap = use_smem ? (nh > 1024 ? 152 * 2 : 152 * 8) : 152 * 8;
  k_levels<<<grid_for(n, 256, cap), 256, use_smem ? smem : 0, s>>>(keys, n, d, mb, B, use_smem,
                                                                   hist);
  return cudaGetLastError();
}

cudaError_t launch_lattice(Cloud* clouds, const CloudRun* crun, int B, int d, int mb,
                           cudaStream_t s) {
  k_lattice<<<(B + 255) / 256, 256, 0, s>>>(clouds, crun, B, d, mb);
  return cudaGetLastError();
}

// Scratch of the tiling (u32 words): 8 masks per window, the window counts,
// the per-CTA totals.
size_t tiles_scratch_words(int n_windows) {
  return (size_t)n_windows * (kTilePts / 32) + n_windows + (n_windows + kTlWindows - 1) / kTlWindows;
}

cudaError_t launch_tiles(const uint32_t* keys, int64_t n, Cloud* clouds, int d, int mb, int B,
                         int cut_div, const unsigned long long* level_hist, int n_windows,
                         const float* xs, const float* ys, const float* zs, unsigned* scratch,
                         int tiles_cap, int2* tiles, float4* tbox, int* tcloud, int* tfirst,
                         int* n_tiles, cudaStream_t s) {
  unsigned* mask = scratch;
  int* wcnt = (int*)(mask + (size_t)n_windows * (kTilePts / 32));
  int* csum = wcnt + n_windows;
  const int g = (n_windows + kTlWindows - 1) / kTlWindows;
  k_choose_levels<<<(B + 255) / 256, 256, 0, s>>>(level_hist, clouds, B, d, mb, cut_div);
  k_tiles_count<<<g, 32 * kTlWindows, 0, s>>>(keys, n, clouds, d, mb, B, n_windows, mask, wcnt,
                                              csum);
  k_tiles_scan<<<1, 1024, 0, s>>>(csum, g, n_tiles);
  k_tiles_write<<<g, 32 * kTlWindows, 0, s>>>(keys, n, d, mb, B, n_windows, xs, ys, zs, mask,
                                              wcnt, csum, tiles_cap, tiles, tbox, tcloud, tfirst);
  return cudaGetLastError();
}

}  // namespace dkm
