// dkm_setup.cu -- one-time point index of a context (sm_103a).
//
// The paper builds a Ball-tree over the points once and keeps it for every
// iteration (Section IV-A, "Indexes on Spatial Vectors and Centroids";
// Algorithm 1, first step).  The GPU analog here: sort the points along a
// Morton (Z-order) curve so that consecutive points are spatially close,
// cut the sorted order into fixed tiles and blocks, and store one static
// axis-aligned bounding box per tile and per block.  Points never move, so
// the boxes stay valid for the whole run.
//
//   k_bbox       bounding box of the input (+ non-finite / range check)
//   k_morton     30-bit Morton key per point (3 x 10 or 2 x 15 bits)
//   k_rs_*       stable LSD radix sort of (key, index), 8-bit digits
//   k_gather     sorted structure-of-arrays copy of the points
//   k_boxes      per-tile and per-block AABBs
#include "dkm_host.h"

namespace dkm {

constexpr int kRsThreads = 256;
constexpr int kRsItems = 8;
constexpr int kRsTile = kRsThreads * kRsItems;   // 2048 keys per CTA
constexpr float kMaxAbsCoord = 1.0e18f;          // larger coordinates are rejected

// ---------------------------------------------------------------------------
// bounding box of an n x d row-major array; which = 0 -> pbox, 1 -> cbox
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_bbox(const float* __restrict__ p, int64_t n, int d,
                                              DevState* st, int which) {
  float lo[3] = {INFINITY, INFINITY, INFINITY};
  float hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  int bad = 0;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    for (int a = 0; a < d; ++a) {
      float v = p[i * d + a];
      if (!(fabsf(v) <= kMaxAbsCoord)) {   // also catches NaN
        bad = 1;
      } else {
        lo[a] = fminf(lo[a], v);
        hi[a] = fmaxf(hi[a], v);
      }
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
    unsigned* box = which == 0 ? st->pbox : st->cbox;
    for (int a = 0; a < d; ++a) {
      if (lo[a] <= hi[a]) {
        atomicMin(&box[a], ord_of(lo[a]));
        atomicMax(&box[3 + a], ord_of(hi[a]));
      }
    }
    if (bad) atomicOr(&st->bad, 1);
  }
}

// reset both boxes to the empty box; 2D contexts pin the z range to [0, 0]
__global__ void k_reset_boxes(DevState* st, int d, int which_mask) {
  int t = threadIdx.x;
  if (t < 3) {
    for (int w = 0; w < 2; ++w) {
      if (!(which_mask & (1 << w))) continue;
      unsigned* box = w == 0 ? st->pbox : st->cbox;
      if (t < d) {
        box[t] = 0xffffffffu;
        box[3 + t] = 0u;
      } else {
        box[t] = ord_of(0.f);
        box[3 + t] = ord_of(0.f);
      }
    }
  }
  if (t == 0) st->bad = 0;
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

__global__ void __launch_bounds__(256) k_morton(const float* __restrict__ p, int64_t n, int d,
                                                float3 lo, float inv, uint32_t* __restrict__ keys,
                                                uint32_t* __restrict__ vals) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float qmax = d == 3 ? 1023.f : 32767.f;
  float q0 = fminf(fmaxf((p[i * d + 0] - lo.x) * inv, 0.f), qmax);
  float q1 = fminf(fmaxf((p[i * d + 1] - lo.y) * inv, 0.f), qmax);
  uint32_t key;
  if (d == 3) {
    float q2 = fminf(fmaxf((p[i * d + 2] - lo.z) * inv, 0.f), qmax);
    key = spread3((uint32_t)q0) | (spread3((uint32_t)q1) << 1) | (spread3((uint32_t)q2) << 2);
  } else {
    key = spread2((uint32_t)q0) | (spread2((uint32_t)q1) << 1);
  }
  keys[i] = key;
  vals[i] = (uint32_t)i;
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort, 8-bit digits.  Per pass: upsweep (per-CTA digit
// counts, digit-major), scan (one CTA per digit), downsweep (stable rank via
// warp match + per-warp counters, then scatter).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kRsThreads) k_rs_upsweep(const uint32_t* __restrict__ keys,
                                                           int64_t n, int shift,
                                                           uint32_t* __restrict__ counts, int nb) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kRsTile;
  int lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < kRsItems; ++j) {
    int64_t i = base + (int64_t)j * kRsThreads + threadIdx.x;
    bool v = i < n;
    uint32_t dig = v ? ((keys[i] >> shift) & 0xffu) : 0x100u;
    uint32_t peers = __match_any_sync(0xffffffffu, dig);
    int leader = __ffs(peers) - 1;
    if (v && lane == leader) atomicAdd(&h[dig], (uint32_t)__popc(peers));
  }
  __syncthreads();
  counts[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of one block-sum per thread across a 256-thread CTA
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

__global__ void __launch_bounds__(256) k_rs_scan(uint32_t* __restrict__ counts, int nb,
                                                 uint32_t* __restrict__ totals) {
  __shared__ uint32_t s_warp[16];
  uint32_t* row = counts + (int64_t)blockIdx.x * nb;
  int per = (nb + 255) / 256;
  int start = threadIdx.x * per;
  uint32_t sum = 0;
  for (int i = start; i < start + per && i < nb; ++i) sum += row[i];
  uint32_t tot;
  uint32_t run = block_exclusive_scan256(sum, s_warp, &tot);
  for (int i = start; i < start + per && i < nb; ++i) {
    uint32_t c = row[i];
    row[i] = run;
    run += c;
  }
  if (threadIdx.x == 0) totals[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kRsThreads) k_rs_downsweep(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    uint32_t* __restrict__ vout, int64_t n, int shift, const uint32_t* __restrict__ counts,
    const uint32_t* __restrict__ totals, int nb) {
  __shared__ uint32_t whist[8][256];
  __shared__ uint32_t goff[256];
  __shared__ uint32_t s_warp[16];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < 8 * 256; t += kRsThreads) (&whist[0][0])[t] = 0;
  uint32_t tot = totals[threadIdx.x];
  uint32_t digit_base = block_exclusive_scan256(tot, s_warp, nullptr);
  goff[threadIdx.x] = digit_base + counts[(int64_t)threadIdx.x * nb + blockIdx.x];
  __syncthreads();

  const int64_t base = (int64_t)blockIdx.x * kRsTile + (int64_t)w * (32 * kRsItems);
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t key[kRsItems], val[kRsItems], rank[kRsItems];
#pragma unroll
  for (int j = 0; j < kRsItems; ++j) {
    int64_t i = base + j * 32 + lane;
    bool v = i < n;
    key[j] = v ? kin[i] : 0u;
    val[j] = v ? vin[i] : 0u;
  }
#pragma unroll
  for (int j = 0; j < kRsItems; ++j) {
    int64_t i = base + j * 32 + lane;
    bool v = i < n;
    uint32_t dig = v ? ((key[j] >> shift) & 0xffu) : 0x100u;
    uint32_t peers = __match_any_sync(0xffffffffu, dig);
    int leader = 31 - __clz(peers);
    uint32_t b = v ? whist[w][dig] : 0u;
    __syncwarp();
    if (v && lane == leader) whist[w][dig] = b + (uint32_t)__popc(peers);
    __syncwarp();
    rank[j] = b + (uint32_t)__popc(peers & lt);
  }
  __syncthreads();
  {   // per digit: exclusive prefix over warps (warp order = input order)
    uint32_t run = 0;
    for (int ww = 0; ww < 8; ++ww) {
      uint32_t c = whist[ww][threadIdx.x];
      whist[ww][threadIdx.x] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kRsItems; ++j) {
    int64_t i = base + j * 32 + lane;
    if (i < n) {
      uint32_t dig = (key[j] >> shift) & 0xffu;
      uint32_t pos = goff[dig] + whist[w][dig] + rank[j];
      kout[pos] = key[j];
      vout[pos] = val[j];
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
  // padding slots (i >= n) repeat the last sorted point; they are never labelled
  int64_t src = order[i < n ? i : n - 1];
  xs[i] = p[src * d + 0];
  ys[i] = p[src * d + 1];
  if (d == 3) zs[i] = p[src * d + 2];
}

// ---------------------------------------------------------------------------
// per-tile and per-block AABBs (one CTA per block, one warp per tile)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlockThreads) k_boxes(const float* __restrict__ xs,
                                                         const float* __restrict__ ys,
                                                         const float* __restrict__ zs, int64_t n,
                                                         int d, float4* __restrict__ tbox,
                                                         float4* __restrict__ bbox) {
  __shared__ float4 s_lo[kWarpsPerBlock], s_hi[kWarpsPerBlock];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t tile = (int64_t)blockIdx.x * kWarpsPerBlock + w;
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int j = 0; j < kTilePts / 32; ++j) {
    int64_t i = tile * kTilePts + j * 32 + lane;
    if (i < n) {
      float v0 = xs[i], v1 = ys[i], v2 = d == 3 ? zs[i] : 0.f;
      lo[0] = fminf(lo[0], v0); hi[0] = fmaxf(hi[0], v0);
      lo[1] = fminf(lo[1], v1); hi[1] = fmaxf(hi[1], v1);
      lo[2] = fminf(lo[2], v2); hi[2] = fmaxf(hi[2], v2);
    }
  }
  for (int a = 0; a < 3; ++a) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
      hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
    }
  }
  if (lane == 0) {
    float4 l = make_float4(lo[0], lo[1], lo[2], 0.f), h = make_float4(hi[0], hi[1], hi[2], 0.f);
    tbox[2 * tile] = l;
    tbox[2 * tile + 1] = h;
    s_lo[w] = l;
    s_hi[w] = h;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float4 l = s_lo[0], h = s_hi[0];
    for (int ww = 1; ww < kWarpsPerBlock; ++ww) {
      l.x = fminf(l.x, s_lo[ww].x); l.y = fminf(l.y, s_lo[ww].y); l.z = fminf(l.z, s_lo[ww].z);
      h.x = fmaxf(h.x, s_hi[ww].x); h.y = fmaxf(h.y, s_hi[ww].y); h.z = fmaxf(h.z, s_hi[ww].z);
    }
    bbox[2 * blockIdx.x] = l;
    bbox[2 * blockIdx.x + 1] = h;
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

cudaError_t launch_bbox(const float* p, int64_t n, int d, DevState* st, int which, int d_ctx,
                        cudaStream_t s) {
  k_reset_boxes<<<1, 32, 0, s>>>(st, d_ctx, which == 0 ? 1 : 2);
  k_bbox<<<grid_for(n, 256, 152 * 8), 256, 0, s>>>(p, n, d, st, which);
  return cudaGetLastError();
}

cudaError_t launch_morton(const float* p, int64_t n, int d, const float* lo, float inv,
                          uint32_t* keys, uint32_t* vals, cudaStream_t s) {
  float3 l = make_float3(lo[0], lo[1], d == 3 ? lo[2] : 0.f);
  k_morton<<<grid_for(n, 256, 1 << 30), 256, 0, s>>>(p, n, d, l, inv, keys, vals);
  return cudaGetLastError();
}

int64_t radix_sort_nb(int64_t n) { return (n + kRsTile - 1) / kRsTile; }

cudaError_t launch_radix_sort(uint32_t* keys[2], uint32_t* vals[2], int64_t n, int bits,
                              uint32_t* counts, uint32_t* totals, int* final_buf,
                              cudaStream_t s) {
  int nb = (int)radix_sort_nb(n);
  int cur = 0;
  for (int shift = 0; shift < bits; shift += 8) {
    k_rs_upsweep<<<nb, kRsThreads, 0, s>>>(keys[cur], n, shift, counts, nb);
    k_rs_scan<<<256, 256, 0, s>>>(counts, nb, totals);
    k_rs_downsweep<<<nb, kRsThreads, 0, s>>>(keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1],
                                             n, shift, counts, totals, nb);
    cur ^= 1;
  }
  *final_buf = cur;
  return cudaGetLastError();
}

cudaError_t launch_gather(const float* p, int64_t n, int d, const uint32_t* order, float* xs,
                          float* ys, float* zs, int64_t n_pad, cudaStream_t s) {
  k_gather<<<grid_for(n_pad, 256, 1 << 30), 256, 0, s>>>(p, n, d, order, xs, ys, zs, n_pad);
  return cudaGetLastError();
}

cudaError_t launch_boxes(const float* xs, const float* ys, const float* zs, int64_t n, int d,
                         int n_blocks, float4* tbox, float4* bbox, cudaStream_t s) {
  k_boxes<<<n_blocks, kBlockThreads, 0, s>>>(xs, ys, zs, n, d, tbox, bbox);
  return cudaGetLastError();
}

}  // namespace dkm
