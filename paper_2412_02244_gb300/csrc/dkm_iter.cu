// dkm_iter.cu -- per-iteration kernels of libdkm (sm_103a).
//
// One Lloyd iteration (Algorithm 1 loop body) is three launches:
//
//   k_search   per block of 2048 Morton-sorted points: find every centroid
//              that can be the nearest one of some point in the block's
//              AABB (the batch pruning of Section IV-A) using the
//              per-iteration centroid grid; write the list sorted by id.
//   k_assign   per point: nearest candidate (ties -> lowest id), label
//              store, and the per-cluster residual sums for the update,
//              aggregated per warp by label and added with integer
//              atomics (exact, order independent).  The BRUTE instance is
//              plain Lloyd: every point against every centroid.
//   k_centroids  refine c_j = c_j + sum(p - c_j)/|S_j| (= the cluster
//              mean; an empty cluster keeps c_j) and rebuild the centroid
//              grid for the next pass.
//
// Distances: d^2 = fma(dz, dz, fma(dy, dy, dx*dx)), dx = p + (-c), each
// step rounded to nearest in FP32; the same expression in every kernel, so
// the indexed and brute-force paths give bit-identical labels.
#include "dkm_host.h"

namespace dkm {

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_min_nonneg(float v) {
  // non-negative floats order like their bit patterns
  return __uint_as_float(__reduce_min_sync(0xffffffffu, __float_as_uint(v)));
}
__device__ __forceinline__ float warp_max_nonneg(float v) {
  return __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(v)));
}

__device__ __forceinline__ void red_add_u64(unsigned long long* p, unsigned long long v) {
  atomicAdd(p, v);
}

// Reduce the spread slots into the run history / last-pass counters and
// clear them.  Called by one full CTA of kBlockThreads threads.
//   t >= 0: pass t of a run (history + early-stop flag)
//   t == -1: a single pass outside a run
//   t == -2: the final-SSE pass of a run (only final_sse is written)
__device__ void collect_slots(const IterArgs& A, int t) {
  __shared__ unsigned long long s_part[5][kBlockThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long v[5] = {0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < kSlots; i += blockDim.x) {
    Slot& s = A.slots[i];
    v[0] += s.sse; v[1] += s.changed; v[2] += s.evals; v[3] += s.cands; v[4] += s.fallback;
    s.sse = 0; s.changed = 0; s.evals = 0; s.cands = 0; s.fallback = 0;
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    if (lane == 0) s_part[q][w] = v[q];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tot[5] = {0, 0, 0, 0, 0};
    for (int q = 0; q < 5; ++q)
      for (int ww = 0; ww < (int)(blockDim.x / 32); ++ww) tot[q] += s_part[q][ww];
    int s_glob, s_sse;
    fixed_exponents(A.st, A.n, &s_glob, &s_sse);
    double sse = (double)(long long)tot[0] * exp2(-(double)s_sse);
    if (t == -2) {   // final SSE of a run: leave the last-pass counters alone
      A.st->final_sse = sse;
      return;
    }
    A.st->last_sse = sse;
    A.st->last_changed = tot[1];
    A.st->last_evals = tot[2];
    A.st->last_cands = tot[3];
    A.st->last_fallback = tot[4];
    if (t >= 0) {
      A.sse_hist[t] = sse;
      A.chg_hist[t] = tot[1];
      if (A.early_stop && tot[1] == 0) A.st->done = 1;
    }
  }
}

__global__ void __launch_bounds__(kBlockThreads) k_collect(IterArgs A, int t) {
  collect_slots(A, t);
}

__global__ void k_reset_run(DevState* st) {
  st->done = 0;
  st->passes = 0;
  st->err = 0;
  st->label_err = 0;
  st->grid_ovf = 0;
}

// ---------------------------------------------------------------------------
// k_centroids: prep (copy user centroids in) or update (refine), then
// optionally insert every centroid into grid parity `par`.
//   mode 0: cw[j] = user_c[j]
//   mode 1: cw[j] += acc mean residual (if the cluster is non-empty); acc cleared
// With t >= 0 (inside a run) an update only happens if pass t ran, and
// CTA 0 first folds the pass's slot counters into the history.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlockThreads) k_centroids(IterArgs A, int mode, int t, int d,
                                                             const float* __restrict__ user_c,
                                                             int insert, int par,
                                                             int32_t* __restrict__ counts_out) {
  if (mode == 1 && t >= 0 && A.st->passes != t + 1) return;   // stopped early
  if (mode == 1 && t >= 0 && blockIdx.x == 0) collect_slots(A, t);
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= A.k) return;
  float4 c;
  if (mode == 0) {
    c.x = user_c[(int64_t)j * d + 0];
    c.y = user_c[(int64_t)j * d + 1];
    c.z = d == 3 ? user_c[(int64_t)j * d + 2] : 0.f;
    c.w = __int_as_float(j);
  } else {
    c = A.cw[j];
    Acc a = A.acc[j];
    A.acc[j] = Acc{{0ull, 0ull, 0ull}, 0ull};
    long long cnt = (long long)a.cnt;
    if (counts_out) counts_out[j] = (int32_t)cnt;
    if (cnt > 0) {
      int s_glob, s_sse;
      fixed_exponents(A.st, A.n, &s_glob, &s_sse);
      const double u = exp2(-(double)s_glob) / (double)cnt;
      c.x = (float)((double)c.x + (double)(long long)a.s[0] * u);
      c.y = (float)((double)c.y + (double)(long long)a.s[1] * u);
      if (d == 3) c.z = (float)((double)c.z + (double)(long long)a.s[2] * u);
    }
  }
  A.cw[j] = c;
  if (insert) {
    const Grid& G = A.grid;
    int cx = cell_coord(c.x, G.g0[0], G.inv_s, G.dims[0]);
    int cy = cell_coord(c.y, G.g0[1], G.inv_s, G.dims[1]);
    int cz = d == 3 ? cell_coord(c.z, G.g0[2], G.inv_s, G.dims[2]) : 0;
    long long cell = ((long long)cz * G.dims[1] + cy) * G.dims[0] + cx;
    int slot = atomicAdd(&A.gcnt[par][cell], 1);
    if (slot < G.cap) {
      A.gbkt[par][cell * G.cap + slot] = c;
    } else {
      int o = atomicAdd(&A.ovf_cnt[par], 1);
      A.ovf[par][o] = c;
      atomicAdd(&A.st->grid_ovf, 1ull);
    }
  }
}

// ---------------------------------------------------------------------------
// k_search: one warp per block of 2048 points.
//   phase A: U^2 = min over centroids in the block's own cells (growing
//            rings if empty) of maxd^2(block box, c) -- any centroid gives
//            an upper bound on every point's nearest distance;
//   phase B: every centroid with mind^2(block box, c) <= U^2 * kKeep, found
//            in the cells overlapping the box grown by U, plus the
//            overflow list.  The true nearest centroid of each point in the
//            box always passes (its distance is <= the distance to the
//            U-defining centroid <= U), which is the ball-node test of
//            Section II-B / IV-A with boxes in place of balls.
// The list is written sorted by centroid id, so a strict < scan gives the
// lowest index on ties.
// ---------------------------------------------------------------------------
constexpr int kSearchWarps = 8;

__device__ __forceinline__ long long cell_index(const Grid& G, int cx, int cy, int cz) {
  return ((long long)cz * G.dims[1] + cy) * G.dims[0] + cx;
}

__global__ void __launch_bounds__(32 * kSearchWarps) k_search(IterArgs A, int par, int d) {
  __shared__ float4 s_list[kSearchWarps][kMaxCand];
  if (A.early_stop && A.st->done) return;
  // clear the other parity's grid for the next rebuild (nobody reads it now)
  {
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c = g; c < A.grid.cells; c += stride) A.gcnt[par ^ 1][c] = 0;
    if (g == 0) A.ovf_cnt[par ^ 1] = 0;
  }
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int b = blockIdx.x * kSearchWarps + wl;
  if (b >= A.n_blocks) return;
  const Grid G = A.grid;
  const float4 lo = A.bbox[2 * b], hi = A.bbox[2 * b + 1];
  const int* __restrict__ gcnt = A.gcnt[par];
  const float4* __restrict__ gbkt = A.gbkt[par];
  const int n_ovf = A.ovf_cnt[par];
  const float4* __restrict__ ovf = A.ovf[par];

  int clo[3], chi[3];
  clo[0] = cell_coord(lo.x, G.g0[0], G.inv_s, G.dims[0]);
  chi[0] = cell_coord(hi.x, G.g0[0], G.inv_s, G.dims[0]);
  clo[1] = cell_coord(lo.y, G.g0[1], G.inv_s, G.dims[1]);
  chi[1] = cell_coord(hi.y, G.g0[1], G.inv_s, G.dims[1]);
  clo[2] = d == 3 ? cell_coord(lo.z, G.g0[2], G.inv_s, G.dims[2]) : 0;
  chi[2] = d == 3 ? cell_coord(hi.z, G.g0[2], G.inv_s, G.dims[2]) : 0;

  // ---- phase A ----
  float u2 = INFINITY;
  for (int ring = 0;; ring = ring ? 2 * ring : 1) {
    int rlo[3], rhi[3];
    long long ncell = 1;
    bool whole = true;
    for (int a = 0; a < 3; ++a) {
      rlo[a] = max(clo[a] - ring, 0);
      rhi[a] = min(chi[a] + ring, G.dims[a] - 1);
      whole = whole && rlo[a] == 0 && rhi[a] == G.dims[a] - 1;
      ncell *= (long long)(rhi[a] - rlo[a] + 1);
    }
    const int nx = rhi[0] - rlo[0] + 1, ny = rhi[1] - rlo[1] + 1;
    float m = INFINITY;
    for (long long q = lane; q < ncell; q += 32) {
      int cx = rlo[0] + (int)(q % nx);
      long long r = q / nx;
      int cy = rlo[1] + (int)(r % ny);
      int cz = rlo[2] + (int)(r / ny);
      long long cell = cell_index(G, cx, cy, cz);
      int cnt = min(gcnt[cell], G.cap);
      for (int e = 0; e < cnt; ++e) {
        float4 c = gbkt[cell * G.cap + e];
        m = fminf(m, maxd2(lo, hi, c.x, c.y, c.z, d));
      }
    }
    for (int q = lane; q < n_ovf; q += 32) {
      float4 c = ovf[q];
      m = fminf(m, maxd2(lo, hi, c.x, c.y, c.z, d));
    }
    u2 = warp_min_nonneg(m);
    if (u2 < INFINITY || whole) break;
  }
  if (!(u2 < INFINITY)) {   // no centroid anywhere: cannot happen for k >= 1
    if (lane == 0) {
      A.bcnt[b] = 0;
      atomicOr(&A.st->err, kErrNoCentroid);
    }
    return;
  }

  // ---- phase B ----
  const float u2k = u2 * kKeep;
  float mag = fmaxf(fmaxf(fabsf(lo.x), fabsf(hi.x)), fmaxf(fabsf(lo.y), fabsf(hi.y)));
  if (d == 3) mag = fmaxf(mag, fmaxf(fabsf(lo.z), fabsf(hi.z)));
  const float ul = sqrtf(u2k) * 1.00002f + 1e-5f * mag + 1e-30f;
  int rlo[3], rhi[3];
  rlo[0] = cell_coord(lo.x - ul, G.g0[0], G.inv_s, G.dims[0]);
  rhi[0] = cell_coord(hi.x + ul, G.g0[0], G.inv_s, G.dims[0]);
  rlo[1] = cell_coord(lo.y - ul, G.g0[1], G.inv_s, G.dims[1]);
  rhi[1] = cell_coord(hi.y + ul, G.g0[1], G.inv_s, G.dims[1]);
  rlo[2] = d == 3 ? cell_coord(lo.z - ul, G.g0[2], G.inv_s, G.dims[2]) : 0;
  rhi[2] = d == 3 ? cell_coord(hi.z + ul, G.g0[2], G.inv_s, G.dims[2]) : 0;
  const int nx = rhi[0] - rlo[0] + 1, ny = rhi[1] - rlo[1] + 1;
  const long long ncell = (long long)nx * ny * (rhi[2] - rlo[2] + 1);
  const unsigned lt = (1u << lane) - 1u;
  int count = 0;
  for (long long q0 = 0; q0 < ncell; q0 += 32) {
    long long q = q0 + lane;
    long long cell = 0;
    int cnt = 0;
    if (q < ncell) {
      int cx = rlo[0] + (int)(q % nx);
      long long r = q / nx;
      int cy = rlo[1] + (int)(r % ny);
      int cz = rlo[2] + (int)(r / ny);
      cell = cell_index(G, cx, cy, cz);
      cnt = min(gcnt[cell], G.cap);
    }
    const int cmax = __reduce_max_sync(0xffffffffu, cnt);
    for (int e = 0; e < cmax; ++e) {
      float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
      bool keep = false;
      if (e < cnt) {
        c = gbkt[cell * G.cap + e];
        keep = mind2(lo, hi, c.x, c.y, c.z, d) <= u2k;
      }
      unsigned bal = __ballot_sync(0xffffffffu, keep);
      int pos = count + __popc(bal & lt);
      if (keep && pos < kMaxCand) s_list[wl][pos] = c;
      count += __popc(bal);
    }
  }
  for (int q0 = 0; q0 < n_ovf; q0 += 32) {
    int q = q0 + lane;
    float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
    bool keep = false;
    if (q < n_ovf) {
      c = ovf[q];
      keep = mind2(lo, hi, c.x, c.y, c.z, d) <= u2k;
    }
    unsigned bal = __ballot_sync(0xffffffffu, keep);
    int pos = count + __popc(bal & lt);
    if (keep && pos < kMaxCand) s_list[wl][pos] = c;
    count += __popc(bal);
  }
  __syncwarp();
  if (count <= kMaxCand) {
    float4* out = A.blist + (int64_t)b * kMaxCand;
    for (int i = lane; i < count; i += 32) {
      float4 c = s_list[wl][i];
      int id = __float_as_int(c.w);
      int rank = 0;
      for (int j2 = 0; j2 < count; ++j2) rank += __float_as_int(s_list[wl][j2].w) < id;
      out[rank] = c;
    }
  }
  if (lane == 0) {
    A.bcnt[b] = count;
    Slot& s = A.slots[b & (kSlots - 1)];
    red_add_u64(&s.cands, (unsigned long long)count);
    if (count > kMaxCand) red_add_u64(&s.fallback, 1ull);
  }
}

// ---------------------------------------------------------------------------
// k_assign<D, BRUTE>: one CTA per block, one warp per tile of 4 rows x 64
// points, two points per lane evaluated as packed f32x2.
// ---------------------------------------------------------------------------
template <int D>
struct Pts {
  float2 x[kRowsPerWarp], y[kRowsPerWarp], z[kRowsPerWarp];
};

template <int D>
__device__ __forceinline__ void eval_list(const float4* __restrict__ s_c,
                                          const unsigned short* __restrict__ idx, int m,
                                          const Pts<D>& P, float2 (&best)[kRowsPerWarp],
                                          int2 (&bid)[kRowsPerWarp]) {
#pragma unroll 2
  for (int j = 0; j < m; ++j) {
    const float4 c = s_c[idx ? idx[j] : j];
    const int id = __float_as_int(c.w);
    const float2 nx = make_float2(-c.x, -c.x);
    const float2 ny = make_float2(-c.y, -c.y);
    const float2 nz = make_float2(-c.z, -c.z);
#pragma unroll
    for (int r = 0; r < kRowsPerWarp; ++r) {
      float2 dx = __fadd2_rn(P.x[r], nx);
      float2 dy = __fadd2_rn(P.y[r], ny);
      float2 s = __fmul2_rn(dx, dx);
      s = __ffma2_rn(dy, dy, s);
      if (D == 3) {
        float2 dz = __fadd2_rn(P.z[r], nz);
        s = __ffma2_rn(dz, dz, s);
      }
      if (s.x < best[r].x) { best[r].x = s.x; bid[r].x = id; }
      if (s.y < best[r].y) { best[r].y = s.y; bid[r].y = id; }
    }
  }
}

// Tile filter: U^2 of the tile box over the list, then the ids of the list
// entries that can be some point's nearest (ascending positions, so the
// filtered list stays sorted by id).  u2_run carries the bound across
// chunks (fallback path).  Returns the filtered length.
template <int D>
__device__ __forceinline__ int filter_tile(const float4* __restrict__ s_c, int q, float4 tlo,
                                           float4 thi, unsigned short* __restrict__ out,
                                           float& u2_run) {
  const int lane = threadIdx.x & 31;
  float m = INFINITY;
  for (int j = lane; j < q; j += 32) {
    float4 c = s_c[j];
    m = fminf(m, maxd2(tlo, thi, c.x, c.y, c.z, D));
  }
  u2_run = fminf(u2_run, warp_min_nonneg(m));
  const float u2k = u2_run * kKeep;
  const unsigned lt = (1u << lane) - 1u;
  int cnt = 0;
  for (int j0 = 0; j0 < q; j0 += 32) {
    int j = j0 + lane;
    bool keep = false;
    if (j < q) {
      float4 c = s_c[j];
      keep = mind2(tlo, thi, c.x, c.y, c.z, D) <= u2k;
    }
    unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (keep) out[cnt + __popc(bal & lt)] = (unsigned short)j;
    cnt += __popc(bal);
  }
  __syncwarp();
  return cnt;
}

// Row epilogue shared by k_assign and k_accum_labels: per-row fixed-point
// residual sums grouped by label, added to the per-centroid accumulators.
// la/lb are the labels of the lane's two points (valid flags va/vb).
__device__ __forceinline__ void accumulate_row(const IterArgs& A, int D, float2 px, float2 py,
                                               float2 pz, int la, int lb, bool va, bool vb,
                                               int s_glob) {
  float rxa = 0.f, rya = 0.f, rza = 0.f, rxb = 0.f, ryb = 0.f, rzb = 0.f;
  if (va) {
    float4 c = __ldg(&A.cw[la]);
    rxa = __fadd_rn(px.x, -c.x); rya = __fadd_rn(py.x, -c.y);
    if (D == 3) rza = __fadd_rn(pz.x, -c.z);
  }
  if (vb) {
    float4 c = __ldg(&A.cw[lb]);
    rxb = __fadd_rn(px.y, -c.x); ryb = __fadd_rn(py.y, -c.y);
    if (D == 3) rzb = __fadd_rn(pz.y, -c.z);
  }
  float ml = fmaxf(fmaxf(fmaxf(fabsf(rxa), fabsf(rya)), fabsf(rza)),
                   fmaxf(fmaxf(fabsf(rxb), fabsf(ryb)), fabsf(rzb)));
  float m = warp_max_nonneg(ml);
  // unit 2^-s_row with 64 * max|r| * 2^s_row < 2^30: int32 warp sums cannot overflow
  int s_row = m > 0.f ? min(24 - exp_bound(m), 127) : 0;
  float sc = pow2f(s_row);
  int qxa = __float2int_rn(rxa * sc), qya = __float2int_rn(rya * sc), qza = __float2int_rn(rza * sc);
  int qxb = __float2int_rn(rxb * sc), qyb = __float2int_rn(ryb * sc), qzb = __float2int_rn(rzb * sc);
  bool pa = va, pb = vb;
  const int lane = threadIdx.x & 31;
  while (true) {
    unsigned ma = __ballot_sync(0xffffffffu, pa);
    unsigned mb = __ballot_sync(0xffffffffu, pb);
    if (!(ma | mb)) break;
    int L = ma ? __shfl_sync(0xffffffffu, la, __ffs(ma) - 1)
               : __shfl_sync(0xffffffffu, lb, __ffs(mb) - 1);
    bool ga = pa && la == L, gb = pb && lb == L;
    int vx = (ga ? qxa : 0) + (gb ? qxb : 0);
    int vy = (ga ? qya : 0) + (gb ? qyb : 0);
    int vz = (ga ? qza : 0) + (gb ? qzb : 0);
    int cnt = __popc(__ballot_sync(0xffffffffu, ga)) + __popc(__ballot_sync(0xffffffffu, gb));
    int sx = __reduce_add_sync(0xffffffffu, vx);
    int sy = __reduce_add_sync(0xffffffffu, vy);
    int sz = D == 3 ? __reduce_add_sync(0xffffffffu, vz) : 0;
    if (lane == 0) {
      Acc* a = &A.acc[L];
      red_add_u64(&a->s[0], (unsigned long long)rescale(sx, s_row, s_glob));
      red_add_u64(&a->s[1], (unsigned long long)rescale(sy, s_row, s_glob));
      if (D == 3) red_add_u64(&a->s[2], (unsigned long long)rescale(sz, s_row, s_glob));
      red_add_u64(&a->cnt, (unsigned long long)cnt);
    }
    pa = pa && !ga;
    pb = pb && !gb;
  }
}

// per-row SSE in fixed point (unit 2^-s_sse), identical on every lane
__device__ __forceinline__ long long row_sse(float d2a, float d2b, bool va, bool vb, int s_sse) {
  float a = va ? d2a : 0.f, b = vb ? d2b : 0.f;
  float m = warp_max_nonneg(fmaxf(a, b));
  int s2 = m > 0.f ? min(24 - exp_bound(m), 127) : 0;
  float sc = pow2f(s2);
  unsigned q = (unsigned)__float2uint_rn(a * sc) + (unsigned)__float2uint_rn(b * sc);
  unsigned s = __reduce_add_sync(0xffffffffu, q);
  return rescale((long long)s, s2, s_sse);
}

__device__ __forceinline__ void load_points(const IterArgs& A, int D, int64_t tile_base,
                                            float2 (&x)[kRowsPerWarp], float2 (&y)[kRowsPerWarp],
                                            float2 (&z)[kRowsPerWarp], bool (&va)[kRowsPerWarp],
                                            bool (&vb)[kRowsPerWarp]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r) {
    int64_t i = tile_base + r * kRowPts + 2 * lane;
    // arrays are padded to a whole block, so the pair load is always in bounds
    x[r] = *reinterpret_cast<const float2*>(A.xs + i);
    y[r] = *reinterpret_cast<const float2*>(A.ys + i);
    z[r] = D == 3 ? *reinterpret_cast<const float2*>(A.zs + i) : make_float2(0.f, 0.f);
    va[r] = i < A.n;
    vb[r] = i + 1 < A.n;
  }
}

template <int D, bool BRUTE>
__global__ void __launch_bounds__(kBlockThreads) k_assign(IterArgs A) {
  __shared__ float4 s_c[kChunk];
  __shared__ unsigned short s_w[kWarpsPerBlock][kChunk];
  if (A.early_stop && A.st->done) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int b = blockIdx.x;
  const int64_t tile = (int64_t)b * kWarpsPerBlock + w;
  const int64_t tile_base = tile * kTilePts;
  const bool tile_live = tile_base < A.n;
  if (b == 0 && threadIdx.x == 0) atomicAdd(&A.st->passes, 1);

  Pts<D> P;
  bool va[kRowsPerWarp], vb[kRowsPerWarp];
  load_points(A, D, tile_base, P.x, P.y, P.z, va, vb);

  float2 best[kRowsPerWarp];
  int2 bid[kRowsPerWarp];
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r) {
    best[r] = make_float2(INFINITY, INFINITY);
    bid[r] = make_int2(0, 0);
  }
  unsigned long long evals = 0;
  float4 tlo = make_float4(0.f, 0.f, 0.f, 0.f), thi = tlo;
  if (!BRUTE && tile_live) {
    tlo = A.tbox[2 * tile];
    thi = A.tbox[2 * tile + 1];
  }
  bool chunked = BRUTE;
  if (!BRUTE) {
    const int q = A.bcnt[b];
    if (q <= kMaxCand) {
      const float4* src = A.blist + (int64_t)b * kMaxCand;
      for (int i = threadIdx.x; i < q; i += kBlockThreads) s_c[i] = src[i];
      __syncthreads();
      if (tile_live) {
        float u2 = INFINITY;
        int m = filter_tile<D>(s_c, q, tlo, thi, s_w[w], u2);
        if (m == 0 && lane == 0) atomicOr(&A.st->err, kErrEmptyList);
        eval_list<D>(s_c, s_w[w], m, P, best, bid);
        evals += (unsigned long long)m;
      }
    } else {
      chunked = true;
    }
  }
  if (chunked) {
    float u2 = INFINITY;
    for (int c0 = 0; c0 < A.k; c0 += kChunk) {
      const int m = min(kChunk, A.k - c0);
      __syncthreads();
      for (int i = threadIdx.x; i < m; i += kBlockThreads) s_c[i] = A.cw[c0 + i];
      __syncthreads();
      if (tile_live) {
        if (BRUTE) {
          eval_list<D>(s_c, nullptr, m, P, best, bid);
          evals += (unsigned long long)m;
        } else {
          int mm = filter_tile<D>(s_c, m, tlo, thi, s_w[w], u2);
          eval_list<D>(s_c, s_w[w], mm, P, best, bid);
          evals += (unsigned long long)mm;
        }
      }
    }
  }
  if (!tile_live) return;

  int s_glob, s_sse;
  fixed_exponents(A.st, A.n, &s_glob, &s_sse);
  long long sse = 0;
  int changed = 0;
  int nvalid = 0;
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r) {
    const int64_t i = tile_base + r * kRowPts + 2 * lane;
    if (tile_base + r * kRowPts >= A.n) break;   // warp-uniform
    const int la = bid[r].x, lb = bid[r].y;
    if (A.track_changes) {
      int pa = va[r] ? A.lab[i] : la, pb = vb[r] ? A.lab[i + 1] : lb;
      changed += (int)(pa != la) + (int)(pb != lb);
    }
    if (va[r] && vb[r]) {
      *reinterpret_cast<int2*>(A.lab + i) = make_int2(la, lb);
    } else if (va[r]) {
      A.lab[i] = la;
    }
    nvalid += (int)va[r] + (int)vb[r];
    sse += row_sse(best[r].x, best[r].y, va[r], vb[r], s_sse);
    accumulate_row(A, D, P.x[r], P.y[r], P.z[r], la, lb, va[r], vb[r], s_glob);
  }
  changed = __reduce_add_sync(0xffffffffu, changed);
  nvalid = __reduce_add_sync(0xffffffffu, nvalid);
  if (lane == 0) {
    Slot& s = A.slots[tile & (kSlots - 1)];
    red_add_u64(&s.sse, (unsigned long long)sse);
    if (changed) red_add_u64(&s.changed, (unsigned long long)changed);
    red_add_u64(&s.evals, evals * (unsigned long long)nvalid);
  }
}

// ---------------------------------------------------------------------------
// k_accum_labels: residual sums for a caller-given labelling (dkm_update).
// ---------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(kBlockThreads) k_accum_labels(IterArgs A,
                                                               const int32_t* __restrict__ ulab,
                                                               const uint32_t* __restrict__ perm) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t tile = (int64_t)blockIdx.x * kWarpsPerBlock + w;
  const int64_t tile_base = tile * kTilePts;
  if (tile_base >= A.n) return;
  float2 x[kRowsPerWarp], y[kRowsPerWarp], z[kRowsPerWarp];
  bool va[kRowsPerWarp], vb[kRowsPerWarp];
  load_points(A, D, tile_base, x, y, z, va, vb);
  int s_glob, s_sse;
  fixed_exponents(A.st, A.n, &s_glob, &s_sse);
  int bad = 0;
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r) {
    const int64_t i = tile_base + r * kRowPts + 2 * lane;
    if (tile_base + r * kRowPts >= A.n) break;
    int la = va[r] ? ulab[perm[i]] : 0;
    int lb = vb[r] ? ulab[perm[i + 1]] : 0;
    bool oka = va[r] && la >= 0 && la < A.k, okb = vb[r] && lb >= 0 && lb < A.k;
    bad |= (va[r] && !oka) || (vb[r] && !okb);
    accumulate_row(A, D, x[r], y[r], z[r], oka ? la : 0, okb ? lb : 0, oka, okb, s_glob);
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&A.st->label_err, 1);
}

// ---------------------------------------------------------------------------
// k_finalize: labels back to the caller's order; optional SSE against the
// current centroids (same FP32 distance expression, fixed-point sum).
// ---------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(kBlockThreads) k_finalize(IterArgs A,
                                                           const uint32_t* __restrict__ perm,
                                                           int32_t* __restrict__ labels_out,
                                                           int do_sse) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t tile = (int64_t)blockIdx.x * kWarpsPerBlock + w;
  const int64_t tile_base = tile * kTilePts;
  if (tile_base >= A.n) return;
  int s_glob, s_sse;
  fixed_exponents(A.st, A.n, &s_glob, &s_sse);
  long long sse = 0;
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r) {
    const int64_t i = tile_base + r * kRowPts + 2 * lane;
    if (tile_base + r * kRowPts >= A.n) break;
    const bool va = i < A.n, vb = i + 1 < A.n;
    const int la = va ? A.lab[i] : 0, lb = vb ? A.lab[i + 1] : 0;
    if (labels_out) {
      if (va) labels_out[perm[i]] = la;
      if (vb) labels_out[perm[i + 1]] = lb;
    }
    if (do_sse) {
      float d2a = 0.f, d2b = 0.f;
      if (va) {
        float4 c = __ldg(&A.cw[la]);
        float dx = __fadd_rn(A.xs[i], -c.x), dy = __fadd_rn(A.ys[i], -c.y);
        d2a = __fmaf_rn(dy, dy, __fmul_rn(dx, dx));
        if (D == 3) { float dz = __fadd_rn(A.zs[i], -c.z); d2a = __fmaf_rn(dz, dz, d2a); }
      }
      if (vb) {
        float4 c = __ldg(&A.cw[lb]);
        float dx = __fadd_rn(A.xs[i + 1], -c.x), dy = __fadd_rn(A.ys[i + 1], -c.y);
        d2b = __fmaf_rn(dy, dy, __fmul_rn(dx, dx));
        if (D == 3) { float dz = __fadd_rn(A.zs[i + 1], -c.z); d2b = __fmaf_rn(dz, dz, d2b); }
      }
      sse += row_sse(d2a, d2b, va, vb, s_sse);
    }
  }
  if (do_sse && lane == 0) red_add_u64(&A.slots[tile & (kSlots - 1)].sse, (unsigned long long)sse);
}

__global__ void k_export(const float4* __restrict__ cw, int k, int d, float* __restrict__ out) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  float4 c = cw[j];
  out[(int64_t)j * d + 0] = c.x;
  out[(int64_t)j * d + 1] = c.y;
  if (d == 3) out[(int64_t)j * d + 2] = c.z;
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

cudaError_t launch_reset_run(DevState* st, cudaStream_t s) {
  k_reset_run<<<1, 1, 0, s>>>(st);
  return cudaGetLastError();
}

cudaError_t launch_centroids(const IterArgs& A, int mode, int t, int d, const float* user_c,
                             int insert, int par, int32_t* counts_out, cudaStream_t s) {
  k_centroids<<<ceil_div(A.k, kBlockThreads), kBlockThreads, 0, s>>>(A, mode, t, d, user_c, insert,
                                                                    par, counts_out);
  return cudaGetLastError();
}

cudaError_t launch_search(const IterArgs& A, int par, int d, cudaStream_t s) {
  k_search<<<ceil_div(A.n_blocks, kSearchWarps), 32 * kSearchWarps, 0, s>>>(A, par, d);
  return cudaGetLastError();
}

cudaError_t launch_assign(const IterArgs& A, int d, int brute, cudaStream_t s) {
  if (d == 3) {
    if (brute) k_assign<3, true><<<A.n_blocks, kBlockThreads, 0, s>>>(A);
    else k_assign<3, false><<<A.n_blocks, kBlockThreads, 0, s>>>(A);
  } else {
    if (brute) k_assign<2, true><<<A.n_blocks, kBlockThreads, 0, s>>>(A);
    else k_assign<2, false><<<A.n_blocks, kBlockThreads, 0, s>>>(A);
  }
  return cudaGetLastError();
}

cudaError_t launch_collect(const IterArgs& A, int t, cudaStream_t s) {
  k_collect<<<1, kBlockThreads, 0, s>>>(A, t);
  return cudaGetLastError();
}

cudaError_t launch_accum_labels(const IterArgs& A, int d, const int32_t* ulab,
                                const uint32_t* perm, cudaStream_t s) {
  if (d == 3) k_accum_labels<3><<<A.n_blocks, kBlockThreads, 0, s>>>(A, ulab, perm);
  else k_accum_labels<2><<<A.n_blocks, kBlockThreads, 0, s>>>(A, ulab, perm);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const IterArgs& A, int d, const uint32_t* perm, int32_t* labels_out,
                            int do_sse, cudaStream_t s) {
  if (d == 3) k_finalize<3><<<A.n_blocks, kBlockThreads, 0, s>>>(A, perm, labels_out, do_sse);
  else k_finalize<2><<<A.n_blocks, kBlockThreads, 0, s>>>(A, perm, labels_out, do_sse);
  return cudaGetLastError();
}

cudaError_t launch_export(const float4* cw, int k, int d, float* out, cudaStream_t s) {
  k_export<<<ceil_div(k, 256), 256, 0, s>>>(cw, k, d, out);
  return cudaGetLastError();
}

}  // namespace dkm
