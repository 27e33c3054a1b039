// dkm_iter.cu -- per-iteration kernels of libdkm (sm_103a).
//
// One Lloyd iteration (Algorithm 1 loop body) is three launches:
//
//   k_search     per tile (<= 256 Morton-sorted points inside one Morton
//                cube): every centroid that can be the nearest one of some
//                point in the tile's AABB (the batch pruning of Section
//                IV-A), found through the per-iteration centroid grid.
//   k_assign     per point: nearest candidate (ties -> lowest id), label
//                store, and the per-cluster residual sums for the update,
//                aggregated per warp by label and added with integer
//                atomics (exact, order independent).  The BRUTE instance is
//                plain Lloyd: every point against every centroid.
//   k_centroids  refine c_j = c_j + sum(p - c_j)/|S_j| (= the cluster
//                mean; an empty cluster keeps c_j) and rebuild the centroid
//                grid for the next pass.
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

// Fold the counters of a pass, per cloud (SSE, changed labels, early stop
// -> CloudRun) and in total (run history, last-pass statistics), and clear
// them.  Called by one full CTA of kBlockThreads threads.
//   t >= 0: pass t of a run (only clouds that executed it)
//   t == -1: a single pass outside a run
//   t == -2: the final-SSE pass of a run (only the final SSEs are written)
// Sums over clouds run in a fixed order, so the totals are deterministic.
__device__ void collect_pass(const IterArgs& A, int t) {
  __shared__ double s_sse[kBlockThreads / 32];
  __shared__ unsigned long long s_part[6][kBlockThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double sse = 0.0;
  unsigned long long v[6] = {0, 0, 0, 0, 0, 0};   // changed, evals, cands, fallback, clouds run, stays
  for (int b = threadIdx.x; b < A.B; b += blockDim.x) {
    CloudRun& r = A.crun[b];
    if (t >= 0 && r.passes != t + 1) continue;   // the cloud stopped earlier
    CloudAcc& a = A.cacc[b];
    unsigned long long qs = 0, qc = 0;
#pragma unroll
    for (int q = 0; q < kCloudSlots; ++q) {
      qs += a.sse[q];
      qc += a.changed[q];
      a.sse[q] = 0;
      a.changed[q] = 0;
    }
    const double e = (double)(long long)qs * exp2(-(double)r.s_sse);
    sse += e;
    if (t == -2) {
      r.final_sse = e;
      continue;
    }
    r.last_sse = e;
    r.last_changed = qc;
    v[0] += qc;
    v[4] += 1;
    if (t >= 0 && A.early_stop && qc == 0) {
      r.done = 1;
      atomicAdd(&A.st->n_done, 1);
    }
  }
  if (t != -2) {
    for (int i = threadIdx.x; i < kSlots; i += blockDim.x) {
      Slot& s = A.slots[i];
      v[1] += s.evals; v[2] += s.cands; v[3] += s.fallback; v[5] += s.stays;
      s.evals = 0; s.cands = 0; s.fallback = 0; s.stays = 0;
    }
  }
  for (int o = 16; o > 0; o >>= 1) sse += __shfl_xor_sync(0xffffffffu, sse, o);
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    if (lane == 0) s_part[q][w] = v[q];
  }
  if (lane == 0) s_sse[w] = sse;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tot[6] = {0, 0, 0, 0, 0, 0};
    double tsse = 0.0;
    for (int ww = 0; ww < (int)(blockDim.x / 32); ++ww) {
      tsse += s_sse[ww];
      for (int q = 0; q < 6; ++q) tot[q] += s_part[q][ww];
    }
    if (t == -2) {   // final SSE of a run: leave the last-pass counters alone
      A.st->final_sse = tsse;
    } else {
      A.st->last_sse = tsse;
      A.st->last_changed = tot[0];
      A.st->last_evals = tot[1];
      A.st->last_cands = tot[2];
      A.st->last_fallback = tot[3];
      A.st->last_stays = tot[5];
      A.st->last_tiles = (unsigned long long)A.n_tiles;
      if (t >= 0 && tot[4] > 0) {
        A.sse_hist[t] = tsse;
        A.chg_hist[t] = tot[0];
        A.st->passes = t + 1;
      }
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kBlockThreads) k_collect(IterArgs A, int t) {
  collect_pass(A, t);
}

// clear the run state of the context and of every cloud
__global__ void k_reset_run(DevState* st, CloudRun* crun, CloudAcc* cacc, int B) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b == 0) {
    st->n_done = 0;
    st->passes = 0;
    st->err = 0;
    st->label_err = 0;
    st->grid_ovf = 0;
  }
  if (b >= B) return;
  crun[b].done = 0;
  crun[b].passes = 0;
  crun[b].last_changed = 0;
  crun[b].last_sse = 0.0;
  crun[b].final_sse = 0.0;
  for (int q = 0; q < kCloudSlots; ++q) {
    cacc[b].sse[q] = 0;
    cacc[b].changed[q] = 0;
  }
}

// ---------------------------------------------------------------------------
// k_centroids: prep (copy user centroids in) or update (refine), then
// optionally insert every centroid into its cloud's grid of parity `par`.
//   mode 0: cw[j] = user_c[j]
//   mode 1: cw[j] += acc mean residual (if the cluster is non-empty); acc cleared
// With t >= 0 (inside a run) a cloud's centroids are only updated if the
// cloud executed pass t, and CTA 0 first folds the pass's counters.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlockThreads) k_centroids(IterArgs A, int mode, int t, int d,
                                                             const float* __restrict__ user_c,
                                                             int insert, int par,
                                                             int32_t* __restrict__ counts_out) {
  // (no kernel-wide early exit: n_done changes inside this kernel, so only
  // the per-cloud pass counts, fixed since k_assign, decide what runs)
  if (mode == 1 && t >= 0 && blockIdx.x == 0 && (A.want_stats || A.early_stop))
    collect_pass(A, t);
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= A.k) return;
  const int b = A.kcloud[j];
  if (mode == 1 && t >= 0 && A.crun[b].passes != t + 1) return;   // stopped earlier
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
      const double u = exp2(-(double)A.crun[b].s_glob) / (double)cnt;
      c.x = (float)((double)c.x + (double)(long long)a.s[0] * u);
      c.y = (float)((double)c.y + (double)(long long)a.s[1] * u);
      if (d == 3) c.z = (float)((double)c.z + (double)(long long)a.s[2] * u);
    }
  }
  A.cw[j] = c;
  if (insert) {
    const Cloud& cl = A.clouds[b];
    const Grid& G = cl.grid;
    int cx = cell_coord(c.x, G.g0[0], G.inv_s, G.dims[0]);
    int cy = cell_coord(c.y, G.g0[1], G.inv_s, G.dims[1]);
    int cz = d == 3 ? cell_coord(c.z, G.g0[2], G.inv_s, G.dims[2]) : 0;
    long long cell = cl.cell0 + ((long long)cz * G.dims[1] + cy) * G.dims[0] + cx;
    int slot = atomicAdd(&A.gcnt[par][cell], 1);
    if (slot < kBucketCap) {
      A.gbkt[par][cell * kBucketCap + slot] = c;
    } else {
      int o = atomicAdd(&A.ovf_cnt[par][b], 1);
      A.ovf[par][cl.c0 + o] = c;
      atomicAdd(&A.st->grid_ovf, 1ull);
    }
  }
}

// ---------------------------------------------------------------------------
// k_search: one warp per tile.
//   phase A: U^2 = min over centroids in the tile's own cells (growing
//            rings if empty) of maxd^2(tile box, c) -- any centroid gives
//            an upper bound on every point's nearest distance;
//   phase B: every centroid with mind^2(tile box, c) <= U^2 * kKeep, found
//            in the cells overlapping the box grown by U, plus the
//            overflow list.  The true nearest centroid of each point in the
//            box always passes (its distance is <= the distance to the
//            U-defining centroid <= U): the ball-node test of Section II-B /
//            IV-A with boxes in place of balls.  A centroid that passes is
//            still dropped when the U-defining centroid r1 dominates it over
//            the whole box (dominated(): every point of the box is closer
//            to r1), which no nearest centroid can be.
// The list is written unordered; k_assign picks the lexicographic minimum
// of (d^2, id), which does not depend on the order.
// ---------------------------------------------------------------------------
constexpr int kSearchWarps = 2;   // independent warps: small CTAs free SM slots early
#ifndef DKM_SEARCH_MIN_BLOCKS
#define DKM_SEARCH_MIN_BLOCKS 20   // 48 registers: many resident warps hide the dependent loads
#endif

__device__ __forceinline__ long long cell_index(const Grid& G, int cx, int cy, int cz) {
  return ((long long)cz * G.dims[1] + cy) * G.dims[0] + cx;
}

// q-th cell (x fastest) of an nx x ny x nz range; q < 2^31 (the cell paths
// only run for ranges below the flat-scan threshold), so 32-bit division
// suffices -- 64-bit division is emulated and far slower.
__device__ __forceinline__ void decode_cell(long long q, int nx, int ny, int& dx, int& dy, int& dz) {
  const unsigned uq = (unsigned)q;
  const unsigned r = uq / (unsigned)nx;
  dx = (int)(uq - r * (unsigned)nx);
  const unsigned z = r / (unsigned)ny;
  dy = (int)(r - z * (unsigned)ny);
  dz = (int)z;
}

// clear the other parity's grids for the next rebuild (nobody reads them
// during this pass)
__device__ __forceinline__ void clear_other_parity(const IterArgs& A, int par) {
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long c = g; c < A.total_cells; c += stride) A.gcnt[par ^ 1][c] = 0;
  for (long long c = g; c < A.B; c += stride) A.ovf_cnt[par ^ 1][c] = 0;
}

// The candidate search of search unit t (one warp), list to tlist / tcnt.
// MULTI = false: a single cloud, whose table entry is read from the kernel
// parameters (constant bank) instead of global memory.
template <bool MULTI>
__device__ __forceinline__ void search_unit(const IterArgs& A, int par, int d, int t) {
  const int lane = threadIdx.x & 31;
  const int b = MULTI ? A.ucloud[t] : 0;
  if (MULTI && A.crun[b].done) return;
  float4* __restrict__ out = A.tlist + (int64_t)t * kTileCap;
  const Cloud& cl = MULTI ? A.clouds[b] : A.cl0;
  const Grid G = cl.grid;
  const int c0 = cl.c0, c1 = cl.c0 + cl.k;
  const float4 lo = A.ubox[2 * t], hi = A.ubox[2 * t + 1];
  if (A.stay) {   // the bound layer: a tile inside half the gap of its last label stays
    const int a = A.tlab[t];
    if (a >= 0) {
      const float4 c = A.cw[a];
      if (maxd2(lo, hi, c.x, c.y, c.z, d) <= kStay * A.cb2[a]) {
        if (lane == 0) {
          out[0] = c;
          A.tcnt[t] = 1;
          if (A.want_stats) {
            Slot& s = A.slots[t & (kSlots - 1)];
            red_add_u64(&s.cands, 1ull);
            red_add_u64(&s.stays, 1ull);
          }
        }
        return;
      }
    }
  }
  const int* __restrict__ gcnt = A.gcnt[par] + cl.cell0;
  const float4* __restrict__ gbkt = A.gbkt[par] + cl.cell0 * kBucketCap;
  const int n_ovf = A.ovf_cnt[par][b];
  const float4* __restrict__ ovf = A.ovf[par] + c0;
  // a range of more than k / 4 cells costs more than reading every centroid
  // of the cloud once, so large ranges scan the flat centroid array instead
  const long long flat_cells = (long long)(cl.k / 4) + 32;

  int clo[3], chi[3];
  clo[0] = cell_coord(lo.x, G.g0[0], G.inv_s, G.dims[0]);
  chi[0] = cell_coord(hi.x, G.g0[0], G.inv_s, G.dims[0]);
  clo[1] = cell_coord(lo.y, G.g0[1], G.inv_s, G.dims[1]);
  chi[1] = cell_coord(hi.y, G.g0[1], G.inv_s, G.dims[1]);
  clo[2] = d == 3 ? cell_coord(lo.z, G.g0[2], G.inv_s, G.dims[2]) : 0;
  chi[2] = d == 3 ? cell_coord(hi.z, G.g0[2], G.inv_s, G.dims[2]) : 0;

  // ---- phase A ----
  // Any centroid of the cloud bounds the nearest distance of every point in
  // the box by maxd(box, c).  The tile's list of the previous pass holds
  // ids near the tile, so its current positions give U in one load round;
  // ids outside the cloud (a list left by another tiling) are skipped.
  // Without a usable list, rings of cells around the box are scanned.
  // The centroid that gives U (r1) also serves as the dominance reference
  // of phase B.
  float u2 = INFINITY;
  float m = INFINITY;
  float4 r1 = make_float4(0.f, 0.f, 0.f, 0.f);   // this lane's best so far
  const int q_old = A.tcnt[t];
  if (q_old >= 1 && q_old <= kTileCap) {
    for (int j = lane; j < q_old; j += 32) {
      const int id = __float_as_int(out[j].w);
      if (id < c0 || id >= c1) continue;
      const float4 c = A.cw[id];
      const float mc = maxd2(lo, hi, c.x, c.y, c.z, d);
      if (mc < m) { m = mc; r1 = c; }
    }
    u2 = warp_min_nonneg(m);   // every lane has read its old ids before any is overwritten
  }
  for (int ring = 0; !(u2 < INFINITY); ring = ring ? 2 * ring : 1) {
    int rlo[3], rhi[3];
    long long ncell = 1;
    bool whole = true;
    for (int a = 0; a < 3; ++a) {
      rlo[a] = max(clo[a] - ring, 0);
      rhi[a] = min(chi[a] + ring, G.dims[a] - 1);
      whole = whole && rlo[a] == 0 && rhi[a] == G.dims[a] - 1;
      ncell *= (long long)(rhi[a] - rlo[a] + 1);
    }
    if (ncell > flat_cells) {
      for (int j = c0 + lane; j < c1; j += 32) {
        const float4 c = A.cw[j];
        const float mc = maxd2(lo, hi, c.x, c.y, c.z, d);
        if (mc < m) { m = mc; r1 = c; }
      }
      u2 = warp_min_nonneg(m);
      break;
    }
    const int nx = rhi[0] - rlo[0] + 1, ny = rhi[1] - rlo[1] + 1;
    for (long long q = lane; q < ncell; q += 32) {
      int ox, oy, oz;
      decode_cell(q, nx, ny, ox, oy, oz);
      long long cell = cell_index(G, rlo[0] + ox, rlo[1] + oy, rlo[2] + oz);
      int cnt = min(gcnt[cell], kBucketCap);
      for (int i = 0; i < cnt; ++i) {
        const float4 e = gbkt[cell * kBucketCap + i];
        const float mc = maxd2(lo, hi, e.x, e.y, e.z, d);
        if (mc < m) { m = mc; r1 = e; }
      }
    }
    for (int q = lane; q < n_ovf; q += 32) {
      const float4 c = ovf[q];
      const float mc = maxd2(lo, hi, c.x, c.y, c.z, d);
      if (mc < m) { m = mc; r1 = c; }
    }
    u2 = warp_min_nonneg(m);
    if (u2 < INFINITY || whole) break;
  }
  if (!(u2 < INFINITY)) {   // no centroid anywhere: cannot happen for k >= 1
    if (lane == 0) {
      A.tcnt[t] = 0;
      atomicOr(&A.st->err, kErrNoCentroid);
    }
    return;
  }

  // r1 = a centroid with maxd^2 = u2 (the lowest such lane's)
  {
    const int src = __ffs(__ballot_sync(0xffffffffu, m == u2)) - 1;
    r1.x = __shfl_sync(0xffffffffu, r1.x, src);
    r1.y = __shfl_sync(0xffffffffu, r1.y, src);
    r1.z = __shfl_sync(0xffffffffu, r1.z, src);
  }

  // ---- phase B ----
  // keep: within the ball bound (mind^2 <= U^2 kKeep) and not dominated
  // over the box by r1
  const float u2k = u2 * kKeep;
  const float slack = dom_slack(lo, hi, u2, u2k, d);
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
  if (ncell > flat_cells) {
    // every centroid of the cloud once; the overflow list is then redundant
    for (int j0 = c0; j0 < c1; j0 += 32) {
      const int j = j0 + lane;
      float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
      bool keep = false;
      if (j < c1) {
        c = A.cw[j];
        keep = mind2(lo, hi, c.x, c.y, c.z, d) <= u2k &&
               !dominated(lo, hi, r1, slack, c.x, c.y, c.z, d);
      }
      unsigned bal = __ballot_sync(0xffffffffu, keep);
      int pos = count + __popc(bal & lt);
      if (keep && pos < kTileCap) out[pos] = c;
      count += __popc(bal);
    }
  } else {
    for (long long q0 = 0; q0 < ncell; q0 += 32) {
      long long q = q0 + lane;
      long long cell = 0;
      int cnt = 0;
      if (q < ncell) {
        int ox, oy, oz;
        decode_cell(q, nx, ny, ox, oy, oz);
        cell = cell_index(G, rlo[0] + ox, rlo[1] + oy, rlo[2] + oz);
        cnt = min(gcnt[cell], kBucketCap);
      }
      const int cmax = __reduce_max_sync(0xffffffffu, cnt);
      for (int i = 0; i < cmax; ++i) {
        float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < cnt) e = gbkt[cell * kBucketCap + i];
        const bool keep = i < cnt && mind2(lo, hi, e.x, e.y, e.z, d) <= u2k &&
                          !dominated(lo, hi, r1, slack, e.x, e.y, e.z, d);
        unsigned bal = __ballot_sync(0xffffffffu, keep);
        int pos = count + __popc(bal & lt);
        if (keep && pos < kTileCap) out[pos] = e;
        count += __popc(bal);
      }
    }
    for (int q0 = 0; q0 < n_ovf; q0 += 32) {
      int q = q0 + lane;
      float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
      bool keep = false;
      if (q < n_ovf) {
        c = ovf[q];
        keep = mind2(lo, hi, c.x, c.y, c.z, d) <= u2k &&
               !dominated(lo, hi, r1, slack, c.x, c.y, c.z, d);
      }
      unsigned bal = __ballot_sync(0xffffffffu, keep);
      int pos = count + __popc(bal & lt);
      if (keep && pos < kTileCap) out[pos] = c;
      count += __popc(bal);
    }
  }
  if (lane == 0) {
    A.tcnt[t] = count;
    if (A.want_stats) {
      Slot& s = A.slots[t & (kSlots - 1)];
      red_add_u64(&s.cands, (unsigned long long)count);
      if (count > kTileCap) red_add_u64(&s.fallback, 1ull);
    }
  }
}

template <bool MULTI>
__global__ void __launch_bounds__(32 * kSearchWarps, DKM_SEARCH_MIN_BLOCKS)
    k_search(const __grid_constant__ IterArgs A, int par, int d) {
  if (A.st->n_done == A.B) return;   // every cloud stopped (fixed during this kernel)
  clear_other_parity(A, par);
  const int t = blockIdx.x * kSearchWarps + (threadIdx.x >> 5);
  if (t >= A.n_units) return;   // t: the search unit (a tile or a group of tiles)
  search_unit<MULTI>(A, par, d, t);
}

// ---------------------------------------------------------------------------
// k_assign<D, BRUTE>: one warp per tile of 4 rows x 64 points, two points
// per lane evaluated as packed f32x2.  Warps are independent (no CTA-wide
// barrier): each stages its own candidate list in shared memory, so small
// CTAs free their SM slot as soon as their own tiles are done.
// ---------------------------------------------------------------------------
#ifndef DKM_ASSIGN_WARPS
#define DKM_ASSIGN_WARPS 1   // one-warp CTAs: 24 per SM, freed as soon as their tile is done
#endif
constexpr int kAssignWarps = DKM_ASSIGN_WARPS;
#ifndef DKM_ASSIGN_MIN_WARPS
#define DKM_ASSIGN_MIN_WARPS 32   // 64 registers: 32 one-warp CTAs per SM
#endif
template <int D>
struct Pts {
  float2 x[kRowsPerWarp], y[kRowsPerWarp], z[kRowsPerWarp];
};

// Keep (s, id) if it is lexicographically smaller than (best, bid): the
// nearest centroid, ties to the lowest index, whatever order the
// candidates arrive in.  s >= 0, so its bit pattern orders like its value
// and the pair compares as one 64-bit key.
__device__ __forceinline__ void take_min(float s, int id, float& best, int& bid) {
  const unsigned long long key = ((unsigned long long)__float_as_uint(s) << 32) | (unsigned)id;
  const unsigned long long cur =
      ((unsigned long long)__float_as_uint(best) << 32) | (unsigned)bid;
  if (key < cur) {
    best = s;
    bid = id;
  }
}

#ifndef DKM_EVAL_UNROLL
#define DKM_EVAL_UNROLL 1
#endif
constexpr int kEvalUnroll = DKM_EVAL_UNROLL;   // candidates per unrolled step
// all rows of the tile against candidates s_c[idx[j]] (idx == nullptr: s_c[j])
template <int D>
__device__ __forceinline__ void eval_list(const float4* __restrict__ s_c,
                                          const unsigned short* __restrict__ idx, int m,
                                          const Pts<D>& P, float2 (&best)[kRowsPerWarp],
                                          int2 (&bid)[kRowsPerWarp]) {
#pragma unroll kEvalUnroll
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
      take_min(s.x, id, best[r].x, bid[r].x);
      take_min(s.y, id, best[r].y, bid[r].y);
    }
  }
}

// one row (64 points, two per lane) against candidates s_c[idx[j]]
template <int D>
__device__ __forceinline__ void eval_row(const float4* __restrict__ s_c,
                                         const unsigned short* __restrict__ idx, int m, float2 px,
                                         float2 py, float2 pz, float2& best, int2& bid) {
#pragma unroll 4
  for (int j = 0; j < m; ++j) {
    const float4 c = s_c[idx[j]];
    const int id = __float_as_int(c.w);
    float2 dx = __fadd2_rn(px, make_float2(-c.x, -c.x));
    float2 dy = __fadd2_rn(py, make_float2(-c.y, -c.y));
    float2 s = __fmul2_rn(dx, dx);
    s = __ffma2_rn(dy, dy, s);
    if (D == 3) {
      float2 dz = __fadd2_rn(pz, make_float2(-c.z, -c.z));
      s = __ffma2_rn(dz, dz, s);
    }
    take_min(s.x, id, best.x, bid.x);
    take_min(s.y, id, best.y, bid.y);
  }
}

// AABB of one row's valid points (warp-wide, identical on every lane).
__device__ __forceinline__ void row_box(float2 px, float2 py, float2 pz, bool va, bool vb,
                                        float4& lo, float4& hi) {
  const float inf = INFINITY;
  float mnx = fminf(va ? px.x : inf, vb ? px.y : inf), mxx = fmaxf(va ? px.x : -inf, vb ? px.y : -inf);
  float mny = fminf(va ? py.x : inf, vb ? py.y : inf), mxy = fmaxf(va ? py.x : -inf, vb ? py.y : -inf);
  float mnz = fminf(va ? pz.x : inf, vb ? pz.y : inf), mxz = fmaxf(va ? pz.x : -inf, vb ? pz.y : -inf);
  lo.x = float_of(__reduce_min_sync(0xffffffffu, ord_of(mnx)));
  lo.y = float_of(__reduce_min_sync(0xffffffffu, ord_of(mny)));
  lo.z = float_of(__reduce_min_sync(0xffffffffu, ord_of(mnz)));
  hi.x = float_of(__reduce_max_sync(0xffffffffu, ord_of(mxx)));
  hi.y = float_of(__reduce_max_sync(0xffffffffu, ord_of(mxy)));
  hi.z = float_of(__reduce_max_sync(0xffffffffu, ord_of(mxz)));
  lo.w = hi.w = 0.f;
}

// Indices of the list entries s_c[0..m) that can hold the nearest centroid
// of some point inside [lo, hi] (same bound as k_search with this box).
// u2_in caps the bound (INFINITY = none); returns the count.
template <int D>
__device__ __forceinline__ int filter_box(const float4* __restrict__ s_c, int m, float4 lo,
                                          float4 hi, float u2_in,
                                          unsigned short* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  float u = u2_in;
  for (int j = lane; j < m; j += 32) {
    const float4 c = s_c[j];
    u = fminf(u, maxd2(lo, hi, c.x, c.y, c.z, D));
  }
  const float u2k = warp_min_nonneg(u) * kKeep;
  const unsigned lt = (1u << lane) - 1u;
  int cnt = 0;
  for (int j0 = 0; j0 < m; j0 += 32) {
    const int j = j0 + lane;
    bool keep = false;
    if (j < m) {
      const float4 c = s_c[j];
      keep = mind2(lo, hi, c.x, c.y, c.z, D) <= u2k;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (keep) out[cnt + __popc(bal & lt)] = (unsigned short)j;
    cnt += __popc(bal);
  }
  __syncwarp();
  return cnt;
}

__device__ __forceinline__ void add_group(const IterArgs& A, int D, int L, int sx, int sy, int sz,
                                          int cnt, int s_q, int s_glob) {
  Acc* a = &A.acc[L];
  red_add_u64(&a->s[0], (unsigned long long)rescale(sx, s_q, s_glob));
  red_add_u64(&a->s[1], (unsigned long long)rescale(sy, s_q, s_glob));
  if (D == 3) red_add_u64(&a->s[2], (unsigned long long)rescale(sz, s_q, s_glob));
  red_add_u64(&a->cnt, (unsigned long long)cnt);
}

// unit exponent s with n_max * max|r| * 2^s < 2^31 for groups of up to
// 2^(31 - 1 - bits) points: 2^bits * max|r| * 2^s < 2^30
__device__ __forceinline__ int group_scale(float m, int bits) {
  return m > 0.f ? min(bits - exp_bound(m), 127) : 0;
}

// The entries of src[0..m) (global memory) that can hold the nearest
// centroid of some point inside [lo, hi], written compactly to out (shared
// memory, m <= kTileCap); returns the count.  U = min over the list of
// maxd(box, c) bounds every point's nearest distance (any centroid of the
// cloud does), and a point's nearest centroid c* has mind(box, c*) <= U.
template <int D>
__device__ __forceinline__ int filter_list(const float4* __restrict__ src, int m, float4 lo,
                                           float4 hi, float4* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  float u = INFINITY;
  for (int j = lane; j < m; j += 32) {
    const float4 c = src[j];
    u = fminf(u, maxd2(lo, hi, c.x, c.y, c.z, D));
  }
  const float u2k = warp_min_nonneg(u) * kKeep;
  const unsigned lt = (1u << lane) - 1u;
  int cnt = 0;
  for (int j0 = 0; j0 < m; j0 += 32) {
    const int j = j0 + lane;
    float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
    bool keep = false;
    if (j < m) {
      c = src[j];
      keep = mind2(lo, hi, c.x, c.y, c.z, D) <= u2k;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (keep) out[cnt + __popc(bal & lt)] = c;
    cnt += __popc(bal);
  }
  __syncwarp();
  return cnt;
}

// Tile epilogue shared by k_assign and k_accum_labels: residuals p - c of
// the tile's points (4 rows x 2 per lane) against their own centroid, in
// 32-bit fixed point with one tile-wide power-of-two scale (256 points *
// max|r| * 2^s < 2^31, so int32 sums cannot overflow), summed per label
// and added to the per-centroid accumulators with 64-bit integer atomics.
// A tile whose points all share one label loads its centroid once and adds
// one group; otherwise every point loads its own centroid and the labels
// are taken one at a time (the smallest pending label of the warp).  The
// sums depend only on the tile and the labels, so every caller gets the
// same sums bit for bit.  Returns the tile's label when all its points
// share one, else -1.
template <int D>
__device__ __forceinline__ int accumulate_tile(const IterArgs& A, const float2 (&px)[kRowsPerWarp],
                                                const float2 (&py)[kRowsPerWarp],
                                                const float2 (&pz)[kRowsPerWarp],
                                                const int2 (&lab)[kRowsPerWarp],
                                                const bool (&va)[kRowsPerWarp],
                                                const bool (&vb)[kRowsPerWarp], int s_glob) {
  constexpr int H = 2 * kRowsPerWarp;
  const int lane = threadIdx.x & 31;
  int lb[H];
  bool pend[H];
  int lmin = INT_MAX;
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r) {
    lb[2 * r] = lab[r].x;
    lb[2 * r + 1] = lab[r].y;
    pend[2 * r] = va[r];
    pend[2 * r + 1] = vb[r];
  }
#pragma unroll
  for (int h = 0; h < H; ++h) lmin = pend[h] ? min(lmin, lb[h]) : lmin;
  int L = __reduce_min_sync(0xffffffffu, lmin);
  if (L == INT_MAX) return -1;   // no valid point
  bool same = true;
#pragma unroll
  for (int h = 0; h < H; ++h) same = same && (!pend[h] || lb[h] == L);
  const bool single = __all_sync(0xffffffffu, same);
  float rx[H], ry[H], rz[H];
  float4 c0 = make_float4(0.f, 0.f, 0.f, 0.f);
  if (single) c0 = __ldg(&A.cw[L]);
  float ml = 0.f;
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r) {
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const int h = 2 * r + hh;
      rx[h] = ry[h] = rz[h] = 0.f;
      if (pend[h]) {
        const float4 c = single ? c0 : __ldg(&A.cw[lb[h]]);
        rx[h] = __fadd_rn(hh ? px[r].y : px[r].x, -c.x);
        ry[h] = __fadd_rn(hh ? py[r].y : py[r].x, -c.y);
        if (D == 3) rz[h] = __fadd_rn(hh ? pz[r].y : pz[r].x, -c.z);
      }
      ml = fmaxf(ml, fmaxf(fmaxf(fabsf(rx[h]), fabsf(ry[h])), fabsf(rz[h])));
    }
  }
  const int s_t = group_scale(warp_max_nonneg(ml), 22);
  const float sc = pow2f(s_t);
  int qx[H], qy[H], qz[H];
#pragma unroll
  for (int h = 0; h < H; ++h) {
    qx[h] = __float2int_rn(rx[h] * sc);
    qy[h] = __float2int_rn(ry[h] * sc);
    qz[h] = D == 3 ? __float2int_rn(rz[h] * sc) : 0;
  }
  while (true) {
    int sx = 0, sy = 0, sz = 0, cnt = 0;
    lmin = INT_MAX;
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const bool g = pend[h] && lb[h] == L;
      sx += g ? qx[h] : 0;
      sy += g ? qy[h] : 0;
      sz += g ? qz[h] : 0;
      cnt += g ? 1 : 0;
      pend[h] = pend[h] && !g;
      lmin = pend[h] ? min(lmin, lb[h]) : lmin;
    }
    sx = __reduce_add_sync(0xffffffffu, sx);
    sy = __reduce_add_sync(0xffffffffu, sy);
    if (D == 3) sz = __reduce_add_sync(0xffffffffu, sz);
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if (lane == 0) add_group(A, D, L, sx, sy, sz, cnt, s_t, s_glob);
    if (single) return L;
    L = __reduce_min_sync(0xffffffffu, lmin);
    if (L == INT_MAX) return -1;
  }
}

// Tile SSE in fixed point (unit 2^-s_sse) with one tile-wide scale
// (256 * max d^2 * 2^s < 2^31), identical on every lane.
__device__ __forceinline__ long long tile_sse(const float2 (&best)[kRowsPerWarp],
                                             const bool (&va)[kRowsPerWarp],
                                             const bool (&vb)[kRowsPerWarp], int s_sse) {
  float ml = 0.f;
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r)
    ml = fmaxf(ml, fmaxf(va[r] ? best[r].x : 0.f, vb[r] ? best[r].y : 0.f));
  const float m = warp_max_nonneg(ml);
  const int s2 = m > 0.f ? min(22 - exp_bound(m), 127) : 0;
  const float sc = pow2f(s2);
  unsigned q = 0;
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r) {
    q += va[r] ? (unsigned)__float2uint_rn(best[r].x * sc) : 0u;
    q += vb[r] ? (unsigned)__float2uint_rn(best[r].y * sc) : 0u;
  }
  return rescale((long long)__reduce_add_sync(0xffffffffu, q), s2, s_sse);
}

// The 4 rows of a 256-window starting at `base` (always inside the padded
// arrays); a point is valid if its sorted index lies in [vlo, vhi).
__device__ __forceinline__ void load_points(const IterArgs& A, int D, int64_t base, int64_t vlo,
                                            int64_t vhi, float2 (&x)[kRowsPerWarp],
                                            float2 (&y)[kRowsPerWarp], float2 (&z)[kRowsPerWarp],
                                            bool (&va)[kRowsPerWarp], bool (&vb)[kRowsPerWarp]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r) {
    int64_t i = base + r * kRowPts + 2 * lane;
    x[r] = *reinterpret_cast<const float2*>(A.xs + i);
    y[r] = *reinterpret_cast<const float2*>(A.ys + i);
    z[r] = D == 3 ? *reinterpret_cast<const float2*>(A.zs + i) : make_float2(0.f, 0.f);
    va[r] = i >= vlo && i < vhi;
    vb[r] = i + 1 >= vlo && i + 1 < vhi;
  }
}

// Assignment of tile t (one warp) from its search unit's candidate list:
// labels, SSE and the update sums.  sc / sr / slbw: the warp's shared
// staging (kTileCap candidates, kTileCap indices, 32 bounds).
template <int D, bool BRUTE, bool MULTI, bool UNITS>
__device__ __forceinline__ void assign_tile(const IterArgs& A, int t, float4* __restrict__ sc,
                                            unsigned short* __restrict__ sr,
                                            float* __restrict__ slbw) {
  const int lane = threadIdx.x & 31;
  const int b = MULTI ? A.tcloud[t] : 0;
  if (MULTI && A.crun[b].done) return;
  const Cloud& cl = MULTI ? A.clouds[b] : A.cl0;
  const int c0 = cl.c0, c1 = cl.c0 + cl.k;
  if (t == (MULTI ? A.tfirst[b] : 0) && lane == 0) A.crun[b].passes += 1;   // one writer per cloud
  const int2 se = A.tiles[t];
  const int64_t base = (int64_t)(se.x / kTilePts) * kTilePts;

  Pts<D> P;
  bool va[kRowsPerWarp], vb[kRowsPerWarp];
  load_points(A, D, base, se.x, se.y, P.x, P.y, P.z, va, vb);
  int nv_row[kRowsPerWarp];
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r)
    nv_row[r] = __popc(__ballot_sync(0xffffffffu, va[r])) + __popc(__ballot_sync(0xffffffffu, vb[r]));
  const int nv_tile = se.y - se.x;

  float2 best[kRowsPerWarp];
  int2 bid[kRowsPerWarp];
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r) {
    best[r] = make_float2(INFINITY, INFINITY);
    bid[r] = make_int2(0, 0);
  }
  unsigned long long evals = 0;   // point x candidate evaluations of this warp
  if (BRUTE) {
    for (int j0 = c0; j0 < c1; j0 += kTileCap) {
      const int m = min(kTileCap, c1 - j0);
      __syncwarp();
      for (int i = lane; i < m; i += 32) sc[i] = A.cw[j0 + i];
      __syncwarp();
      eval_list<D>(sc, nullptr, m, P, best, bid);
    }
    evals = (unsigned long long)cl.k * nv_tile;
  } else {
    const int u = UNITS ? A.tunit[t] : t;   // the tile's search unit
    const int qs = A.tcnt[u];
    if (qs == 0 && lane == 0) atomicOr(&A.st->err, kErrEmptyList);
    if (qs <= kTileCap) {
      const float4* __restrict__ src = A.tlist + (int64_t)u * kTileCap;
      int q = qs;
      if (UNITS) {
        // the unit's list holds every candidate of the group's box; narrow
        // it with this tile's own box (the bound of k_search)
        q = filter_list<D>(src, qs, A.tbox[2 * t], A.tbox[2 * t + 1], sc);
      } else {
        for (int i = lane; i < qs; i += 32) sc[i] = src[i];
        __syncwarp();
      }
      if (q <= A.sort_max) {   // sort_max <= 32
        // Short list: order it by the lower bound mind^2(tile box, c) and
        // stop once the next bound exceeds every point's current best (the
        // kNN pruning rule of Algorithm 1's kNN function, with the tile box
        // as the query node).  (d^2, id) keys make the result order
        // independent.
        const float4 tlo = A.tbox[2 * t], thi = A.tbox[2 * t + 1];
        const bool has = lane < q;
        const float4 c = has ? sc[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float lb = has ? mind2(tlo, thi, c.x, c.y, c.z, D) : INFINITY;
        const unsigned long long key =
            ((unsigned long long)__float_as_uint(lb) << 32) | (unsigned)lane;
        int rank = 0;
        for (int m = 0; m < q; ++m) rank += __shfl_sync(0xffffffffu, key, m) < key;
        if (has) {
          sr[rank] = (unsigned short)lane;
          slbw[rank] = lb;
        }
        __syncwarp();
        int done = 0;
        for (int j0 = 0; j0 < q; j0 += 4) {
          if (j0 > 0) {
            float mb = 0.f;
#pragma unroll
            for (int r = 0; r < kRowsPerWarp; ++r)
              mb = fmaxf(mb, fmaxf(va[r] ? best[r].x : 0.f, vb[r] ? best[r].y : 0.f));
            if (slbw[j0] > warp_max_nonneg(mb) * kKeep) break;
          }
          const int m = min(4, q - j0);
          eval_list<D>(sc, sr + j0, m, P, best, bid);
          done = j0 + m;
        }
        evals = (unsigned long long)done * nv_tile;
      } else if (q > A.row_filter_min) {
        // long list: narrow it again per row of 64 points
#pragma unroll
        for (int r = 0; r < kRowsPerWarp; ++r) {
          if (nv_row[r] == 0) continue;
          float4 rlo, rhi;
          row_box(P.x[r], P.y[r], P.z[r], va[r], vb[r], rlo, rhi);
          const int mr = filter_box<D>(sc, q, rlo, rhi, INFINITY, sr);
          eval_row<D>(sc, sr, mr, P.x[r], P.y[r], P.z[r], best[r], bid[r]);
          evals += (unsigned long long)mr * nv_row[r];
        }
      } else {
        eval_list<D>(sc, nullptr, q, P, best, bid);
        evals = (unsigned long long)q * nv_tile;
      }
    } else {
      // The list overflowed: take the tile bound over every centroid first,
      // then stream every centroid once, keep the ones that pass the bound
      // in shared memory and evaluate them whenever the buffer fills.
      const float4 tlo = A.tbox[2 * t], thi = A.tbox[2 * t + 1];
      float u = INFINITY;
#pragma unroll 8
      for (int j = c0 + lane; j < c1; j += 32) {
        const float4 c = __ldg(&A.cw[j]);
        u = fminf(u, maxd2(tlo, thi, c.x, c.y, c.z, D));
      }
      const float u2k = warp_min_nonneg(u) * kKeep;
      const unsigned lt = (1u << lane) - 1u;
      int cnt = 0;
      for (int j0 = c0; j0 < c1; j0 += 4 * 32) {
        float4 c[4];
#pragma unroll
        for (int b4 = 0; b4 < 4; ++b4) {
          const int j = j0 + b4 * 32 + lane;
          c[b4] = j < c1 ? __ldg(&A.cw[j]) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int b4 = 0; b4 < 4; ++b4) {
          const int j = j0 + b4 * 32 + lane;
          const bool keep = j < c1 && mind2(tlo, thi, c[b4].x, c[b4].y, c[b4].z, D) <= u2k;
          const unsigned bal = __ballot_sync(0xffffffffu, keep);
          if (keep) sc[cnt + __popc(bal & lt)] = c[b4];
          cnt += __popc(bal);
        }
        if (cnt > kTileCap - 4 * 32 || j0 + 4 * 32 >= c1) {
          __syncwarp();
          eval_list<D>(sc, nullptr, cnt, P, best, bid);
          evals += (unsigned long long)cnt * nv_tile;
          cnt = 0;
          __syncwarp();
        }
      }
    }
  }

  const int s_glob = A.crun[b].s_glob, s_sse = A.crun[b].s_sse;
  long long sse = 0;
  int changed = 0;
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r) {
    if (nv_row[r] == 0) continue;   // warp-uniform
    const int64_t i = base + r * kRowPts + 2 * lane;
    const int la = bid[r].x, lb = bid[r].y;
    if (A.track_changes) {
      int pa = va[r] ? A.lab[i] : la, pb = vb[r] ? A.lab[i + 1] : lb;
      changed += (int)(pa != la) + (int)(pb != lb);
    }
    if (va[r] && vb[r]) {
      *reinterpret_cast<int2*>(A.lab + i) = make_int2(la, lb);
    } else if (va[r]) {
      A.lab[i] = la;
    } else if (vb[r]) {
      A.lab[i + 1] = lb;
    }
  }
  if (A.want_sse) sse = tile_sse(best, va, vb, s_sse);
  const int single = accumulate_tile<D>(A, P.x, P.y, P.z, bid, va, vb, s_glob);
  changed = __reduce_add_sync(0xffffffffu, changed);
  if (lane == 0) {
    if (A.stay) A.tlab[t] = single;
    CloudAcc& ca = A.cacc[b];
    red_add_u64(&ca.sse[t & (kCloudSlots - 1)], (unsigned long long)sse);
    if (changed) red_add_u64(&ca.changed[t & (kCloudSlots - 1)], (unsigned long long)changed);
    if (A.want_stats) red_add_u64(&A.slots[t & (kSlots - 1)].evals, evals);
  }
}


// UNITS: tiles share search units (tile_group > 1) and filter their unit's
// list with their own box.
template <int D, bool BRUTE, bool MULTI, bool UNITS>
__global__ void __launch_bounds__(32 * kAssignWarps, DKM_ASSIGN_MIN_WARPS / kAssignWarps)
    k_assign(const __grid_constant__ IterArgs A) {
  __shared__ float4 s_c[kAssignWarps][kTileCap];
  __shared__ unsigned short s_r[kAssignWarps][kTileCap];
  __shared__ float slb[kAssignWarps][32];
  if (A.st->n_done == A.B) return;   // every cloud stopped (fixed during this kernel)
  const int w = threadIdx.x >> 5;
  const int t = blockIdx.x * kAssignWarps + w;
  if (t >= A.n_tiles) return;   // warp-level exits, no CTA barrier below
  assign_tile<D, BRUTE, MULTI, UNITS>(A, t, s_c[w], s_r[w], slb[w]);
}

// ---------------------------------------------------------------------------
// k_accum_labels: residual sums for a caller-given labelling (dkm_update;
// cloud-local labels).  One warp per tile, grouped exactly like k_assign,
// so both produce the same sums bit for bit for the same labels.
// ---------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(kBlockThreads) k_accum_labels(IterArgs A,
                                                               const int32_t* __restrict__ ulab,
                                                               const uint32_t* __restrict__ perm) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int t = blockIdx.x * kWarpsPerBlock + w;
  if (t >= A.n_tiles) return;
  const int2 se = A.tiles[t];
  const int b = A.tcloud[t];
  const int c0 = A.clouds[b].c0, kb = A.clouds[b].k;
  const int64_t base = (int64_t)(se.x / kTilePts) * kTilePts;
  float2 x[kRowsPerWarp], y[kRowsPerWarp], z[kRowsPerWarp];
  bool va[kRowsPerWarp], vb[kRowsPerWarp];
  load_points(A, D, base, se.x, se.y, x, y, z, va, vb);
  int bad = 0;
  int2 lab[kRowsPerWarp];
  bool oka[kRowsPerWarp], okb[kRowsPerWarp];
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r) {
    const int64_t i = base + r * kRowPts + 2 * lane;
    const int la = va[r] ? ulab[perm[i]] : 0;
    const int lb = vb[r] ? ulab[perm[i + 1]] : 0;
    oka[r] = va[r] && la >= 0 && la < kb;
    okb[r] = vb[r] && lb >= 0 && lb < kb;
    bad |= (va[r] && !oka[r]) || (vb[r] && !okb[r]);
    lab[r] = make_int2(c0 + (oka[r] ? la : 0), c0 + (okb[r] ? lb : 0));
  }
  accumulate_tile<D>(A, x, y, z, lab, oka, okb, A.crun[b].s_glob);
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&A.st->label_err, 1);
}

// ---------------------------------------------------------------------------
// k_finalize: labels back to the caller's order as cloud-local indices;
// optional SSE against the current centroids (same FP32 distance
// expression, fixed-point tile sums per cloud).  One warp per tile.
// ---------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(kBlockThreads) k_finalize(IterArgs A,
                                                           const uint32_t* __restrict__ perm,
                                                           int32_t* __restrict__ labels_out,
                                                           int do_sse) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int t = blockIdx.x * kWarpsPerBlock + w;
  if (t >= A.n_tiles) return;
  const int2 se = A.tiles[t];
  const int b = A.tcloud[t];
  const int c0 = A.clouds[b].c0;
  const int64_t base = (int64_t)(se.x / kTilePts) * kTilePts;
  float2 x[kRowsPerWarp], y[kRowsPerWarp], z[kRowsPerWarp];
  bool va[kRowsPerWarp], vb[kRowsPerWarp];
  load_points(A, D, base, se.x, se.y, x, y, z, va, vb);
  float2 d2[kRowsPerWarp];
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r) {
    const int64_t i = base + r * kRowPts + 2 * lane;
    const int la = va[r] ? A.lab[i] : c0, lb = vb[r] ? A.lab[i + 1] : c0;
    if (labels_out) {
      if (va[r]) labels_out[perm[i]] = la - c0;
      if (vb[r]) labels_out[perm[i + 1]] = lb - c0;
    }
    d2[r] = make_float2(0.f, 0.f);
    if (do_sse) {
      const float4 ca = __ldg(&A.cw[la]), cb = __ldg(&A.cw[lb]);
      float dx = __fadd_rn(x[r].x, -ca.x), dy = __fadd_rn(y[r].x, -ca.y);
      float s = __fmaf_rn(dy, dy, __fmul_rn(dx, dx));
      if (D == 3) { float dz = __fadd_rn(z[r].x, -ca.z); s = __fmaf_rn(dz, dz, s); }
      d2[r].x = s;
      dx = __fadd_rn(x[r].y, -cb.x); dy = __fadd_rn(y[r].y, -cb.y);
      s = __fmaf_rn(dy, dy, __fmul_rn(dx, dx));
      if (D == 3) { float dz = __fadd_rn(z[r].y, -cb.z); s = __fmaf_rn(dz, dz, s); }
      d2[r].y = s;
    }
  }
  if (do_sse) {
    const long long sse = tile_sse(d2, va, vb, A.crun[b].s_sse);
    if (lane == 0) red_add_u64(&A.cacc[b].sse[t & (kCloudSlots - 1)], (unsigned long long)sse);
  }
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

cudaError_t launch_reset_run(const IterArgs& A, cudaStream_t s) {
  k_reset_run<<<ceil_div(A.B, 256), 256, 0, s>>>(A.st, A.crun, A.cacc, A.B);
  return cudaGetLastError();
}

cudaError_t launch_centroids(const IterArgs& A, int mode, int t, int d, const float* user_c,
                             int insert, int par, int32_t* counts_out, cudaStream_t s) {
  k_centroids<<<ceil_div(A.k, kBlockThreads), kBlockThreads, 0, s>>>(A, mode, t, d, user_c, insert,
                                                                    par, counts_out);
  return cudaGetLastError();
}

cudaError_t launch_search(const IterArgs& A, int par, int d, cudaStream_t s) {
  const int g = ceil_div(A.n_units, kSearchWarps);
  if (A.B > 1) k_search<true><<<g, 32 * kSearchWarps, 0, s>>>(A, par, d);
  else k_search<false><<<g, 32 * kSearchWarps, 0, s>>>(A, par, d);
  return cudaGetLastError();
}

template <int D, bool BRUTE>
void assign_multi(const IterArgs& A, int g, cudaStream_t s) {
  constexpr int thr = 32 * kAssignWarps;
  if (!BRUTE && A.unit_g > 1) {
    if (A.B > 1) k_assign<D, false, true, true><<<g, thr, 0, s>>>(A);
    else k_assign<D, false, false, true><<<g, thr, 0, s>>>(A);
    return;
  }
  if (A.B > 1) k_assign<D, BRUTE, true, false><<<g, thr, 0, s>>>(A);
  else k_assign<D, BRUTE, false, false><<<g, thr, 0, s>>>(A);
}

cudaError_t launch_assign(const IterArgs& A, int d, int brute, cudaStream_t s) {
  const int g = ceil_div(A.n_tiles, kAssignWarps);
  if (d == 3) {
    if (brute) assign_multi<3, true>(A, g, s);
    else assign_multi<3, false>(A, g, s);
  } else {
    if (brute) assign_multi<2, true>(A, g, s);
    else assign_multi<2, false>(A, g, s);
  }
  return cudaGetLastError();
}

cudaError_t launch_collect(const IterArgs& A, int t, cudaStream_t s) {
  k_collect<<<1, kBlockThreads, 0, s>>>(A, t);
  return cudaGetLastError();
}

cudaError_t launch_accum_labels(const IterArgs& A, int d, const int32_t* ulab,
                                const uint32_t* perm, cudaStream_t s) {
  const int g = ceil_div(A.n_tiles, kWarpsPerBlock);
  if (d == 3) k_accum_labels<3><<<g, kBlockThreads, 0, s>>>(A, ulab, perm);
  else k_accum_labels<2><<<g, kBlockThreads, 0, s>>>(A, ulab, perm);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const IterArgs& A, int d, const uint32_t* perm, int32_t* labels_out,
                            int do_sse, cudaStream_t s) {
  const int g = ceil_div(A.n_tiles, kWarpsPerBlock);
  if (d == 3) k_finalize<3><<<g, kBlockThreads, 0, s>>>(A, perm, labels_out, do_sse);
  else k_finalize<2><<<g, kBlockThreads, 0, s>>>(A, perm, labels_out, do_sse);
  return cudaGetLastError();
}

cudaError_t launch_export(const float4* cw, int k, int d, float* out, cudaStream_t s) {
  k_export<<<ceil_div(k, 256), 256, 0, s>>>(cw, k, d, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// k_cbound: cb2[j] = squared distance from centroid j to the nearest other
// centroid of its cloud (the paper's per-iteration kNN(2) over the
// centroids), from the grid of parity `par` just built.  Rings of cells
// around c_j's cell are scanned until the best distance found is within
// the ring's lower bound: a centroid whose cell lies beyond ring r is at
// least r cell edges away.  Both the bound and the final value err low
// (slack 2^-8), so cb2 never exceeds the true squared gap by more than
// rounding and the stay test stays conservative.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlockThreads) k_cbound(IterArgs A, int par, int d) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= A.k) return;
  const int b = A.kcloud[j];
  if (A.crun[b].done) return;
  const Cloud& cl = A.clouds[b];
  const float4 c = A.cw[j];
  float best = INFINITY;
  auto take = [&](const float4& e) {
    if (__float_as_int(e.w) == j) return;
    const float dx = __fadd_rn(e.x, -c.x), dy = __fadd_rn(e.y, -c.y), dz = __fadd_rn(e.z, -c.z);
    best = fminf(best, __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx))));
  };
  const int n_ovf = A.ovf_cnt[par][b];
  for (int q = 0; q < n_ovf; ++q) take(A.ovf[par][cl.c0 + q]);
  const Grid& G = cl.grid;
  const int* __restrict__ gcnt = A.gcnt[par] + cl.cell0;
  const float4* __restrict__ gbkt = A.gbkt[par] + cl.cell0 * kBucketCap;
  const int cc[3] = {cell_coord(c.x, G.g0[0], G.inv_s, G.dims[0]),
                     cell_coord(c.y, G.g0[1], G.inv_s, G.dims[1]),
                     d == 3 ? cell_coord(c.z, G.g0[2], G.inv_s, G.dims[2]) : 0};
  const float edge = 1.0f / G.inv_s;
  // cell coordinates carry FP32 rounding of up to ~dims * 2^-24 cells
  const int dmax = max(max(G.dims[0], G.dims[1]), G.dims[2]);
  const float margin = 1.0f / 64.0f + (float)dmax * (1.0f / 1048576.0f);
  const long long flat_cells = (long long)(cl.k / 4) + 32;
  for (int r = 0;; ++r) {
    int lo[3], hi[3];
    long long ncell = 1;
    bool whole = true;
    for (int a = 0; a < 3; ++a) {
      lo[a] = max(cc[a] - r, 0);
      hi[a] = min(cc[a] + r, G.dims[a] - 1);
      whole = whole && lo[a] == 0 && hi[a] == G.dims[a] - 1;
      ncell *= (long long)(hi[a] - lo[a] + 1);
    }
    if (ncell > flat_cells) {   // large rings: every centroid of the cloud once
      best = INFINITY;
      for (int q = cl.c0; q < cl.c0 + cl.k; ++q) take(A.cw[q]);
      break;
    }
    // the shell of ring r (cells at Chebyshev distance exactly r)
    for (int z = lo[2]; z <= hi[2]; ++z)
      for (int y = lo[1]; y <= hi[1]; ++y)
        for (int x = lo[0]; x <= hi[0]; ++x) {
          const int cheb = max(max(abs(x - cc[0]), abs(y - cc[1])), abs(z - cc[2]));
          if (cheb != r) continue;
          const long long cell = ((long long)z * G.dims[1] + y) * G.dims[0] + x;
          const int cnt = min(gcnt[cell], kBucketCap);
          for (int i = 0; i < cnt; ++i) take(gbkt[cell * kBucketCap + i]);
        }
    if (whole) break;
    const float lb = fmaxf((float)r - margin, 0.f) * edge;
    if (best <= lb * lb * (1.0f - 1.0f / 256.0f)) break;
  }
  A.cb2[j] = best * (1.0f - 1.0f / 256.0f);
}

cudaError_t launch_cbound(const IterArgs& A, int par, int d, cudaStream_t s) {
  k_cbound<<<ceil_div(A.k, kBlockThreads), kBlockThreads, 0, s>>>(A, par, d);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Search units of tile_group > 1: unit u covers tiles [ufirst[u],
// ufirst[u+1]) of one cloud (at most 32); its box is the union of theirs.
// One warp per unit.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlockThreads) k_unit_boxes(const float4* __restrict__ tbox,
                                                              const int* __restrict__ tcloud,
                                                              const int* __restrict__ ufirst,
                                                              int n_units, float4* __restrict__ ubox,
                                                              int* __restrict__ ucloud,
                                                              int* __restrict__ tunit) {
  const int lane = threadIdx.x & 31;
  const int u = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (u >= n_units) return;
  const int f = ufirst[u], cnt = ufirst[u + 1] - f;
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  if (lane < cnt) {
    const float4 a = tbox[2 * (f + lane)], z = tbox[2 * (f + lane) + 1];
    lo[0] = a.x; lo[1] = a.y; lo[2] = a.z;
    hi[0] = z.x; hi[1] = z.y; hi[2] = z.z;
    tunit[f + lane] = u;
  }
  for (int k = 0; k < 3; ++k) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
      hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
    }
  }
  if (lane == 0) {
    ubox[2 * u] = make_float4(lo[0], lo[1], lo[2], 0.f);
    ubox[2 * u + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
    ucloud[u] = tcloud[f];
  }
}

cudaError_t launch_unit_boxes(const float4* tbox, const int* tcloud, const int* ufirst,
                              int n_units, float4* ubox, int* ucloud, int* tunit,
                              cudaStream_t s) {
  k_unit_boxes<<<ceil_div(n_units, kWarpsPerBlock), kBlockThreads, 0, s>>>(tbox, tcloud, ufirst,
                                                                          n_units, ubox, ucloud,
                                                                          tunit);
  return cudaGetLastError();
}

}  // namespace dkm
