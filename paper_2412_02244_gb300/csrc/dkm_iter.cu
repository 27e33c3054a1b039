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
  __shared__ unsigned long long s_part[7][kBlockThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double sse = 0.0;
  // changed, evals, cands, fallback, clouds run, stayed tiles, stayed points
  unsigned long long v[7] = {0, 0, 0, 0, 0, 0, 0};
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
      v[1] += s.evals; v[2] += s.cands; v[3] += s.fallback; v[5] += s.stays; v[6] += s.pstays;
      s.evals = 0; s.cands = 0; s.fallback = 0; s.stays = 0; s.pstays = 0;
    }
  }
  for (int o = 16; o > 0; o >>= 1) sse += __shfl_xor_sync(0xffffffffu, sse, o);
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    if (lane == 0) s_part[q][w] = v[q];
  }
  if (lane == 0) s_sse[w] = sse;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tot[7] = {0, 0, 0, 0, 0, 0, 0};
    double tsse = 0.0;
    for (int ww = 0; ww < (int)(blockDim.x / 32); ++ww) {
      tsse += s_sse[ww];
      for (int q = 0; q < 7; ++q) tot[q] += s_part[q][ww];
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
      A.st->last_pstays = tot[6];
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
  crun[b].dmax[0] = 0u;
  crun[b].dmax[1] = 0u;
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
// cloud executed pass t, and an extra CTA folds the pass's counters.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlockThreads) k_centroids(IterArgs A, int mode, int t, int d,
                                                             const float* __restrict__ user_c,
                                                             int insert, int par,
                                                             int32_t* __restrict__ counts_out) {
  // (no kernel-wide early exit: n_done changes inside this kernel, so only
  // the per-cloud pass counts, fixed since k_assign, decide what runs)
  // The last CTA, beyond the centroids' CTAs, folds the pass's counters, so
  // that the fold and the updates run side by side (nothing here reads what
  // the fold writes).
  const bool fold = mode == 1 && t >= 0 && (A.want_stats || A.early_stop);
  if (fold && blockIdx.x == gridDim.x - 1) {
    collect_pass(A, t);
    return;
  }
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= A.k) return;
  const int b = A.B > 1 ? A.kcloud[j] : 0;
  // a cloud that stopped earlier (only early-stopping runs stop clouds)
  if (mode == 1 && t >= 0 && A.early_stop && A.crun[b].passes != t + 1) return;
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
    const float4 c_old = c;
    if (cnt > 0) {
      const int s_glob = A.crun[b].s_glob;
      c.x = refine_coord(c.x, (long long)a.s[0], cnt, s_glob);
      c.y = refine_coord(c.y, (long long)a.s[1], cnt, s_glob);
      if (d == 3) c.z = refine_coord(c.z, (long long)a.s[2], cnt, s_glob);
    }
    if (A.stay && t >= 0) {
      // the drift Delta[j] of Algorithm 1's refine step (rounded up) and
      // the cloud's max drift, for the next inter-bound search: the
      // maximum is taken over the warp's lanes of the same cloud first, so
      // that one atomic per warp and cloud reaches the shared word
      const float dx = c.x - c_old.x, dy = c.y - c_old.y, dz = c.z - c_old.z;
      const float dl = sqrtf(dx * dx + dy * dy + dz * dz) * 1.0001f;
      A.drift[j] = dl;
      CloudRun& r = A.crun[b];
      const unsigned peers = __match_any_sync(__activemask(), b);
      const unsigned wmax = __reduce_max_sync(peers, __float_as_uint(dl));
      if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicMax(&r.dmax[t & 1], wmax);
      if (j == A.clouds[b].c0) r.dmax[(t + 1) & 1] = 0u;
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

// floor(a / b) for 0 <= a < 2^22 and b >= 1 by one FP32 reciprocal: the
// error of (a + 0.5) * rn(1/b) stays below 2^-23 (a + 0.5) / b < 0.5 / b,
// the distance of (a + 0.5) / b from the nearest integer, so the floor is
// exact.  (Integer division by a runtime divisor is a long emulated
// sequence.)
__device__ __forceinline__ unsigned div_small(unsigned a, unsigned b, float rb) {
  return (unsigned)__fmul_rn((float)a + 0.5f, rb);
}

// q-th cell (x fastest) of an nx x ny x nz range; q < 2^31 (the cell paths
// only run for ranges below the flat-scan threshold), so 32-bit division
// suffices -- 64-bit division is emulated and far slower; below 2^22 cells
// the reciprocal form above replaces it.
__device__ __forceinline__ void decode_cell(long long q, int nx, int ny, int& dx, int& dy, int& dz) {
  const unsigned uq = (unsigned)q;
  unsigned r, z;
  if (uq < (1u << 22)) {
    r = div_small(uq, (unsigned)nx, __frcp_rn((float)nx));
    z = div_small(r, (unsigned)ny, __frcp_rn((float)ny));
  } else {
    r = uq / (unsigned)nx;
    z = r / (unsigned)ny;
  }
  dx = (int)(uq - r * (unsigned)nx);
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

// Keep the candidate with the smallest maxd^2 over the box seen so far (the
// best bound of the next pass's phase A).
__device__ __forceinline__ void note_ref(const float4& lo, const float4& hi, const float4& c,
                                         int d, float& ref_m, int& ref_id) {
  const float mc = maxd2(lo, hi, c.x, c.y, c.z, d);
  if (mc < ref_m) {
    ref_m = mc;
    ref_id = __float_as_int(c.w);
  }
}

// The candidate search of search unit t (one warp), list to tlist / tcnt.
// MULTI = false: a single cloud, whose table entry is read from the kernel
// parameters (constant bank) instead of global memory.
template <bool MULTI, int D>
__device__ __forceinline__ void search_unit(const IterArgs& A, int par, int t) {
  constexpr int d = D;
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
          A.tref[t] = a;
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

  // ---- phase A ----
  // Any centroid of the cloud bounds the nearest distance of every point in
  // the box by maxd(box, c).  The candidate of the previous pass's list with
  // the smallest maxd over the box (tref) lies near the tile, so its
  // current position gives U in one load; an id outside the cloud (left by
  // another tiling) is not used.  Without a usable reference, rings of cells around the box
  // are scanned.  The centroid that gives U (r1) also serves as the
  // dominance reference of phase B (the kNN bound inherited from the
  // previous pass, in the spirit of Section IV-A's bounds from parent
  // nodes).
  float u2 = INFINITY;
  float m = INFINITY;
  float4 r1 = make_float4(0.f, 0.f, 0.f, 0.f);   // this lane's best so far
  const int ref = A.tref[t];
  if (ref >= c0 && ref < c1) {
    // the previous pass's reference centroid, at its current position: one
    // dependent load, the same on every lane
    r1 = A.cw[ref];
    m = maxd2(lo, hi, r1.x, r1.y, r1.z, d);
    u2 = m;
  }
  int clo[3], chi[3];   // the box's own cells (only the ring search needs them)
  if (!(u2 < INFINITY)) {
    clo[0] = cell_coord(lo.x, G.g0[0], G.inv_s, G.dims[0]);
    chi[0] = cell_coord(hi.x, G.g0[0], G.inv_s, G.dims[0]);
    clo[1] = cell_coord(lo.y, G.g0[1], G.inv_s, G.dims[1]);
    chi[1] = cell_coord(hi.y, G.g0[1], G.inv_s, G.dims[1]);
    clo[2] = d == 3 ? cell_coord(lo.z, G.g0[2], G.inv_s, G.dims[2]) : 0;
    chi[2] = d == 3 ? cell_coord(hi.z, G.g0[2], G.inv_s, G.dims[2]) : 0;
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
    r1.w = __shfl_sync(0xffffffffu, r1.w, src);
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
  float ref_m = INFINITY;   // the kept candidate with the smallest maxd^2: the next reference
  int ref_id = -1;
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
      if (keep) note_ref(lo, hi, c, d, ref_m, ref_id);
      unsigned bal = __ballot_sync(0xffffffffu, keep);
      int pos = count + __popc(bal & lt);
      if (keep && pos < kTileCap) out[pos] = c;
      count += __popc(bal);
    }
  } else {
    // The range's cells, 32 per round, one per lane; their bucket entries
    // are then taken 32 at a time across the lanes (each lane finds the
    // cell that holds its entry by a binary search over the cells'
    // exclusive count prefix), so a round costs ceil(entries / 32) tests
    // instead of the fullest cell's count.
    bool any_ovf = false;   // a cell of the range overflowed into the list
    for (long long q0 = 0; q0 < ncell; q0 += 32) {
      const long long q = q0 + lane;
      int cell = 0;   // within the cloud's grid (fewer than 2^31 cells: they fit device memory)
      int cnt = 0;
      if (q < ncell) {
        int ox, oy, oz;
        decode_cell(q, nx, ny, ox, oy, oz);
        cell = ((rlo[2] + oz) * G.dims[1] + (rlo[1] + oy)) * G.dims[0] + (rlo[0] + ox);
        const int raw = gcnt[cell];
        any_ovf = any_ovf || raw > kBucketCap;
        cnt = min(raw, kBucketCap);
      }
      int incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      const int excl = incl - cnt;
      for (int j0 = 0; j0 < total; j0 += 32) {
        const int j = j0 + lane;
        int L = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const int e = __shfl_sync(0xffffffffu, excl, L + step);
          if (e <= j) L += step;
        }
        const int cl = __shfl_sync(0xffffffffu, cell, L);
        const int slot = j - __shfl_sync(0xffffffffu, excl, L);
        float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
        bool keep = false;
        if (j < total) {
          e = gbkt[cl * kBucketCap + slot];
          keep = mind2(lo, hi, e.x, e.y, e.z, d) <= u2k &&
                 !dominated(lo, hi, r1, slack, e.x, e.y, e.z, d);
          if (keep) note_ref(lo, hi, e, d, ref_m, ref_id);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        const int pos = count + __popc(bal & lt);
        if (keep && pos < kTileCap) out[pos] = e;
        count += __popc(bal);
      }
    }
    // overflow entries live only in cells counted above kBucketCap
    if (__any_sync(0xffffffffu, any_ovf)) {
      for (int q0 = 0; q0 < n_ovf; q0 += 32) {
        int q = q0 + lane;
        float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
        bool keep = false;
        if (q < n_ovf) {
          c = ovf[q];
          keep = mind2(lo, hi, c.x, c.y, c.z, d) <= u2k &&
                 !dominated(lo, hi, r1, slack, c.x, c.y, c.z, d);
          if (keep) note_ref(lo, hi, c, d, ref_m, ref_id);
        }
        unsigned bal = __ballot_sync(0xffffffffu, keep);
        int pos = count + __popc(bal & lt);
        if (keep && pos < kTileCap) out[pos] = c;
        count += __popc(bal);
      }
    }
  }
  {
    const float bm = warp_min_nonneg(ref_m);
    const int src = __ffs(__ballot_sync(0xffffffffu, ref_m == bm)) - 1;
    const int rid = __shfl_sync(0xffffffffu, ref_id, src);
    if (lane == 0) A.tref[t] = rid;
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

template <bool MULTI, int D>
__global__ void __launch_bounds__(32 * kSearchWarps, DKM_SEARCH_MIN_BLOCKS)
    k_search(const __grid_constant__ IterArgs A, int par) {
  // every cloud stopped (fixed during this kernel; only early-stopping runs stop)
  if (A.early_stop && A.st->n_done == A.B) return;
  clear_other_parity(A, par);
  const int t = blockIdx.x * kSearchWarps + (threadIdx.x >> 5);
  if (t >= A.n_units) return;   // t: the search unit (a tile or a group of tiles)
  search_unit<MULTI, D>(A, par, t);
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

// The same choice when the candidates arrive in ascending id order: a
// strictly smaller distance is then the only way to win (an equal distance
// came with a lower id earlier), one compare instead of the 64-bit key's two.
__device__ __forceinline__ void take_min_ordered(float s, int id, float& best, int& bid) {
  if (s < best) {
    best = s;
    bid = id;
  }
}

#ifndef DKM_EVAL_UNROLL
#define DKM_EVAL_UNROLL 1
#endif
constexpr int kEvalUnroll = DKM_EVAL_UNROLL;   // candidates per unrolled step
// all rows of the tile against candidates s_c[idx[j]] (idx == nullptr:
// s_c[j]); ORD: the candidates come in ascending id order
template <int D, bool ORD = false>
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
      if (ORD) {
        take_min_ordered(s.x, id, best[r].x, bid[r].x);
        take_min_ordered(s.y, id, best[r].y, bid[r].y);
      } else {
        take_min(s.x, id, best[r].x, bid[r].x);
        take_min(s.y, id, best[r].y, bid[r].y);
      }
    }
  }
}

// one row (64 points, two per lane) against candidates s_c[idx[j]]
template <int D, bool ORD = false>
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
    if (ORD) {
      take_min_ordered(s.x, id, best.x, bid.x);
      take_min_ordered(s.y, id, best.y, bid.y);
    } else {
      take_min(s.x, id, best.x, bid.x);
      take_min(s.y, id, best.y, bid.y);
    }
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

// The entries of src[0..m) (global memory) that can hold the nearest
// centroid of some point inside [lo, hi], written compactly to out (shared
// memory, m <= kTileCap); returns the count.  U = min over the list of
// maxd(box, c) bounds every point's nearest distance (any centroid of the
// cloud does), and a point's nearest centroid c* has mind(box, c*) <= U.
template <int D>
__device__ __forceinline__ int filter_list(const float4* __restrict__ src, int m, float4 lo,
                                           float4 hi, float4* __restrict__ out, bool slot_keys) {
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
    const int pos = cnt + __popc(bal & lt);
    if (slot_keys) c.w = __int_as_float((__float_as_int(c.w) << 8) | pos);
    if (keep) out[pos] = c;
    cnt += __popc(bal);
  }
  __syncwarp();
  return cnt;
}

// ---------------------------------------------------------------------------
// Update sums of one tile (the refine step's sv(j) of Algorithm 1, in exact
// integer arithmetic).  Each point's residual r = p - c_label (FP32, the
// same p + (-c) as the distance) is scaled by one tile-wide power of two
// 2^s and rounded to an integer q; the q of a label's points are summed in
// int32 across the warp and added, rescaled to the cloud's unit 2^-s_glob,
// to that centroid's 64-bit accumulators with integer atomics.  Integer
// addition is exact and order independent, so the centroids do not depend
// on the order of the atomics.
//
// Scale: every |r_axis| <= sqrt(max d^2) < 2^ceil(e2/2) with max d^2 <
// 2^e2 over the tile's points, so s = 22 - ceil(e2/2) keeps |r * 2^s| below
// 2^22 and a 256-point sum below 2^30.  Rounding: fma(r, 2^s, 1.5 * 2^23)
// leaves round-to-nearest-even(r * 2^s) in the low bits of the float
// (exact while |r * 2^s| <= 2^22); the raw bit patterns are summed with
// wrap-around and the 0x4B400000 offset of the cnt summands is taken off
// once per group.
//
// Every caller (k_assign's list and global paths, k_accum_labels for
// caller-given labels) passes the same residuals and squared norms for the
// same labels, so the sums agree bit for bit whatever grouping it uses.
// ---------------------------------------------------------------------------
constexpr int kPts = 2 * kRowsPerWarp;      // points per lane
constexpr float kMagic = 12582912.0f;       // 1.5 * 2^23
constexpr unsigned kMagicBits = 0x4B400000u;

__device__ __forceinline__ int residual_scale(float m2) {
  if (!(m2 > 0.f)) return 0;
  const int e2 = exp_bound(m2);
  return min(22 - ((e2 + 1) >> 1), 127);
}

__device__ __forceinline__ void add_group(const IterArgs& A, int D, int L, int sx, int sy, int sz,
                                          int cnt, int s_q, int s_glob) {
  Acc* a = &A.acc[L];
  red_add_u64(&a->s[0], (unsigned long long)rescale(sx, s_q, s_glob));
  red_add_u64(&a->s[1], (unsigned long long)rescale(sy, s_q, s_glob));
  if (D == 3) red_add_u64(&a->s[2], (unsigned long long)rescale(sz, s_q, s_glob));
  red_add_u64(&a->cnt, (unsigned long long)cnt);
}

// q(r) = the raw float bits of fma(r, 2^s, 1.5 * 2^23): round(r * 2^s) +
// 0x4B400000 for |r * 2^s| <= 2^22.
__device__ __forceinline__ unsigned quantize(float r, float scl) {
  return __float_as_uint(__fmaf_rn(r, scl, kMagic));
}

// Groups are keyed by g: the label itself, or (slots) the candidate-list
// position whose entry sc[g] carries (label << 8 | g) in .w.  q*: the
// quantized residuals (quantize) at scale 2^s_t.  With mask_keys every key
// is below 32 and the distinct keys are taken from one warp-wide bit mask;
// otherwise the smallest pending key is taken in turn.  Returns the tile's
// label when all its points share one, else -1.
template <int D>
__device__ __forceinline__ int tile_sums(const IterArgs& A, const unsigned (&qx)[kPts],
                                         const unsigned (&qy)[kPts], const unsigned (&qz)[kPts],
                                         const int (&g)[kPts], const bool (&pv)[kPts], int s_t,
                                         bool slots, bool mask_keys,
                                         const float4* __restrict__ sc, int s_glob) {
  const int lane = threadIdx.x & 31;
  auto label_of = [&](int key) { return slots ? (__float_as_int(sc[key].w) >> 8) : key; };
  auto flush = [&](int key, bool all) {
    unsigned sx = 0, sy = 0, sz = 0, cnt = 0;
#pragma unroll
    for (int h = 0; h < kPts; ++h) {
      const bool in = pv[h] && (all || g[h] == key);
      sx += in ? qx[h] : 0u;
      sy += in ? qy[h] : 0u;
      if (D == 3) sz += in ? qz[h] : 0u;
      cnt += in ? 1u : 0u;
    }
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    sx = __reduce_add_sync(0xffffffffu, sx) - cnt * kMagicBits;
    sy = __reduce_add_sync(0xffffffffu, sy) - cnt * kMagicBits;
    if (D == 3) sz = __reduce_add_sync(0xffffffffu, sz) - cnt * kMagicBits;
    if (lane == 0)
      add_group(A, D, label_of(key), (int)sx, (int)sy, (int)sz, (int)cnt, s_t, s_glob);
  };
  if (mask_keys) {
    unsigned m = 0;
#pragma unroll
    for (int h = 0; h < kPts; ++h) m |= pv[h] ? (1u << g[h]) : 0u;
    m = __reduce_or_sync(0xffffffffu, m);
    if (m == 0) return -1;
    if ((m & (m - 1)) == 0) {   // one group: every valid point
      const int key = __ffs(m) - 1;
      flush(key, true);
      return label_of(key);
    }
    while (m) {
      const int key = __ffs(m) - 1;
      m &= m - 1;
      flush(key, false);
    }
    return -1;
  }
  int lmin = INT_MAX, lmax = INT_MIN;
#pragma unroll
  for (int h = 0; h < kPts; ++h) {
    lmin = pv[h] ? min(lmin, g[h]) : lmin;
    lmax = pv[h] ? max(lmax, g[h]) : lmax;
  }
  int key = __reduce_min_sync(0xffffffffu, lmin);
  if (key == INT_MAX) return -1;
  if (__reduce_max_sync(0xffffffffu, lmax) == key) {   // one group
    flush(key, true);
    return label_of(key);
  }
  while (key != INT_MAX) {
    flush(key, false);
    lmin = INT_MAX;
#pragma unroll
    for (int h = 0; h < kPts; ++h) lmin = (pv[h] && g[h] > key) ? min(lmin, g[h]) : lmin;
    key = __reduce_min_sync(0xffffffffu, lmin);
  }
  return -1;
}

// The same sums for a tile whose points are keyed by candidate-list
// position (sc[g].w = label << 8 | g): each group reads its centroid once
// from shared memory and quantizes its points' residuals on the fly, so no
// per-point residual is kept in registers.  The residual and its rounding
// are those of quantize(p + (-c)), as in every other caller.
template <int D>
__device__ __forceinline__ int tile_sums_slots(const IterArgs& A, const Pts<D>& P,
                                               const unsigned (&gs)[2], unsigned pm, int s_t,
                                               int q, const float4* __restrict__ sc, int s_glob) {
  // gs: the points' list positions, one byte each (point h in byte h & 3 of
  // gs[h >> 2]); pm: bit h set for a valid point h
  const int lane = threadIdx.x & 31;
  const float scl = pow2f(s_t);
  auto slot = [&](int h) { return (int)((gs[h >> 2] >> (8 * (h & 3))) & 0xffu); };
  auto flush = [&](int key, bool all) {
    const float4 c = sc[key];
    unsigned sx = 0, sy = 0, sz = 0, cnt = 0;
#pragma unroll
    for (int r = 0; r < kRowsPerWarp; ++r) {
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int h = 2 * r + hh;
        const bool in = ((pm >> h) & 1u) && (all || slot(h) == key);
        const unsigned ux = quantize(__fadd_rn(hh ? P.x[r].y : P.x[r].x, -c.x), scl);
        const unsigned uy = quantize(__fadd_rn(hh ? P.y[r].y : P.y[r].x, -c.y), scl);
        sx += in ? ux : 0u;
        sy += in ? uy : 0u;
        if (D == 3) {
          const unsigned uz = quantize(__fadd_rn(hh ? P.z[r].y : P.z[r].x, -c.z), scl);
          sz += in ? uz : 0u;
        }
        cnt += in ? 1u : 0u;
      }
    }
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    sx = __reduce_add_sync(0xffffffffu, sx) - cnt * kMagicBits;
    sy = __reduce_add_sync(0xffffffffu, sy) - cnt * kMagicBits;
    if (D == 3) sz = __reduce_add_sync(0xffffffffu, sz) - cnt * kMagicBits;
    if (lane == 0)
      add_group(A, D, __float_as_int(c.w) >> 8, (int)sx, (int)sy, (int)sz, (int)cnt, s_t, s_glob);
    return __float_as_int(c.w) >> 8;
  };
  if (q <= 32) {
    unsigned m = 0;
#pragma unroll
    for (int h = 0; h < kPts; ++h) m |= ((pm >> h) & 1u) ? (1u << slot(h)) : 0u;
    m = __reduce_or_sync(0xffffffffu, m);
    if (m == 0) return -1;
    if ((m & (m - 1)) == 0) return flush(__ffs(m) - 1, true);   // one group
    while (m) {
      const int key = __ffs(m) - 1;
      m &= m - 1;
      flush(key, false);
    }
    return -1;
  }
  int lmin = INT_MAX, lmax = INT_MIN;
#pragma unroll
  for (int h = 0; h < kPts; ++h) {
    const bool v = (pm >> h) & 1u;
    lmin = v ? min(lmin, slot(h)) : lmin;
    lmax = v ? max(lmax, slot(h)) : lmax;
  }
  int key = __reduce_min_sync(0xffffffffu, lmin);
  if (key == INT_MAX) return -1;
  if (__reduce_max_sync(0xffffffffu, lmax) == key) return flush(key, true);
  while (key != INT_MAX) {
    flush(key, false);
    lmin = INT_MAX;
#pragma unroll
    for (int h = 0; h < kPts; ++h)
      lmin = (((pm >> h) & 1u) && slot(h) > key) ? min(lmin, slot(h)) : lmin;
    key = __reduce_min_sync(0xffffffffu, lmin);
  }
  return -1;
}

// The same sums, row by row, for a tile whose staged list has at most 32
// entries (keys are list positions < 32).  Each point quantizes its residual
// to its own staged centroid once; every row (64 points) then adds each of
// its groups to a per-warp shared-memory accumulator of that list position
// (one writer, lane 0, so no atomics), and the warp's lanes flush the
// positions that received points to the global accumulators together.
// Rows hold fewer distinct labels than whole tiles, so each point is
// visited by fewer groups.  Int32 accumulation cannot overflow: a tile's
// points sum below 2^30 per axis (residual_scale).  Returns the tile's
// label when all its points share one, else -1.
template <int D>
__device__ __forceinline__ int tile_sums_rows(const IterArgs& A, const Pts<D>& P,
                                              const int2 (&bid)[kRowsPerWarp],
                                              const bool (&va)[kRowsPerWarp],
                                              const bool (&vb)[kRowsPerWarp],
                                              const int (&nv_row)[kRowsPerWarp], int s_t, int q,
                                              const float4* __restrict__ sc,
                                              int4* __restrict__ sacc, int s_glob) {
  const int lane = threadIdx.x & 31;
  const float scl = pow2f(s_t);
  if (lane < q) sacc[lane] = make_int4(0, 0, 0, 0);
  __syncwarp();
  unsigned tile_mask = 0;
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r) {
    if (nv_row[r] == 0) continue;   // warp-uniform
    const int ga = bid[r].x & 255, gb = bid[r].y & 255;
    const float4 ca = sc[ga], cb = sc[gb];
    const unsigned ax = quantize(__fadd_rn(P.x[r].x, -ca.x), scl);
    const unsigned ay = quantize(__fadd_rn(P.y[r].x, -ca.y), scl);
    const unsigned az = D == 3 ? quantize(__fadd_rn(P.z[r].x, -ca.z), scl) : kMagicBits;
    const unsigned bx = quantize(__fadd_rn(P.x[r].y, -cb.x), scl);
    const unsigned by = quantize(__fadd_rn(P.y[r].y, -cb.y), scl);
    const unsigned bz = D == 3 ? quantize(__fadd_rn(P.z[r].y, -cb.z), scl) : kMagicBits;
    unsigned m = (va[r] ? 1u << ga : 0u) | (vb[r] ? 1u << gb : 0u);
    m = __reduce_or_sync(0xffffffffu, m);
    tile_mask |= m;
    while (m) {
      const int key = __ffs(m) - 1;
      m &= m - 1;
      const bool ia = va[r] && ga == key, ib = vb[r] && gb == key;
      unsigned sx = (ia ? ax : 0u) + (ib ? bx : 0u);
      unsigned sy = (ia ? ay : 0u) + (ib ? by : 0u);
      unsigned sz = (ia ? az : 0u) + (ib ? bz : 0u);
      const unsigned cnt = __reduce_add_sync(0xffffffffu, (unsigned)ia + (unsigned)ib);
      sx = __reduce_add_sync(0xffffffffu, sx) - cnt * kMagicBits;
      sy = __reduce_add_sync(0xffffffffu, sy) - cnt * kMagicBits;
      if (D == 3) sz = __reduce_add_sync(0xffffffffu, sz) - cnt * kMagicBits;
      if (lane == 0) {
        int4 a = sacc[key];
        a.x += (int)sx;
        a.y += (int)sy;
        a.z += (int)sz;
        a.w += (int)cnt;
        sacc[key] = a;
      }
    }
  }
  __syncwarp();
  if (lane < q) {
    const int4 a = sacc[lane];
    if (a.w > 0)
      add_group(A, D, __float_as_int(sc[lane].w) >> 8, a.x, a.y, a.z, a.w, s_t, s_glob);
  }
  if (tile_mask != 0 && (tile_mask & (tile_mask - 1)) == 0)
    return __float_as_int(sc[__ffs(tile_mask) - 1].w) >> 8;
  return -1;
}

// Quantized residuals of a tile's points against their labels' centroids
// read from the working centroids (global memory); returns the scale
// exponent s_t (residual_scale of the tile's max squared residual norm).
template <int D>
__device__ __forceinline__ int residuals_global(const IterArgs& A,
                                                const float2 (&px)[kRowsPerWarp],
                                                const float2 (&py)[kRowsPerWarp],
                                                const float2 (&pz)[kRowsPerWarp],
                                                const int (&lb)[kPts], const bool (&pv)[kPts],
                                                unsigned (&qx)[kPts], unsigned (&qy)[kPts],
                                                unsigned (&qz)[kPts]) {
  float rx[kPts], ry[kPts], rz[kPts];
  float m2 = 0.f;
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r) {
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const int h = 2 * r + hh;
      rx[h] = ry[h] = rz[h] = 0.f;
      if (pv[h]) {
        const float4 c = __ldg(&A.cw[lb[h]]);
        rx[h] = __fadd_rn(hh ? px[r].y : px[r].x, -c.x);
        ry[h] = __fadd_rn(hh ? py[r].y : py[r].x, -c.y);
        if (D == 3) rz[h] = __fadd_rn(hh ? pz[r].y : pz[r].x, -c.z);
        float d2 = __fmaf_rn(ry[h], ry[h], __fmul_rn(rx[h], rx[h]));
        if (D == 3) d2 = __fmaf_rn(rz[h], rz[h], d2);
        m2 = fmaxf(m2, d2);
      }
    }
  }
  const int s_t = residual_scale(warp_max_nonneg(m2));
  const float scl = pow2f(s_t);
#pragma unroll
  for (int h = 0; h < kPts; ++h) {
    qx[h] = quantize(rx[h], scl);
    qy[h] = quantize(ry[h], scl);
    qz[h] = quantize(rz[h], scl);
  }
  return s_t;
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
  // window-relative 32-bit offsets: one 64-bit address per coordinate row
  const float* __restrict__ px = A.xs + base;
  const float* __restrict__ py = A.ys + base;
  const float* __restrict__ pz = A.zs + base;
  const int lo = (int)(vlo - base), hi = (int)(vhi - base);
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r) {
    const int o = r * kRowPts + 2 * lane;
    x[r] = *reinterpret_cast<const float2*>(px + o);
    y[r] = *reinterpret_cast<const float2*>(py + o);
    z[r] = D == 3 ? *reinterpret_cast<const float2*>(pz + o) : make_float2(0.f, 0.f);
    va[r] = o >= lo && o < hi;
    vb[r] = o + 1 >= lo && o + 1 < hi;
  }
}

// Assignment of tile t (one warp) from its search unit's candidate list:
// labels, SSE and the update sums.  sc / sr / slbw: the warp's shared
// staging (kTileCap candidates, kTileCap indices, 32 bounds).
template <int D, bool BRUTE, bool MULTI, bool UNITS, bool PSTAY>
__device__ __forceinline__ void assign_tile(const IterArgs& A, int t, float4* __restrict__ sc,
                                            unsigned short* __restrict__ sr,
                                            float* __restrict__ slbw, int4* __restrict__ sacc) {
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
  // valid points per row: the tile's range [lo, hi) of the window cut by
  // the row's [64 r, 64 r + 64) (warp-uniform arithmetic)
  int nv_row[kRowsPerWarp];
  {
    const int lo = se.x - (int)base, hi = se.y - (int)base;
#pragma unroll
    for (int r = 0; r < kRowsPerWarp; ++r)
      nv_row[r] = max(0, min(hi, (r + 1) * kRowPts) - max(lo, r * kRowPts));
  }
  const int nv_tile = se.y - se.x;

  float2 best[kRowsPerWarp];
  int2 bid[kRowsPerWarp];
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r) {
    best[r] = make_float2(INFINITY, INFINITY);
    bid[r] = make_int2(0, 0);
  }
  unsigned long long evals = 0;   // point x candidate evaluations of this warp
  bool slots = false;             // candidate keys carry list positions (see below)
  bool ordered = false;           // the staged list is in ascending id order
  int q_tile = 0;                 // length of the staged list
  // point stay test (stay == 2): per point its kept label (or -1) and its
  // squared distance; rows whose valid points all stay
  int sl[kPts];
  float sd[kPts];
  unsigned row_stay = 0u;
  int n_pstay = 0;
  bool any_pstay = false;
  if (BRUTE) {
    for (int j0 = c0; j0 < c1; j0 += kTileCap) {
      const int m = min(kTileCap, c1 - j0);
      __syncwarp();
      for (int i = lane; i < m; i += 32) sc[i] = A.cw[j0 + i];
      __syncwarp();
      eval_list<D, true>(sc, nullptr, m, P, best, bid);   // ids ascend with j
    }
    evals = (unsigned long long)cl.k * nv_tile;
  } else {
    const int u = UNITS ? A.tunit[t] : t;   // the tile's search unit
    const int qs = A.tcnt[u];
    if (qs == 0 && lane == 0) atomicOr(&A.st->err, kErrEmptyList);
    if (qs <= kTileCap) {
      const float4* __restrict__ src = A.tlist + (int64_t)u * kTileCap;
      // Staged entries carry (id << 8 | list position) in .w when ids fit
      // 24 bits: the (d^2, key) order is the (d^2, id) order, and the
      // winner's position finds its centroid in shared memory for the
      // update sums.
      slots = A.slot_keys != 0;
      int q = qs;
      if (UNITS) {
        // the unit's list holds every candidate of the group's box; narrow
        // it with this tile's own box (the bound of k_search)
        q = filter_list<D>(src, qs, A.tbox[2 * t], A.tbox[2 * t + 1], sc, slots);
      } else if (qs <= 32) {
        // a short list is placed in ascending id order (the rank of each
        // entry among the list's distinct ids), so that the candidate loops
        // below can keep the lowest id of equal distances by order alone
        const bool has = lane < qs;
        float4 c = has ? src[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
        const int id = has ? __float_as_int(c.w) : INT_MAX;
        int rank = 0;
        for (int m2 = 0; m2 < qs; ++m2) rank += __shfl_sync(0xffffffffu, id, m2) < id;
        if (has) {
          if (slots) c.w = __int_as_float((id << 8) | rank);
          sc[rank] = c;
        }
        __syncwarp();
        ordered = true;
      } else {
        for (int i = lane; i < qs; i += 32) {
          float4 c = src[i];
          if (slots) c.w = __int_as_float((__float_as_int(c.w) << 8) | i);
          sc[i] = c;
        }
        __syncwarp();
      }
      q_tile = q;
      if (PSTAY) {
        // The point test of the bound layer (Eq. interbound1; the leaf
        // branch of Algorithm 1's Assign): a point within cb[a]/2 of its
        // last centroid c_a still has c_a as its unique nearest centroid.
        // Rows whose points all pass skip the candidate loop.
#pragma unroll
        for (int r = 0; r < kRowsPerWarp; ++r) {
          bool ok[2];
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            const int h = 2 * r + hh;
            const bool v = hh ? vb[r] : va[r];
            ok[hh] = !v;
            sl[h] = -1;
            if (v) {
              const int a = A.lab[base + r * kRowPts + 2 * lane + hh];
              if (a >= c0 && a < c1) {
                const float4 c = __ldg(&A.cw[a]);
                const float dx = __fadd_rn(hh ? P.x[r].y : P.x[r].x, -c.x);
                const float dy = __fadd_rn(hh ? P.y[r].y : P.y[r].x, -c.y);
                float d2 = __fmaf_rn(dy, dy, __fmul_rn(dx, dx));
                if (D == 3) {
                  const float dz = __fadd_rn(hh ? P.z[r].y : P.z[r].x, -c.z);
                  d2 = __fmaf_rn(dz, dz, d2);
                }
                if (d2 <= kStay * __ldg(&A.cb2[a])) {
                  sl[h] = a;
                  sd[h] = d2;
                  ok[hh] = true;
                  ++n_pstay;
                }
              }
            }
          }
          if (__all_sync(0xffffffffu, ok[0] && ok[1])) row_stay |= 1u << r;
        }
        any_pstay = __any_sync(0xffffffffu, n_pstay > 0);
      }
      if (PSTAY && row_stay == 0xfu) {
        // every point keeps its label: no candidate is evaluated
      } else if (PSTAY && row_stay != 0u) {
        for (int i = lane; i < q; i += 32) sr[i] = (unsigned short)i;
        __syncwarp();
#pragma unroll
        for (int r = 0; r < kRowsPerWarp; ++r) {
          if (nv_row[r] == 0 || ((row_stay >> r) & 1u)) continue;   // warp-uniform
          if (ordered) eval_row<D, true>(sc, sr, q, P.x[r], P.y[r], P.z[r], best[r], bid[r]);
          else eval_row<D>(sc, sr, q, P.x[r], P.y[r], P.z[r], best[r], bid[r]);
          evals += (unsigned long long)q * nv_row[r];
        }
      } else if (q <= A.sort_max) {   // sort_max <= 32
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
          const int mr = filter_box<D>(sc, q, rlo, rhi, INFINITY, sr);   // keeps the order
          if (ordered) eval_row<D, true>(sc, sr, mr, P.x[r], P.y[r], P.z[r], best[r], bid[r]);
          else eval_row<D>(sc, sr, mr, P.x[r], P.y[r], P.z[r], best[r], bid[r]);
          evals += (unsigned long long)mr * nv_row[r];
        }
      } else if (ordered) {
        eval_list<D, true>(sc, nullptr, q, P, best, bid);
        evals = (unsigned long long)q * nv_tile;
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
  int lb[kPts], gk[kPts];   // label (context-wide id) and group key of each point
  bool pv[kPts];
  float m2 = 0.f;           // max squared distance of the lane's valid points
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r) {
    const int ka = bid[r].x, kb = bid[r].y;
    lb[2 * r] = slots ? ka >> 8 : ka;
    lb[2 * r + 1] = slots ? kb >> 8 : kb;
    if (PSTAY && any_pstay) {   // points that kept their label: theirs, with its distance
      if (sl[2 * r] >= 0) {
        lb[2 * r] = sl[2 * r];
        best[r].x = sd[2 * r];
      }
      if (sl[2 * r + 1] >= 0) {
        lb[2 * r + 1] = sl[2 * r + 1];
        best[r].y = sd[2 * r + 1];
      }
    }
    gk[2 * r] = slots ? ka & 255 : lb[2 * r];
    gk[2 * r + 1] = slots ? kb & 255 : lb[2 * r + 1];
    pv[2 * r] = va[r];
    pv[2 * r + 1] = vb[r];
    m2 = fmaxf(m2, fmaxf(va[r] ? best[r].x : 0.f, vb[r] ? best[r].y : 0.f));
  }
  if (PSTAY && any_pstay) slots = false;   // the kept labels carry no list position
  int32_t* __restrict__ wlab = A.lab + base;   // the window's labels (32-bit offsets)
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r) {
    if (nv_row[r] == 0) continue;   // warp-uniform
    const int o = r * kRowPts + 2 * lane;
    const int la = lb[2 * r], lc = lb[2 * r + 1];
    if (A.track_changes) {
      int pa = va[r] ? wlab[o] : la, pb = vb[r] ? wlab[o + 1] : lc;
      changed += (int)(pa != la) + (int)(pb != lc);
    }
    if (va[r] && vb[r]) {
      *reinterpret_cast<int2*>(wlab + o) = make_int2(la, lc);
    } else if (va[r]) {
      wlab[o] = la;
    } else if (vb[r]) {
      wlab[o + 1] = lc;
    }
  }
  if (A.want_sse) sse = tile_sse(best, va, vb, s_sse);
  int single;
  if (slots) {
    // the tile's max squared residual norm is its max best d^2
    const int s_t = residual_scale(warp_max_nonneg(m2));
    if (q_tile <= 32) {
      single = tile_sums_rows<D>(A, P, bid, va, vb, nv_row, s_t, q_tile, sc, sacc, s_glob);
    } else if (MULTI) {
      // Batches of dense clouds (where most long lists occur): each point's
      // residual quantized once against its own staged centroid, then
      // grouped by list position over the whole tile.  (The single-cloud
      // kernel keeps the form below: these registers would spill on its
      // hot path.)
      const float scl = pow2f(s_t);
      unsigned qx[kPts], qy[kPts], qz[kPts];
#pragma unroll
      for (int r = 0; r < kRowsPerWarp; ++r) {
        const float4 ca = sc[gk[2 * r]], cb = sc[gk[2 * r + 1]];
        qx[2 * r] = quantize(__fadd_rn(P.x[r].x, -ca.x), scl);
        qy[2 * r] = quantize(__fadd_rn(P.y[r].x, -ca.y), scl);
        qz[2 * r] = D == 3 ? quantize(__fadd_rn(P.z[r].x, -ca.z), scl) : kMagicBits;
        qx[2 * r + 1] = quantize(__fadd_rn(P.x[r].y, -cb.x), scl);
        qy[2 * r + 1] = quantize(__fadd_rn(P.y[r].y, -cb.y), scl);
        qz[2 * r + 1] = D == 3 ? quantize(__fadd_rn(P.z[r].y, -cb.z), scl) : kMagicBits;
      }
      single = tile_sums<D>(A, qx, qy, qz, gk, pv, s_t, true, false, sc, s_glob);
    } else {
      // each group re-quantizes its points on the fly (no per-point
      // residuals kept in registers)
      unsigned gs[2] = {0u, 0u}, pm = 0u;
#pragma unroll
      for (int h = 0; h < kPts; ++h) {
        gs[h >> 2] |= (unsigned)gk[h] << (8 * (h & 3));
        pm |= pv[h] ? (1u << h) : 0u;
      }
      single = tile_sums_slots<D>(A, P, gs, pm, s_t, q_tile, sc, s_glob);
    }
  } else {
    unsigned qx[kPts], qy[kPts], qz[kPts];
    const int s_t = residuals_global<D>(A, P.x, P.y, P.z, lb, pv, qx, qy, qz);
    single = tile_sums<D>(A, qx, qy, qz, lb, pv, s_t, false, false, sc, s_glob);
  }
  changed = __reduce_add_sync(0xffffffffu, changed);
  if (lane == 0) {
    if (A.stay) A.tlab[t] = single;
    CloudAcc& ca = A.cacc[b];
    if (sse) red_add_u64(&ca.sse[t & (kCloudSlots - 1)], (unsigned long long)sse);
    if (changed) red_add_u64(&ca.changed[t & (kCloudSlots - 1)], (unsigned long long)changed);
    if (A.want_stats) red_add_u64(&A.slots[t & (kSlots - 1)].evals, evals);
  }
  if (PSTAY && A.want_stats && any_pstay) {
    const int np = __reduce_add_sync(0xffffffffu, n_pstay);
    if (lane == 0) red_add_u64(&A.slots[t & (kSlots - 1)].pstays, (unsigned long long)np);
  }
}


// UNITS: tiles share search units (tile_group > 1) and filter their unit's
// list with their own box.  PSTAY: the point stay test of the bound layer.
template <int D, bool BRUTE, bool MULTI, bool UNITS, bool PSTAY>
__global__ void __launch_bounds__(32 * kAssignWarps, DKM_ASSIGN_MIN_WARPS / kAssignWarps)
    k_assign(const __grid_constant__ IterArgs A) {
  __shared__ float4 s_c[kAssignWarps][kTileCap];
  __shared__ unsigned short s_r[kAssignWarps][kTileCap];
  __shared__ float slb[kAssignWarps][32];
  __shared__ int4 s_acc[kAssignWarps][32];
  // every cloud stopped (fixed during this kernel; only early-stopping runs stop)
  if (A.early_stop && A.st->n_done == A.B) return;
  const int w = threadIdx.x >> 5;
  const int t = blockIdx.x * kAssignWarps + w;
  if (t >= A.n_tiles) return;   // warp-level exits, no CTA barrier below
  assign_tile<D, BRUTE, MULTI, UNITS, PSTAY>(A, t, s_c[w], s_r[w], slb[w], s_acc[w]);
}

// ---------------------------------------------------------------------------
// k_accum_labels: residual sums for a caller-given labelling (dkm_update;
// cloud-local labels).  One warp per tile with k_assign's per-tile scale, so
// both produce the same sums bit for bit for the same labels.
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
  int lab[kPts];
  bool ok[kPts];
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r) {
    const int64_t i = base + r * kRowPts + 2 * lane;
    const int la = va[r] ? ulab[perm[i]] : 0;
    const int lc = vb[r] ? ulab[perm[i + 1]] : 0;
    ok[2 * r] = va[r] && la >= 0 && la < kb;
    ok[2 * r + 1] = vb[r] && lc >= 0 && lc < kb;
    bad |= (va[r] && !ok[2 * r]) || (vb[r] && !ok[2 * r + 1]);
    lab[2 * r] = c0 + (ok[2 * r] ? la : 0);
    lab[2 * r + 1] = c0 + (ok[2 * r + 1] ? lc : 0);
  }
  unsigned qx[kPts], qy[kPts], qz[kPts];
  const int s_t = residuals_global<D>(A, x, y, z, lab, ok, qx, qy, qz);
  tile_sums<D>(A, qx, qy, qz, lab, ok, s_t, false, false, nullptr, A.crun[b].s_glob);
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
  const bool fold = mode == 1 && t >= 0 && (A.want_stats || A.early_stop);   // one more CTA
  k_centroids<<<ceil_div(A.k, kBlockThreads) + (fold ? 1 : 0), kBlockThreads, 0, s>>>(
      A, mode, t, d, user_c, insert, par, counts_out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// k_seed_refs: a starting reference for every search unit that has none (a
// fresh context, or tiles re-cut since the last run): the centroid nearest
// to the centre of the unit's box among the centroids of the grid cell
// holding that centre or, if it is empty, of the first non-empty shell of
// cells around it (up to kSeedRings shells).  The reference only sets the
// search's starting bound U = maxd(box, reference), which any centroid of
// the cloud bounds validly, so the search's result does not depend on it;
// without it the first search scans rings of cells with a looser bound and
// keeps longer lists.  Units that already have a reference return at once.
// One thread per unit; grid of parity `par`.
// ---------------------------------------------------------------------------
constexpr int kSeedRings = 3;

__global__ void __launch_bounds__(kBlockThreads) k_seed_refs(const __grid_constant__ IterArgs A,
                                                             int par, int d) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= A.n_units) return;
  const int b = A.B > 1 ? A.ucloud[t] : 0;
  const Cloud& cl = A.B > 1 ? A.clouds[b] : A.cl0;
  const int ref = A.tref[t];
  if (ref >= cl.c0 && ref < cl.c0 + cl.k) return;
  if (A.B > 1 && A.crun[b].done) return;
  const Grid G = cl.grid;
  const float4 lo = A.ubox[2 * t], hi = A.ubox[2 * t + 1];
  const float px = 0.5f * (lo.x + hi.x), py = 0.5f * (lo.y + hi.y),
              pz = d == 3 ? 0.5f * (lo.z + hi.z) : 0.f;
  const int cx = cell_coord(px, G.g0[0], G.inv_s, G.dims[0]);
  const int cy = cell_coord(py, G.g0[1], G.inv_s, G.dims[1]);
  const int cz = d == 3 ? cell_coord(pz, G.g0[2], G.inv_s, G.dims[2]) : 0;
  const int* __restrict__ gcnt = A.gcnt[par] + cl.cell0;
  const float4* __restrict__ gbkt = A.gbkt[par] + cl.cell0 * kBucketCap;
  float best = INFINITY;
  int best_id = -1;
  for (int r = 0; r <= kSeedRings && best_id < 0; ++r) {
    const int zr = d == 3 ? r : 0;
    for (int z = cz - zr; z <= cz + zr; ++z) {
      if (z < 0 || z >= G.dims[2]) continue;
      for (int y = cy - r; y <= cy + r; ++y) {
        if (y < 0 || y >= G.dims[1]) continue;
        for (int x = cx - r; x <= cx + r; ++x) {
          if (x < 0 || x >= G.dims[0]) continue;
          // the shell of Chebyshev radius r only
          if (max(max(abs(x - cx), abs(y - cy)), abs(z - cz)) != r) continue;
          const long long cell = ((long long)z * G.dims[1] + y) * G.dims[0] + x;
          const int cnt = min(gcnt[cell], kBucketCap);
          for (int i = 0; i < cnt; ++i) {
            const float4 c = gbkt[cell * kBucketCap + i];
            const float dx = c.x - px, dy = c.y - py, dz = c.z - pz;
            const float dd = dx * dx + dy * dy + (d == 3 ? dz * dz : 0.f);
            if (dd < best) {
              best = dd;
              best_id = __float_as_int(c.w);
            }
          }
        }
      }
    }
  }
  if (best_id >= 0) A.tref[t] = best_id;   // else the search scans rings itself
}

cudaError_t launch_seed_refs(const IterArgs& A, int par, int d, cudaStream_t s) {
  k_seed_refs<<<ceil_div(A.n_units, kBlockThreads), kBlockThreads, 0, s>>>(A, par, d);
  return cudaGetLastError();
}

cudaError_t launch_search(const IterArgs& A, int par, int d, cudaStream_t s) {
  const int g = ceil_div(A.n_units, kSearchWarps);
  if (d == 3) {
    if (A.B > 1) k_search<true, 3><<<g, 32 * kSearchWarps, 0, s>>>(A, par);
    else k_search<false, 3><<<g, 32 * kSearchWarps, 0, s>>>(A, par);
  } else {
    if (A.B > 1) k_search<true, 2><<<g, 32 * kSearchWarps, 0, s>>>(A, par);
    else k_search<false, 2><<<g, 32 * kSearchWarps, 0, s>>>(A, par);
  }
  return cudaGetLastError();
}

template <int D, bool BRUTE>
void assign_multi(const IterArgs& A, int g, cudaStream_t s) {
  constexpr int thr = 32 * kAssignWarps;
  if (!BRUTE && A.unit_g > 1) {
    if (A.B > 1) k_assign<D, false, true, true, false><<<g, thr, 0, s>>>(A);
    else k_assign<D, false, false, true, false><<<g, thr, 0, s>>>(A);
    return;
  }
  if (!BRUTE && A.stay == 2) {
    if (A.B > 1) k_assign<D, false, true, false, true><<<g, thr, 0, s>>>(A);
    else k_assign<D, false, false, false, true><<<g, thr, 0, s>>>(A);
    return;
  }
  if (A.B > 1) k_assign<D, BRUTE, true, false, false><<<g, thr, 0, s>>>(A);
  else k_assign<D, BRUTE, false, false, false><<<g, thr, 0, s>>>(A);
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
//
// use_ub (after an update inside a run): the search starts from the upper
// bound of Eq. ub, ub = cb[j] + Delta[j] + max(Delta) -- c_j's previous
// nearest neighbour is still a centroid, now at most that far -- and
// skips every cell whose box lies farther than ub from c_j, as the kNN
// prunes centroid nodes beyond its bound.  max(Delta) is read as the
// cloud's largest drift (a safe bound).  If nothing lies within ub after
// rounding, the search runs again without it.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlockThreads) k_cbound(IterArgs A, int par, int d, int use_ub) {
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
  float ub = INFINITY;
  if (use_ub && A.cb2[j] < INFINITY) {
    const float cbp = sqrtf(A.cb2[j] * (256.0f / 255.0f));
    const float dm = __uint_as_float(A.crun[b].dmax[(par ^ 1) & 1]);
    ub = (cbp + A.drift[j] + dm) * 1.0001f;
  }
  // lower bound on the distance from c_j to any point of the cell at
  // offsets (x, y, z) from its own cell, per axis (the faces toward c_j)
  const float cpos[3] = {c.x, c.y, c.z};
  auto cell_lb2 = [&](int x, int y, int z) {
    const int o[3] = {x, y, z};
    float s2 = 0.f;
    for (int a = 0; a < 3; ++a) {
      if (a == 2 && d != 3) break;
      float g = 0.f;
      if (o[a] < cc[a]) g = cpos[a] - (G.g0[a] + (float)(o[a] + 1) * edge);
      else if (o[a] > cc[a]) g = (G.g0[a] + (float)o[a] * edge) - cpos[a];
      g = fmaxf(g - margin * edge, 0.f);
      s2 += g * g;
    }
    return s2;
  };
  for (int attempt = 0; attempt < 2; ++attempt) {
    const float ub2 = ub * ub;
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
            if (ub < INFINITY && cell_lb2(x, y, z) > ub2) continue;   // beyond the bound
            const long long cell = ((long long)z * G.dims[1] + y) * G.dims[0] + x;
            const int cnt = min(gcnt[cell], kBucketCap);
            for (int i = 0; i < cnt; ++i) take(gbkt[cell * kBucketCap + i]);
          }
      if (whole) break;
      const float lb = fmaxf((float)r - margin, 0.f) * edge;
      if (best <= lb * lb * (1.0f - 1.0f / 256.0f)) break;
      if (lb > ub) break;   // every centroid beyond lies farther than the bound
    }
    if (best < INFINITY || !(ub < INFINITY)) break;
    ub = INFINITY;   // nothing within the bound after rounding: search unbounded
  }
  A.cb2[j] = best * (1.0f - 1.0f / 256.0f);
}

cudaError_t launch_cbound(const IterArgs& A, int par, int d, int use_ub, cudaStream_t s) {
  k_cbound<<<ceil_div(A.k, kBlockThreads), kBlockThreads, 0, s>>>(A, par, d, use_ub);
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
