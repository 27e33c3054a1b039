// dkm_soft.cu -- differentiable k-means losses of a batch of point clouds
// (sm_103a).
//
// The paper optimises the k-means objective of Eq. 1 with Lloyd's
// algorithm.  The differentiable extension exposes two losses and their
// gradients with respect to the points and the initial centroids:
//
//   hard SSE   L_h = sum_i min_j ||p_i - c_j||^2; dL/dp_i = 2 (p_i - c_a(i)),
//              dL/dc_j = -2 sum_{a(i)=j} (p_i - c_j)
//   soft       T unrolled soft k-means steps at a fixed temperature tau:
//              w^t_ij = softmax_j(-||p_i - c^t_j||^2 / tau),
//              c^{t+1}_j = sum_i w^t_ij p_i / sum_i w^t_ij,
//              L_s = sum_ij w^T_ij ||p_i - c^T_j||^2.
//
// Every (point, centroid) quantity is recomputed, never stored: row passes
// (two points per thread, reducing over the cloud's centroids in shared
// memory) and column passes (two centroids per thread, reducing over a
// split of the cloud's points staged in shared memory), both in packed
// f32x2 arithmetic, whose lanes round as the scalar operations do.  The backward recomputes
// the weights of step t from the checkpointed centroids c^t.  Column sums
// run in FP32 over chunks of 64 points and in FP64 across chunks; splits
// are combined in a fixed order, so results are deterministic.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "dkm_host.h"

namespace dkm {
namespace {

constexpr int kRowThreads = 256;
constexpr int kSplit = 512;        // points per column-pass CTA (several CTAs per SM for latency hiding)
constexpr int kColChunk = 256;     // points staged in shared memory per round
constexpr int kSubChunk = 64;      // FP32 accumulation run before the FP64 add

struct SoftArgs {
  const float* P;         // n_total x D, row-major
  const int64_t* off;     // B + 1 cloud offsets
  int B, k, ns;           // clouds, centroids per cloud, splits per cloud
  const float* tau;       // B
  float* m;               // per point: min_j D_ij
  float* iz;              // per point: 1 / sum_j exp((m - D_ij) / tau)
  float* aux;             // per point: rho_i (soft step) or E_i (loss stage)
  double* part;           // B x ns x k x 4 column partials
  int use_stats;          // kRowStep: m and iz given (from the forward), not recomputed
  int* bad;               // set when a given label lies outside [0, k)
};

enum RowMode {
  kRowStats = 0, kRowLoss = 1, kRowStep = 2, kRowLossBwd = 3, kRowHard = 4, kRowHardBwd = 5
};
enum ColMode { kColMean = 0, kColStep = 1, kColLoss = 2, kColHard = 3 };

template <int D>
__device__ __forceinline__ float3 load_pt(const float* P, int64_t i) {
  return make_float3(P[i * D + 0], P[i * D + 1], D == 3 ? P[i * D + 2] : 0.f);
}

template <int D>
__device__ __forceinline__ float sqd(float3 p, float4 c, float3& diff) {
  diff.x = __fadd_rn(p.x, -c.x);
  diff.y = __fadd_rn(p.y, -c.y);
  diff.z = D == 3 ? __fadd_rn(p.z, -c.z) : 0.f;
  float s = __fmaf_rn(diff.y, diff.y, __fmul_rn(diff.x, diff.x));
  if (D == 3) s = __fmaf_rn(diff.z, diff.z, s);
  return s;
}

template <int D>
__device__ __forceinline__ float4 load_c(const float* C, int64_t j, float w) {
  return make_float4(C[j * D + 0], C[j * D + 1], D == 3 ? C[j * D + 2] : 0.f, w);
}

__device__ __forceinline__ float2 dup2(float x) { return make_float2(x, x); }

// sqd for two points at once (packed f32x2: each lane rounds as the scalar
// form does)
template <int D>
__device__ __forceinline__ float2 sqd2(float2 px, float2 py, float2 pz, float4 c, float2& dx,
                                       float2& dy, float2& dz) {
  dx = __fadd2_rn(px, dup2(-c.x));
  dy = __fadd2_rn(py, dup2(-c.y));
  dz = D == 3 ? __fadd2_rn(pz, dup2(-c.z)) : make_float2(0.f, 0.f);
  float2 s = __fmul2_rn(dx, dx);
  s = __ffma2_rn(dy, dy, s);
  if (D == 3) s = __ffma2_rn(dz, dz, s);
  return s;
}

// softmax weights exp((m - s) / tau) / Z of two points
__device__ __forceinline__ float2 weight2(float2 m, float2 s, float it, float2 iz) {
  const float2 a = __fmul2_rn(__fadd2_rn(m, make_float2(-s.x, -s.y)), dup2(it));
  return __fmul2_rn(make_float2(__expf(a.x), __expf(a.y)), iz);
}

// one point's step of the online normaliser: z = sum_j exp((m - D_ij) / tau)
// against the running minimum m, rescaled by exp((m_new - m_old) / tau)
// whenever the minimum drops.  The exponent is -|s - m| / tau either way.
__device__ __forceinline__ void online_norm(float s, float& m, float& z, float it) {
  const float e = __expf(-fabsf(__fadd_rn(s, -m)) * it);
  const bool lower = s < m;
  z = lower ? __fmaf_rn(z, e, 1.f) : __fadd_rn(z, e);
  m = lower ? s : m;
}

// Row pass: each thread takes two points of its cloud, i and i + kRowThreads
// of the CTA's 2 kRowThreads, evaluated together in packed f32x2 arithmetic
// (each centroid read from shared memory once for both).  Shared memory:
// c^t (k), and for kRowStep c^{t+1} with .w = 1/N (k) and the upstream
// gradient of c^{t+1} (k).
constexpr int kRowPoints = 2 * kRowThreads;   // points per row-pass CTA

template <int D, int MODE>
__global__ void __launch_bounds__(kRowThreads) k_soft_row(SoftArgs A, const float* __restrict__ Ct,
                                                          const float* __restrict__ Cn,
                                                          const float* __restrict__ Nn,
                                                          const float* __restrict__ Gn,
                                                          const double* __restrict__ dloss,
                                                          float* __restrict__ gP,
                                                          int32_t* __restrict__ labels,
                                                          double* __restrict__ loss_part) {
  extern __shared__ float4 sm[];
  __shared__ double s_red[kRowThreads / 32];
  const int b = blockIdx.y, k = A.k;
  const int64_t o0 = A.off[b], o1 = A.off[b + 1];
  float4* sc = sm;
  float4* scn = sm + k;
  float4* sg = sm + 2 * k;
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const int64_t g = (int64_t)b * k + j;
    sc[j] = load_c<D>(Ct, g, 0.f);
    if (MODE == kRowStep) {
      const float n = Nn[g];
      scn[j] = load_c<D>(Cn, g, n > 0.f ? 1.f / n : 0.f);
      sg[j] = load_c<D>(Gn, g, 0.f);
    }
  }
  __syncthreads();
  const int64_t i0 = o0 + (int64_t)blockIdx.x * kRowPoints + threadIdx.x;
  const int64_t ii[2] = {i0, i0 + kRowThreads};
  const bool vv[2] = {ii[0] < o1, ii[1] < o1};
  const float3 pa = vv[0] ? load_pt<D>(A.P, ii[0]) : make_float3(0.f, 0.f, 0.f);
  const float3 pb = vv[1] ? load_pt<D>(A.P, ii[1]) : make_float3(0.f, 0.f, 0.f);
  const float it = 1.f / A.tau[b];
  double contrib = 0.0;
  if (MODE == kRowHardBwd || MODE == kRowHard) {
    // kRowHard: both points' nearest centroids first, in packed arithmetic;
    // centroids come in ascending index order, so a strictly smaller
    // distance is the only way to win and ties keep the lowest index
    float2 hard_best = dup2(INFINITY);
    int2 hard_a = make_int2(0, 0);
    if (MODE == kRowHard) {
      const float2 px = make_float2(pa.x, pb.x), py = make_float2(pa.y, pb.y),
                   pz = make_float2(pa.z, pb.z);
      float2 dx, dy, dz;
      for (int j = 0; j < k; ++j) {
        const float2 s = sqd2<D>(px, py, pz, sc[j], dx, dy, dz);
        if (s.x < hard_best.x) {
          hard_best.x = s.x;
          hard_a.x = j;
        }
        if (s.y < hard_best.y) {
          hard_best.y = s.y;
          hard_a.y = j;
        }
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t i = ii[h];
      const bool valid = vv[h];
      const float3 p = h ? pb : pa;
      float3 dv;
      if (MODE == kRowHardBwd) {
        // dOut/dp_i = dloss[b] * 2 (p_i - c_a(i)), a(i) the forward's label
        if (valid) {
          const int a = labels[i];
          if (a < 0 || a >= k) {
            atomicOr(A.bad, 1);
            gP[i * D + 0] = gP[i * D + 1] = 0.f;
            if (D == 3) gP[i * D + 2] = 0.f;
          } else {
            sqd<D>(p, sc[a], dv);
            const float s2 = 2.f * (float)dloss[b];
            gP[i * D + 0] = s2 * dv.x;
            gP[i * D + 1] = s2 * dv.y;
            if (D == 3) gP[i * D + 2] = s2 * dv.z;
          }
        }
      } else {
        if (valid) {
          const int a = h ? hard_a.y : hard_a.x;
          labels[i] = a;
          contrib += h ? hard_best.y : hard_best.x;
          if (gP) {
            sqd<D>(p, sc[a], dv);
            gP[i * D + 0] = 2.f * dv.x;
            gP[i * D + 1] = 2.f * dv.y;
            if (D == 3) gP[i * D + 2] = 2.f * dv.z;
          }
        }
      }
    }
  } else {
    const float2 px = make_float2(pa.x, pb.x), py = make_float2(pa.y, pb.y),
                 pz = make_float2(pa.z, pb.z);
    float2 dx, dy, dz;
    const bool given = MODE == kRowStep && A.use_stats;
    float2 m = dup2(INFINITY), iz = dup2(0.f);
    if (given) {   // the forward's statistics of this step (same values, bit for bit)
      if (vv[0]) {
        m.x = A.m[ii[0]];
        iz.x = A.iz[ii[0]];
      }
      if (vv[1]) {
        m.y = A.m[ii[1]];
        iz.y = A.iz[ii[1]];
      }
    } else {
      // one sweep (online softmax normaliser, Milakov & Gimelshein 2018)
      float2 z = dup2(0.f);
      for (int j = 0; j < k; ++j) {
        const float2 s = sqd2<D>(px, py, pz, sc[j], dx, dy, dz);
        online_norm(s.x, m.x, z.x, it);
        online_norm(s.y, m.y, z.y, it);
      }
      iz = make_float2(1.f / z.x, 1.f / z.y);
    }
    if (MODE == kRowLoss || MODE == kRowLossBwd) {
      // E = sum_j w D;  B = sum_j w (p - c);  F = sum_j w D (p - c)
      float2 E = dup2(0.f);
      float2 Bx = E, By = E, Bz = E, Fx = E, Fy = E, Fz = E;
      for (int j = 0; j < k; ++j) {
        const float2 s = sqd2<D>(px, py, pz, sc[j], dx, dy, dz);
        const float2 w = weight2(m, s, it, iz);
        E = __ffma2_rn(w, s, E);
        if (MODE == kRowLossBwd) {
          Bx = __ffma2_rn(w, dx, Bx);
          By = __ffma2_rn(w, dy, By);
          Bz = __ffma2_rn(w, dz, Bz);
          const float2 ws = __fmul2_rn(w, s);
          Fx = __ffma2_rn(ws, dx, Fx);
          Fy = __ffma2_rn(ws, dy, Fy);
          Fz = __ffma2_rn(ws, dz, Fz);
        }
      }
      const float sc2 = MODE == kRowLossBwd ? 2.f * (float)dloss[b] : 0.f;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (!vv[h]) continue;
        const int64_t i = ii[h];
        const float e = h ? E.y : E.x;
        contrib += e;
        if (MODE == kRowLossBwd) {
          // dL/dp_i = 2 sum_l w_il (1 - (D_il - E_i)/tau) (p_i - c_l)
          const float bx = h ? Bx.y : Bx.x, by = h ? By.y : By.x, bz = h ? Bz.y : Bz.x;
          const float fx = h ? Fx.y : Fx.x, fy = h ? Fy.y : Fy.x, fz = h ? Fz.y : Fz.x;
          gP[i * D + 0] = sc2 * (bx - it * (fx - e * bx));
          gP[i * D + 1] = sc2 * (by - it * (fy - e * by));
          if (D == 3) gP[i * D + 2] = sc2 * (bz - it * (fz - e * bz));
          A.aux[i] = e;
        }
      }
    } else if (MODE == kRowStep) {
      // rho = sum_j w g;  Av = sum_j w g (p - c^t);  Bv = sum_j w (p - c^t);
      // Dir = sum_j w gbar_j / N_j,  g_ij = gbar_j . (p_i - c^{t+1}_j) / N_j
      float2 rho = dup2(0.f);
      float2 Ax = rho, Ay = rho, Az = rho, Bx = rho, By = rho, Bz = rho, Dx = rho, Dy = rho,
             Dz = rho;
      for (int j = 0; j < k; ++j) {
        const float2 s = sqd2<D>(px, py, pz, sc[j], dx, dy, dz);
        const float2 w = weight2(m, s, it, iz);
        const float4 cn = scn[j], gb = sg[j];
        float2 nx, ny, nz;
        sqd2<D>(px, py, pz, cn, nx, ny, nz);
        float2 g = __fmul2_rn(dup2(gb.x), nx);
        g = __ffma2_rn(dup2(gb.y), ny, g);
        if (D == 3) g = __ffma2_rn(dup2(gb.z), nz, g);
        g = __fmul2_rn(g, dup2(cn.w));
        const float2 wg = __fmul2_rn(w, g);
        rho = __fadd2_rn(rho, wg);
        Ax = __ffma2_rn(wg, dx, Ax);
        Ay = __ffma2_rn(wg, dy, Ay);
        Az = __ffma2_rn(wg, dz, Az);
        Bx = __ffma2_rn(w, dx, Bx);
        By = __ffma2_rn(w, dy, By);
        Bz = __ffma2_rn(w, dz, Bz);
        const float2 wn = __fmul2_rn(w, dup2(cn.w));
        Dx = __ffma2_rn(wn, dup2(gb.x), Dx);
        Dy = __ffma2_rn(wn, dup2(gb.y), Dy);
        Dz = __ffma2_rn(wn, dup2(gb.z), Dz);
      }
      // dL/dp_i += Dir + sum_j dD_ij 2 (p_i - c_j),  dD_ij = -(1/tau) w (g - rho)
      const float two_it = 2.f * it;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (!vv[h]) continue;
        const int64_t i = ii[h];
        const float r = h ? rho.y : rho.x;
        gP[i * D + 0] += (h ? Dx.y : Dx.x) - two_it * ((h ? Ax.y : Ax.x) - r * (h ? Bx.y : Bx.x));
        gP[i * D + 1] += (h ? Dy.y : Dy.x) - two_it * ((h ? Ay.y : Ay.x) - r * (h ? By.y : By.x));
        if (D == 3)
          gP[i * D + 2] += (h ? Dz.y : Dz.x) - two_it * ((h ? Az.y : Az.x) - r * (h ? Bz.y : Bz.x));
        A.aux[i] = r;
      }
    }
    if (!given) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (!vv[h]) continue;
        A.m[ii[h]] = h ? m.y : m.x;
        A.iz[ii[h]] = h ? iz.y : iz.x;
      }
    }
  }
  if (MODE == kRowLoss || MODE == kRowHard) {
    // deterministic per-CTA partial of the loss
    double v = contrib;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < kRowThreads / 32; ++w) t += s_red[w];
      loss_part[(int64_t)b * gridDim.x + blockIdx.x] = t;
    }
  }
}

// Column pass: each thread takes two centroids of cloud blockIdx.y, j and
// j + blockDim.x, over the points of split blockIdx.x, evaluated together in
// packed f32x2 arithmetic (each staged point read once for both).  Writes
// part[b][s][j][0..3].
template <int D, int MODE>
__global__ void k_soft_col(SoftArgs A, const float* __restrict__ Ct, const float* __restrict__ Cn,
                           const float* __restrict__ Nn, const float* __restrict__ Gn,
                           const double* __restrict__ dloss, const int32_t* __restrict__ labels) {
  __shared__ float4 s_p[kColChunk];   // x, y, z, m
  __shared__ float4 s_q[kColChunk];   // iz, aux, label bits, -
  const int b = blockIdx.y, s = blockIdx.x, k = A.k;
  const int jj[2] = {(int)threadIdx.x, (int)(threadIdx.x + blockDim.x)};
  const int64_t o0 = A.off[b], o1 = A.off[b + 1];
  const int64_t lo = o0 + (int64_t)s * kSplit, hi = min(lo + kSplit, o1);
  const bool live[2] = {jj[0] < k, jj[1] < k};
  float4 c[2], cn[2], gb[2];
  float in[2] = {0.f, 0.f};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int64_t g = (int64_t)b * k + (live[h] ? jj[h] : 0);
    c[h] = load_c<D>(Ct, g, 0.f);
    cn[h] = c[h];
    gb[h] = c[h];
    if (MODE == kColStep) {
      cn[h] = load_c<D>(Cn, g, 0.f);
      gb[h] = load_c<D>(Gn, g, 0.f);
      const float n = Nn[g];
      in[h] = n > 0.f ? 1.f / n : 0.f;
    }
  }
  const float2 ncx = make_float2(-c[0].x, -c[1].x), ncy = make_float2(-c[0].y, -c[1].y),
               ncz = make_float2(-c[0].z, -c[1].z);
  const float2 nnx = make_float2(-cn[0].x, -cn[1].x), nny = make_float2(-cn[0].y, -cn[1].y),
               nnz = make_float2(-cn[0].z, -cn[1].z);
  const float2 gbx = make_float2(gb[0].x, gb[1].x), gby = make_float2(gb[0].y, gb[1].y),
               gbz = make_float2(gb[0].z, gb[1].z), in2 = make_float2(in[0], in[1]);
  const float it = 1.f / A.tau[b];
  const float scl = MODE == kColLoss ? (float)dloss[b] : 1.f;
  double acc[2][4] = {{0.0, 0.0, 0.0, 0.0}, {0.0, 0.0, 0.0, 0.0}};
  for (int64_t c0 = lo; c0 < hi; c0 += kColChunk) {
    const int m = (int)min((int64_t)kColChunk, hi - c0);
    __syncthreads();
    for (int q = threadIdx.x; q < m; q += blockDim.x) {
      const float3 p = load_pt<D>(A.P, c0 + q);
      if (MODE == kColHard) {
        s_p[q] = make_float4(p.x, p.y, p.z, 0.f);
        s_q[q] = make_float4(0.f, 0.f, __int_as_float(labels[c0 + q]), 0.f);
      } else {
        s_p[q] = make_float4(p.x, p.y, p.z, A.m[c0 + q]);
        s_q[q] = make_float4(A.iz[c0 + q], MODE == kColMean ? 0.f : A.aux[c0 + q], 0.f, 0.f);
      }
    }
    __syncthreads();
    if (!live[0]) continue;   // (then j + blockDim.x is out of range too)
    for (int q0 = 0; q0 < m; q0 += kSubChunk) {
      float2 f0 = dup2(0.f), f1 = f0, f2 = f0, f3 = f0;   // .x: centroid j, .y: j + blockDim
      const int qe = min(q0 + kSubChunk, m);
      for (int q = q0; q < qe; ++q) {
        const float4 pq = s_p[q], aq = s_q[q];
        if (MODE == kColHard) {
          const int lq = __float_as_int(aq.z);
          if (threadIdx.x == 0 && (lq < 0 || lq >= k)) atomicOr(A.bad, 1);
          if (lq == jj[0] || lq == jj[1]) {
            const int h = lq == jj[1];
            float3 dv;
            sqd<D>(make_float3(pq.x, pq.y, pq.z), c[h], dv);
            if (h) {
              f0.y += dv.x; f1.y += dv.y; f2.y += dv.z;
            } else {
              f0.x += dv.x; f1.x += dv.y; f2.x += dv.z;
            }
          }
          continue;
        }
        const float2 dx = __fadd2_rn(dup2(pq.x), ncx), dy = __fadd2_rn(dup2(pq.y), ncy);
        const float2 dz = D == 3 ? __fadd2_rn(dup2(pq.z), ncz) : dup2(0.f);
        float2 sd = __fmul2_rn(dx, dx);
        sd = __ffma2_rn(dy, dy, sd);
        if (D == 3) sd = __ffma2_rn(dz, dz, sd);
        const float2 a = __fmul2_rn(__fadd2_rn(dup2(pq.w), make_float2(-sd.x, -sd.y)), dup2(it));
        const float2 w = __fmul2_rn(make_float2(__expf(a.x), __expf(a.y)), dup2(aq.x));
        if (MODE == kColMean) {
          f0 = __ffma2_rn(w, dup2(pq.x), f0);
          f1 = __ffma2_rn(w, dup2(pq.y), f1);
          f2 = __ffma2_rn(w, dup2(pq.z), f2);
          f3 = __fadd2_rn(f3, w);
        } else if (MODE == kColStep) {
          const float2 ex = __fadd2_rn(dup2(pq.x), nnx), ey = __fadd2_rn(dup2(pq.y), nny);
          const float2 ez = D == 3 ? __fadd2_rn(dup2(pq.z), nnz) : dup2(0.f);
          float2 gg = __fmul2_rn(gbx, ex);
          gg = __ffma2_rn(gby, ey, gg);
          if (D == 3) gg = __ffma2_rn(gbz, ez, gg);
          // dL/dD_ij = -(1/tau) w (g_ij - rho_i)
          const float2 dd = __fmul2_rn(__fmul2_rn(dup2(-it), w),
                                       __ffma2_rn(gg, in2, dup2(-aq.y)));
          f0 = __ffma2_rn(dd, dx, f0);
          f1 = __ffma2_rn(dd, dy, f1);
          f2 = __ffma2_rn(dd, dz, f2);
        } else {   // kColLoss: dL/dD_ij = w (1 - (D_ij - E_i) / tau)
          const float2 u = __ffma2_rn(__fadd2_rn(sd, dup2(-aq.y)), dup2(-it), dup2(1.f));
          const float2 dd = __fmul2_rn(__fmul2_rn(dup2(scl), w), u);
          f0 = __ffma2_rn(dd, dx, f0);
          f1 = __ffma2_rn(dd, dy, f1);
          f2 = __ffma2_rn(dd, dz, f2);
        }
      }
      acc[0][0] += (double)f0.x; acc[0][1] += (double)f1.x;
      acc[0][2] += (double)f2.x; acc[0][3] += (double)f3.x;
      acc[1][0] += (double)f0.y; acc[1][1] += (double)f1.y;
      acc[1][2] += (double)f2.y; acc[1][3] += (double)f3.y;
    }
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if (!live[h]) continue;
    double* out = A.part + (((int64_t)b * A.ns + s) * k + jj[h]) * 4;
    out[0] = acc[h][0];
    out[1] = acc[h][1];
    out[2] = acc[h][2];
    out[3] = acc[h][3];
  }
}

// Combine the splits in order.  mean: c_next = S / N (or c if N == 0),
// N_out = N.  grad: G_out = -2 * sum (the dL/dc of the pass), times
// scale[b] if given; with Nn and Gin (an update step of the backward), a
// centroid whose weights all underflowed (Nn = 0) kept its position in the
// forward (c^{t+1} = c^t), so the upstream gradient Gin of c^{t+1} also
// flows on to c^t unchanged.
__global__ void k_soft_reduce(SoftArgs A, int D, int mode, const float* __restrict__ Ct,
                              float* __restrict__ Cnext, float* __restrict__ Nout,
                              float* __restrict__ Gout, const float* __restrict__ Nn,
                              const float* __restrict__ Gin, const double* __restrict__ scale) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)A.B * A.k) return;
  const int b = (int)(idx / A.k), j = (int)(idx % A.k);
  double t[4] = {0.0, 0.0, 0.0, 0.0};
  for (int s = 0; s < A.ns; ++s) {
    const double* in = A.part + (((int64_t)b * A.ns + s) * A.k + j) * 4;
    for (int a = 0; a < 4; ++a) t[a] += in[a];
  }
  if (mode == 0) {
    if (Nout) Nout[idx] = (float)t[3];
    if (Cnext)
      for (int a = 0; a < D; ++a)
        Cnext[idx * D + a] = t[3] > 0.0 ? (float)(t[a] / t[3]) : Ct[idx * D + a];
  } else {
    const double f = scale ? -2.0 * scale[b] : -2.0;
    const bool through = Nn && Gin && !(Nn[idx] > 0.f);
    for (int a = 0; a < D; ++a)
      Gout[idx * D + a] = (float)(f * t[a]) + (through ? Gin[idx * D + a] : 0.f);
  }
}

__global__ void k_soft_loss(const double* __restrict__ part, int gx, int B, double* __restrict__ loss) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double t = 0.0;
  for (int q = 0; q < gx; ++q) t += part[(int64_t)b * gx + q];
  loss[b] = t;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct SoftPlan {
  std::vector<int64_t> off;
  int64_t n_total = 0, max_n = 0;
  int gx = 0, ns = 0;
};

dkm_status soft_fail(dkm_status s, const char* msg, cudaError_t e = cudaSuccess) {
  std::string m = msg;
  if (e != cudaSuccess) {
    m += ": ";
    m += cudaGetErrorString(e);
  }
  dkm_set_last_error(m.c_str());
  return s;
}

#define SOFT_CK(call)                                                         \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      cudaGetLastError();                                                     \
      return soft_fail(DKM_ECUDA, #call, e_);                                 \
    }                                                                         \
  } while (0)

dkm_status soft_plan(const int64_t* offsets, int B, int d, int k, SoftPlan* P) {
  if (B < 1) return soft_fail(DKM_EINVAL, "B must be >= 1");
  if (d != 2 && d != 3) return soft_fail(DKM_EINVAL, "d must be 2 or 3");
  if (k < 1 || k > 1024) return soft_fail(DKM_EINVAL, "k must be in [1, 1024]");
  if (!offsets) return soft_fail(DKM_EINVAL, "null offsets");
  P->off.resize((size_t)B + 1);
  cudaError_t e = cudaMemcpy(P->off.data(), offsets, sizeof(int64_t) * (B + 1), cudaMemcpyDefault);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return soft_fail(DKM_EINVAL, "offsets not readable", e);
  }
  if (P->off[0] != 0) return soft_fail(DKM_EINVAL, "offsets[0] must be 0");
  for (int b = 0; b < B; ++b) {
    const int64_t nb = P->off[b + 1] - P->off[b];
    if (nb < 1) return soft_fail(DKM_EINVAL, "every cloud needs at least one point");
    P->max_n = std::max(P->max_n, nb);
  }
  P->n_total = P->off[B];
  P->gx = (int)((P->max_n + kRowPoints - 1) / kRowPoints);
  P->ns = (int)((P->max_n + kSplit - 1) / kSplit);
  return DKM_OK;
}

// scratch laid out in one stream-ordered allocation
struct SoftScratch {
  void* base = nullptr;
  cudaStream_t stream = nullptr;
  // released (stream-ordered) on every exit path of the call that made it
  ~SoftScratch() {
    if (base) cudaFreeAsync(base, stream);
  }
  SoftScratch() = default;
  SoftScratch(const SoftScratch&) = delete;
  SoftScratch& operator=(const SoftScratch&) = delete;
  SoftArgs A{};
  double* loss_part = nullptr;
  double* loss_dev = nullptr;
  float* N = nullptr;
  float* G[2] = {nullptr, nullptr};
  int32_t* labels = nullptr;
};

dkm_status soft_alloc(const SoftPlan& P, int B, int d, int k, const float* tau, cudaStream_t st,
                      SoftScratch* S) {
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t n = (size_t)P.n_total;
  size_t o_off = 0, o_tau = o_off + al(sizeof(int64_t) * (B + 1)), o_m = o_tau + al(sizeof(float) * B),
         o_iz = o_m + al(4 * n), o_aux = o_iz + al(4 * n), o_part = o_aux + al(4 * n),
         o_lp = o_part + al(sizeof(double) * 4 * (size_t)B * P.ns * k),
         o_ld = o_lp + al(sizeof(double) * (size_t)B * P.gx), o_N = o_ld + al(sizeof(double) * B),
         o_G0 = o_N + al(4 * (size_t)B * k), o_G1 = o_G0 + al(4 * (size_t)B * k * d),
         o_lab = o_G1 + al(4 * (size_t)B * k * d), o_bad = o_lab + al(4 * n),
         total = o_bad + al(sizeof(int));
  SOFT_CK(cudaMallocAsync(&S->base, total, st));
  S->stream = st;
  char* c = (char*)S->base;
  SoftArgs& A = S->A;
  A.off = (const int64_t*)(c + o_off);
  A.tau = (const float*)(c + o_tau);
  A.m = (float*)(c + o_m);
  A.iz = (float*)(c + o_iz);
  A.aux = (float*)(c + o_aux);
  A.part = (double*)(c + o_part);
  A.B = B;
  A.k = k;
  A.ns = P.ns;
  S->loss_part = (double*)(c + o_lp);
  S->loss_dev = (double*)(c + o_ld);
  S->N = (float*)(c + o_N);
  S->G[0] = (float*)(c + o_G0);
  S->G[1] = (float*)(c + o_G1);
  S->labels = (int32_t*)(c + o_lab);
  A.bad = (int*)(c + o_bad);
  SOFT_CK(cudaMemsetAsync(A.bad, 0, sizeof(int), st));
  SOFT_CK(cudaMemcpyAsync((void*)A.off, P.off.data(), sizeof(int64_t) * (B + 1),
                          cudaMemcpyHostToDevice, st));
  SOFT_CK(cudaMemcpyAsync((void*)A.tau, tau, sizeof(float) * B, cudaMemcpyDefault, st));
  return DKM_OK;
}

// Launchers.  A is the scratch's argument block, possibly with the row
// statistics of one step pointed at the caller's arrays (step_args).
template <int D, int MODE>
void launch_row(const SoftArgs& A, const SoftScratch& S, const SoftPlan& P, const float* Ct,
                const float* Cn, const float* Nn, const float* Gn, const double* dloss, float* gP,
                int32_t* lab, cudaStream_t st) {
  const size_t smem = sizeof(float4) * (size_t)A.k * (MODE == kRowStep ? 3 : 1);
  k_soft_row<D, MODE><<<dim3(P.gx, A.B), kRowThreads, smem, st>>>(A, Ct, Cn, Nn, Gn, dloss, gP,
                                                                 lab, S.loss_part);
}

template <int D, int MODE>
void launch_col(const SoftArgs& A, const SoftPlan& P, const float* Ct, const float* Cn,
                const float* Nn, const float* Gn, const double* dloss, const int32_t* lab,
                cudaStream_t st) {
  const int half = (A.k + 1) / 2;   // two centroids per thread
  const int thr = std::max(32, (half + 31) / 32 * 32);
  k_soft_col<D, MODE><<<dim3(P.ns, A.B), thr, 0, st>>>(A, Ct, Cn, Nn, Gn, dloss, lab);
}

void launch_reduce(const SoftArgs& A, int d, int mode, const float* Ct, float* Cnext, float* Nout,
                   float* Gout, cudaStream_t st, const float* Nn = nullptr,
                   const float* Gin = nullptr, const double* scale = nullptr) {
  const int64_t tot = (int64_t)A.B * A.k;
  k_soft_reduce<<<(int)((tot + 255) / 256), 256, 0, st>>>(A, d, mode, Ct, Cnext, Nout, Gout, Nn,
                                                          Gin, scale);
}

dkm_status finish_loss(const SoftScratch& S, const SoftPlan& P, int B, double* loss, cudaStream_t st) {
  k_soft_loss<<<(B + 127) / 128, 128, 0, st>>>(S.loss_part, P.gx, B, S.loss_dev);
  SOFT_CK(cudaGetLastError());
  if (loss) {
    SOFT_CK(cudaMemcpyAsync(loss, S.loss_dev, sizeof(double) * B, cudaMemcpyDefault, st));
  }
  return DKM_OK;
}

// the argument block with the row statistics of step t in the caller's
// arrays (stats: T x [m | iz] x n_total)
SoftArgs step_args(const SoftScratch& S, const SoftPlan& P, const float* stats, int t) {
  SoftArgs A = S.A;
  if (stats) {
    const size_t n = (size_t)P.n_total;
    A.m = const_cast<float*>(stats) + (size_t)(2 * t) * n;
    A.iz = const_cast<float*>(stats) + (size_t)(2 * t + 1) * n;
  }
  return A;
}

template <int D>
dkm_status soft_forward_impl(const float* pts, const SoftPlan& P, int B, int k, const float* init,
                             int T, const float* tau, float* ckpt, double* loss, float* stats,
                             float* norms, cudaStream_t st) {
  SoftScratch S;
  dkm_status r = soft_alloc(P, B, D, k, tau, st, &S);
  if (r != DKM_OK) return r;
  S.A.P = pts;
  const size_t ck = (size_t)B * k * D;   // floats per checkpoint
  SOFT_CK(cudaMemcpyAsync(ckpt, init, sizeof(float) * ck, cudaMemcpyDefault, st));
  for (int t = 0; t < T; ++t) {
    const float* Ct = ckpt + t * ck;
    const SoftArgs At = step_args(S, P, stats, t);
    launch_row<D, kRowStats>(At, S, P, Ct, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                             st);
    launch_col<D, kColMean>(At, P, Ct, nullptr, nullptr, nullptr, nullptr, nullptr, st);
    launch_reduce(At, D, 0, Ct, ckpt + (t + 1) * ck, norms ? norms + (size_t)t * B * k : nullptr,
                  nullptr, st);
  }
  launch_row<D, kRowLoss>(S.A, S, P, ckpt + T * ck, nullptr, nullptr, nullptr, nullptr, nullptr,
                          nullptr, st);
  r = finish_loss(S, P, B, loss, st);
  if (r != DKM_OK) return r;
  SOFT_CK(cudaGetLastError());
  SOFT_CK(cudaStreamSynchronize(st));
  return DKM_OK;
}

template <int D>
dkm_status soft_backward_impl(const float* pts, const SoftPlan& P, int B, int k, const float* ckpt,
                              int T, const float* tau, const double* dloss, const float* stats,
                              const float* norms, float* gp, float* gi, cudaStream_t st) {
  SoftScratch S;
  dkm_status r = soft_alloc(P, B, D, k, tau, st, &S);
  if (r != DKM_OK) return r;
  S.A.P = pts;
  double* dl = S.loss_dev;   // upstream gradient per cloud, on the device
  SOFT_CK(cudaMemcpyAsync(dl, dloss, sizeof(double) * B, cudaMemcpyDefault, st));
  const size_t ck = (size_t)B * k * D;
  // loss stage
  const float* CT = ckpt + T * ck;
  launch_row<D, kRowLossBwd>(S.A, S, P, CT, nullptr, nullptr, nullptr, dl, gp, nullptr, st);
  launch_col<D, kColLoss>(S.A, P, CT, nullptr, nullptr, nullptr, dl, nullptr, st);
  int cur = 0;
  launch_reduce(S.A, D, 1, CT, nullptr, nullptr, S.G[cur], st);
  // the updates, last first
  const bool given = stats && norms;   // the forward's per-step statistics
  for (int t = T - 1; t >= 0; --t) {
    const float* Ct = ckpt + t * ck;
    const float* Cn = ckpt + (t + 1) * ck;
    SoftArgs At = S.A;
    const float* N = S.N;
    if (given) {
      At = step_args(S, P, stats, t);
      At.use_stats = 1;
      N = norms + (size_t)t * B * k;
    } else {
      launch_row<D, kRowStats>(S.A, S, P, Ct, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                               st);
      launch_col<D, kColMean>(S.A, P, Ct, nullptr, nullptr, nullptr, nullptr, nullptr, st);
      launch_reduce(S.A, D, 0, Ct, nullptr, S.N, nullptr, st);
    }
    launch_row<D, kRowStep>(At, S, P, Ct, Cn, N, S.G[cur], nullptr, gp, nullptr, st);
    launch_col<D, kColStep>(At, P, Ct, Cn, N, S.G[cur], nullptr, nullptr, st);
    launch_reduce(At, D, 1, Ct, nullptr, nullptr, S.G[cur ^ 1], st, N, S.G[cur]);
    cur ^= 1;
  }
  SOFT_CK(cudaMemcpyAsync(gi, S.G[cur], sizeof(float) * ck, cudaMemcpyDefault, st));
  SOFT_CK(cudaGetLastError());
  SOFT_CK(cudaStreamSynchronize(st));
  return DKM_OK;
}

template <int D>
dkm_status hard_impl(const float* pts, const SoftPlan& P, int B, int k, const float* C,
                     int32_t* labels, double* loss, float* gp, float* gc, cudaStream_t st) {
  SoftScratch S;
  std::vector<float> ones((size_t)B, 1.f);   // the temperature is unused here
  dkm_status r = soft_alloc(P, B, D, k, ones.data(), st, &S);
  if (r != DKM_OK) return r;
  S.A.P = pts;
  int32_t* lab = labels ? labels : S.labels;
  launch_row<D, kRowHard>(S.A, S, P, C, nullptr, nullptr, nullptr, nullptr, gp, lab, st);
  r = finish_loss(S, P, B, loss, st);
  if (r != DKM_OK) return r;
  if (gc) {
    launch_col<D, kColHard>(S.A, P, C, nullptr, nullptr, nullptr, nullptr, lab, st);
    launch_reduce(S.A, D, 1, C, nullptr, nullptr, gc, st);
  }
  SOFT_CK(cudaGetLastError());
  SOFT_CK(cudaStreamSynchronize(st));
  return DKM_OK;
}

template <int D>
dkm_status hard_backward_impl(const float* pts, const SoftPlan& P, int B, int k, const float* C,
                              const int32_t* labels, const double* dloss, float* gp, float* gc,
                              cudaStream_t st) {
  SoftScratch S;
  std::vector<float> ones((size_t)B, 1.f);   // the temperature is unused here
  dkm_status r = soft_alloc(P, B, D, k, ones.data(), st, &S);
  if (r != DKM_OK) return r;
  S.A.P = pts;
  double* dl = S.loss_dev;   // upstream gradient per cloud, on the device
  SOFT_CK(cudaMemcpyAsync(dl, dloss, sizeof(double) * B, cudaMemcpyDefault, st));
  if (gp)
    launch_row<D, kRowHardBwd>(S.A, S, P, C, nullptr, nullptr, nullptr, dl, gp,
                               const_cast<int32_t*>(labels), st);
  if (gc) {
    launch_col<D, kColHard>(S.A, P, C, nullptr, nullptr, nullptr, nullptr, labels, st);
    launch_reduce(S.A, D, 1, C, nullptr, nullptr, gc, st, nullptr, nullptr, dl);
  }
  int bad = 0;
  SOFT_CK(cudaGetLastError());
  SOFT_CK(cudaMemcpyAsync(&bad, S.A.bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  SOFT_CK(cudaStreamSynchronize(st));
  if (bad) return soft_fail(DKM_EINVAL, "dkm_hard_sse_backward: a label lies outside [0, k)");
  return DKM_OK;
}

// tau_b = frac * squared diagonal of cloud b's bounding box: one CTA per
// cloud; the extents are FP32 differences of the box corners and the
// squares are summed in FP64.
__global__ void __launch_bounds__(512) k_soft_tau(const float* __restrict__ P,
                                                 const int64_t* __restrict__ off, int d,
                                                 double frac, float* __restrict__ tau) {
  __shared__ float s_lo[3][16], s_hi[3][16];
  const int b = blockIdx.x;
  const int64_t o0 = off[b], o1 = off[b + 1];
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = o0 + threadIdx.x; i < o1; i += blockDim.x)
    for (int a = 0; a < d; ++a) {
      const float v = P[i * d + a];
      lo[a] = fminf(lo[a], v);
      hi[a] = fmaxf(hi[a], v);
    }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int a = 0; a < 3; ++a) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
      hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
    }
    if (lane == 0) {
      s_lo[a][w] = lo[a];
      s_hi[a][w] = hi[a];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double q = 0.0;
    for (int a = 0; a < d; ++a) {
      float l = INFINITY, h = -INFINITY;
      for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) {
        l = fminf(l, s_lo[a][ww]);
        h = fmaxf(h, s_hi[a][ww]);
      }
      const double e = (double)__fsub_rn(h, l);
      q += e * e;
    }
    tau[b] = (float)(frac * q);
  }
}

}  // namespace
}  // namespace dkm

using namespace dkm;

extern "C" {

DKM_API dkm_status dkm_soft_forward(const float* points, const int64_t* offsets, int B, int d,
                                    int k, const float* init_centroids, int T, const float* tau,
                                    float* ckpt, double* loss, float* stats, float* norms,
                                    void* stream) {
  SoftPlan P;
  dkm_status r = soft_plan(offsets, B, d, k, &P);
  if (r != DKM_OK) return r;
  if (T < 0) return soft_fail(DKM_EINVAL, "T must be >= 0");
  if (!points || !init_centroids || !tau || !ckpt) return soft_fail(DKM_EINVAL, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  return d == 3 ? soft_forward_impl<3>(points, P, B, k, init_centroids, T, tau, ckpt, loss, stats,
                                       norms, st)
                : soft_forward_impl<2>(points, P, B, k, init_centroids, T, tau, ckpt, loss, stats,
                                       norms, st);
}

DKM_API dkm_status dkm_soft_backward(const float* points, const int64_t* offsets, int B, int d,
                                     int k, const float* ckpt, int T, const float* tau,
                                     const double* dloss, const float* stats, const float* norms,
                                     float* grad_points, float* grad_init, void* stream) {
  SoftPlan P;
  dkm_status r = soft_plan(offsets, B, d, k, &P);
  if (r != DKM_OK) return r;
  if (T < 0) return soft_fail(DKM_EINVAL, "T must be >= 0");
  if (!points || !ckpt || !tau || !dloss || !grad_points || !grad_init)
    return soft_fail(DKM_EINVAL, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  return d == 3 ? soft_backward_impl<3>(points, P, B, k, ckpt, T, tau, dloss, stats, norms,
                                        grad_points, grad_init, st)
                : soft_backward_impl<2>(points, P, B, k, ckpt, T, tau, dloss, stats, norms,
                                        grad_points, grad_init, st);
}

DKM_API dkm_status dkm_hard_sse_backward(const float* points, const int64_t* offsets, int B,
                                         int d, int k, const float* centroids,
                                         const int32_t* labels, const double* dloss,
                                         float* grad_points, float* grad_centroids,
                                         void* stream) {
  SoftPlan P;
  dkm_status r = soft_plan(offsets, B, d, k, &P);
  if (r != DKM_OK) return r;
  if (!points || !centroids || !labels || !dloss) return soft_fail(DKM_EINVAL, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  return d == 3 ? hard_backward_impl<3>(points, P, B, k, centroids, labels, dloss, grad_points,
                                        grad_centroids, st)
                : hard_backward_impl<2>(points, P, B, k, centroids, labels, dloss, grad_points,
                                        grad_centroids, st);
}

DKM_API dkm_status dkm_soft_temperature(const float* points, const int64_t* offsets, int B, int d,
                                        double frac, float* tau, void* stream) {
  SoftPlan P;
  dkm_status r = soft_plan(offsets, B, d, 1, &P);
  if (r != DKM_OK) return r;
  if (!points || !tau) return soft_fail(DKM_EINVAL, "null argument");
  if (!(frac > 0.0) || !std::isfinite(frac)) return soft_fail(DKM_EINVAL, "frac must be > 0");
  cudaStream_t st = (cudaStream_t)stream;
  char* buf = nullptr;
  const size_t ob = sizeof(int64_t) * (B + 1);
  SOFT_CK(cudaMallocAsync((void**)&buf, ob + sizeof(float) * B, st));
  int64_t* doff = (int64_t*)buf;
  float* dtau = (float*)(buf + ob);
  cudaError_t e = cudaMemcpyAsync(doff, P.off.data(), ob, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    k_soft_tau<<<B, 512, 0, st>>>(points, doff, d, frac, dtau);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(tau, dtau, sizeof(float) * B, cudaMemcpyDefault, st);
  cudaFreeAsync(buf, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return soft_fail(DKM_ECUDA, "dkm_soft_temperature", e);
  }
  return DKM_OK;
}

DKM_API dkm_status dkm_hard_sse(const float* points, const int64_t* offsets, int B, int d, int k,
                                const float* centroids, int32_t* labels, double* loss,
                                float* grad_points, float* grad_centroids, void* stream) {
  SoftPlan P;
  dkm_status r = soft_plan(offsets, B, d, k, &P);
  if (r != DKM_OK) return r;
  if (!points || !centroids) return soft_fail(DKM_EINVAL, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  return d == 3 ? hard_impl<3>(points, P, B, k, centroids, labels, loss, grad_points,
                               grad_centroids, st)
                : hard_impl<2>(points, P, B, k, centroids, labels, loss, grad_points,
                               grad_centroids, st);
}

}  // extern "C"
