// dkm_noalloc.cu -- one Lloyd step that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a host
// framework which owns all device memory through its own allocator, or a
// latency-critical loop where cudaMalloc / cudaFree would synchronise the
// device.  dkm_lloyd_step_noalloc serves them: the caller passes every input
// and output, and the only scratch the step needs (per-cluster sums, the
// SSE counters, a bounding box) lives in one fixed-size file-scope device
// array below.  The paper has no counterpart to this entry point.
//
// The step is plain Lloyd (every point against every centroid), with the
// same FP32 distance expression and lowest-index tie rule as the rest of
// libdkm, so its labels equal dkm_assign's for the same centroids.
#include <algorithm>
#include <mutex>
#include <string>

#include "dkm_host.h"

namespace dkm {
namespace {

constexpr int kNaMaxK = DKM_NOALLOC_MAX_K;
constexpr int kNaSlots = 256;
constexpr int kNaChunk = 1024;   // centroids staged in shared memory per round

// What the host reads back after a step (one copy).
struct NaResult {
  double sse;   // SSE of the labels against the input centroids (NaN if bad)
  int bad;      // a point or centroid coordinate was NaN or infinite
  int pad;
};

struct NaScratch {
  Acc acc[kNaMaxK];                  // per-cluster residual sums (fixed point) + counts
  unsigned long long sse[kNaSlots];  // spread SSE counters (fixed point)
  DevState st;                       // bounding boxes for the fixed-point scale
  NaResult res;
};

// Every GPU that loads the library holds this array until the process
// exits.  Host code must not take its address directly (that is a host-side
// stand-in); it uses the address returned by cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_na_scratch[sizeof(NaScratch)];

__global__ void k_na_clear(NaScratch* s, int k, int d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < k) s->acc[i] = Acc{{0ull, 0ull, 0ull}, 0ull};
  if (i < kNaSlots) s->sse[i] = 0ull;
  if (i == 0) s->res.bad = 0;
  if (i < 3) {
    unsigned lo = i < d ? 0xffffffffu : ord_of(0.f), hi = i < d ? 0u : ord_of(0.f);
    s->st.pbox[i] = lo;
    s->st.pbox[3 + i] = hi;
    s->st.cbox[i] = lo;
    s->st.cbox[3 + i] = hi;
  }
}

// bounding box of an m x d array into pbox (which = 0) or cbox (which = 1);
// a NaN or infinite coordinate sets res.bad
__global__ void k_na_bbox(const float* __restrict__ p, int64_t m, int d, NaScratch* s, int which) {
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int a = 0; a < d; ++a) {
      const float v = p[i * d + a];
      bad = bad || !isfinite(v);
      lo[a] = fminf(lo[a], v);
      hi[a] = fmaxf(hi[a], v);
    }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&s->res.bad, 1);
  for (int a = 0; a < 3; ++a)
    for (int o = 16; o > 0; o >>= 1) {
      lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
      hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
    }
  if ((threadIdx.x & 31) == 0) {
    unsigned* box = which == 0 ? s->st.pbox : s->st.cbox;
    for (int a = 0; a < d; ++a)
      if (lo[a] <= hi[a]) {
        atomicMin(&box[a], ord_of(lo[a]));
        atomicMax(&box[3 + a], ord_of(hi[a]));
      }
  }
}

// One thread per point (input order), centroids staged through shared
// memory in id order, strict < so ties keep the lowest index.  Residual
// sums are grouped by label per warp in 32-bit fixed point and added with
// 64-bit integer atomics (exact, order independent).
template <int D>
__global__ void __launch_bounds__(256) k_na_assign(const float* __restrict__ pts, int64_t n, int k,
                                                   const float* __restrict__ C,
                                                   int32_t* __restrict__ labels, NaScratch* s) {
  __shared__ float4 s_c[kNaChunk];
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool v = i < n;
  if (s->res.bad) {   // non-finite input (the same flag for every thread): no labels
    if (v) labels[i] = -1;
    return;
  }
  float px = 0.f, py = 0.f, pz = 0.f;
  if (v) {
    px = pts[i * D + 0];
    py = pts[i * D + 1];
    if (D == 3) pz = pts[i * D + 2];
  }
  float best = INFINITY;
  int bid = 0;
  for (int c0 = 0; c0 < k; c0 += kNaChunk) {
    const int m = min(kNaChunk, k - c0);
    __syncthreads();
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      const int64_t g = c0 + j;
      s_c[j] = make_float4(C[g * D + 0], C[g * D + 1], D == 3 ? C[g * D + 2] : 0.f, 0.f);
    }
    __syncthreads();
    for (int j = 0; j < m; ++j) {
      const float4 c = s_c[j];
      const float dx = __fadd_rn(px, -c.x), dy = __fadd_rn(py, -c.y);
      float d2 = __fmaf_rn(dy, dy, __fmul_rn(dx, dx));
      if (D == 3) {
        const float dz = __fadd_rn(pz, -c.z);
        d2 = __fmaf_rn(dz, dz, d2);
      }
      if (d2 < best) {
        best = d2;
        bid = c0 + j;
      }
    }
  }
  if (v) labels[i] = bid;

  int s_glob, s_sse;
  fixed_exponents(&s->st, n, &s_glob, &s_sse);
  // residual to the chosen centroid, then a per-warp power-of-two scale
  float rx = 0.f, ry = 0.f, rz = 0.f;
  if (v) {
    rx = __fadd_rn(px, -C[(int64_t)bid * D + 0]);
    ry = __fadd_rn(py, -C[(int64_t)bid * D + 1]);
    if (D == 3) rz = __fadd_rn(pz, -C[(int64_t)bid * D + 2]);
  }
  const float ml = fmaxf(fmaxf(fabsf(rx), fabsf(ry)), fabsf(rz));
  const float mr = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(ml)));
  const int s_row = mr > 0.f ? min(24 - exp_bound(mr), 127) : 0;
  const float sc = pow2f(s_row);
  const int qx = __float2int_rn(rx * sc), qy = __float2int_rn(ry * sc), qz = __float2int_rn(rz * sc);
  bool pend = v;
  while (true) {
    const unsigned mk = __ballot_sync(0xffffffffu, pend);
    if (!mk) break;
    const int L = __shfl_sync(0xffffffffu, bid, __ffs(mk) - 1);
    const bool g = pend && bid == L;
    const int sx = __reduce_add_sync(0xffffffffu, g ? qx : 0);
    const int sy = __reduce_add_sync(0xffffffffu, g ? qy : 0);
    const int sz = D == 3 ? __reduce_add_sync(0xffffffffu, g ? qz : 0) : 0;
    const int cnt = __popc(__ballot_sync(0xffffffffu, g));
    if (lane == 0) {
      Acc* a = &s->acc[L];
      atomicAdd(&a->s[0], (unsigned long long)rescale(sx, s_row, s_glob));
      atomicAdd(&a->s[1], (unsigned long long)rescale(sy, s_row, s_glob));
      if (D == 3) atomicAdd(&a->s[2], (unsigned long long)rescale(sz, s_row, s_glob));
      atomicAdd(&a->cnt, (unsigned long long)cnt);
    }
    pend = pend && !g;
  }
  // SSE of this pass, same fixed-point scheme
  const float d2 = v ? best : 0.f;
  const float m2 = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(d2)));
  const int s2 = m2 > 0.f ? min(24 - exp_bound(m2), 127) : 0;
  const unsigned q2 = __reduce_add_sync(0xffffffffu, (unsigned)__float2uint_rn(d2 * pow2f(s2)));
  if (lane == 0)
    atomicAdd(&s->sse[(i >> 5) & (kNaSlots - 1)], (unsigned long long)rescale(q2, s2, s_sse));
}

__global__ void k_na_update(const float* __restrict__ C, int k, int d, int64_t n,
                            float* __restrict__ out, NaScratch* s) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const bool bad = s->res.bad != 0;
  if (j == 0) {
    int s_glob, s_sse;
    fixed_exponents(&s->st, n, &s_glob, &s_sse);
    unsigned long long t = 0;
    for (int q = 0; q < kNaSlots; ++q) t += s->sse[q];
    s->res.sse = bad ? __longlong_as_double(0x7ff8000000000000ll)
                     : (double)(long long)t * exp2(-(double)s_sse);
  }
  if (j >= k) return;
  if (bad) {   // non-finite input: the centroids pass through unchanged
    for (int t = 0; t < d; ++t) out[(int64_t)j * d + t] = C[(int64_t)j * d + t];
    return;
  }
  const Acc a = s->acc[j];
  const long long cnt = (long long)a.cnt;
  int s_glob, s_sse;
  fixed_exponents(&s->st, n, &s_glob, &s_sse);
  for (int t = 0; t < d; ++t) {
    const float c = C[(int64_t)j * d + t];
    out[(int64_t)j * d + t] = cnt > 0 ? refine_coord(c, (long long)a.s[t], cnt, s_glob) : c;
  }
}

std::mutex g_na_mutex;
void* g_na_ptr[128] = {};

thread_local std::string g_na_err;

dkm_status na_fail(dkm_status st, const char* msg, cudaError_t e = cudaSuccess) {
  g_na_err = msg;
  if (e != cudaSuccess) {
    g_na_err += ": ";
    g_na_err += cudaGetErrorString(e);
  }
  dkm_set_last_error(g_na_err.c_str());
  return st;
}

}  // namespace
}  // namespace dkm

using namespace dkm;

extern "C" DKM_API dkm_status dkm_lloyd_step_noalloc(const float* points, int64_t n, int d, int k,
                                                     const float* centroids,
                                                     float* centroids_out, int32_t* labels,
                                                     double* sse_out, void* stream) {
  if (d != 2 && d != 3) return na_fail(DKM_EINVAL, "dkm_lloyd_step_noalloc: d must be 2 or 3");
  if (n < 1 || n > (int64_t(1) << 31) - 1)
    return na_fail(DKM_EINVAL, "dkm_lloyd_step_noalloc: n out of range");
  if (k < 1 || k > kNaMaxK)
    return na_fail(DKM_EINVAL,
                   "dkm_lloyd_step_noalloc: k must be in [1, DKM_NOALLOC_MAX_K]; the fixed "
                   "scratch holds that many clusters");
  if (!points || !centroids || !centroids_out || !labels)
    return na_fail(DKM_EINVAL, "dkm_lloyd_step_noalloc: null pointer");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 128) {
    cudaGetLastError();
    return na_fail(DKM_ECUDA, "dkm_lloyd_step_noalloc: no usable CUDA device", e);
  }
  void* ptr = nullptr;
  {
    // set-up, once per device, with that device current
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
      e = cudaGetSymbolAddress(&ptr, g_na_scratch);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return na_fail(DKM_ECUDA, "dkm_lloyd_step_noalloc: cudaGetSymbolAddress failed", e);
      }
      g_na_ptr[dev] = ptr;
    }
    ptr = g_na_ptr[dev];
  }
  NaScratch* s = (NaScratch*)ptr;
  cudaStream_t st = (cudaStream_t)stream;
  const int nb = (int)((n + 255) / 256);
  k_na_clear<<<(std::max(k, kNaSlots) + 255) / 256, 256, 0, st>>>(s, k, d);
  k_na_bbox<<<std::min(nb, 1216), 256, 0, st>>>(points, n, d, s, 0);
  k_na_bbox<<<(k + 255) / 256, 256, 0, st>>>(centroids, k, d, s, 1);
  if (d == 3) k_na_assign<3><<<nb, 256, 0, st>>>(points, n, k, centroids, labels, s);
  else k_na_assign<2><<<nb, 256, 0, st>>>(points, n, k, centroids, labels, s);
  k_na_update<<<(k + 255) / 256, 256, 0, st>>>(centroids, k, d, n, centroids_out, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(DKM_ECUDA, "dkm_lloyd_step_noalloc: launch failed", e);
  if (sse_out) {
    NaResult res;
    e = cudaMemcpyAsync(&res, &s->res, sizeof(NaResult), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return na_fail(DKM_ECUDA, "dkm_lloyd_step_noalloc: SSE read-back", e);
    *sse_out = res.sse;
    if (res.bad)
      return na_fail(DKM_EINVAL, "dkm_lloyd_step_noalloc: a point or centroid coordinate is NaN "
                                 "or infinite (labels set to -1, centroids copied through)");
  }
  return DKM_OK;
}
