// dkm_probe.cu -- device peak probe for roofline reporting (sm_103a).
//
// The ALU-bound kernels of libdkm (the brute-force assignment, the soft
// k-means row and column passes) are reported as a fraction of the FP32
// FMA throughput this device actually sustains.  dkm_device_peaks measures
// it with two plain FMA-chain kernels: scalar fmaf and packed f32x2
// __ffma2_rn (Blackwell issues two FP32 FMAs per packed instruction), each
// timed with CUDA events over a grid of eight 256-thread CTAs per SM.
#include <algorithm>
#include <string>

#include "dkm_host.h"

namespace dkm {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;     // independent FMA chains per thread
constexpr int kProbeIters = 2048;

__global__ void __launch_bounds__(kProbeThreads) k_fma_scalar(float* out, float b, float c) {
  float a[kProbeChains];
#pragma unroll
  for (int q = 0; q < kProbeChains; ++q) a[q] = (float)(threadIdx.x + q) * 1e-3f;
  for (int i = 0; i < kProbeIters; ++i) {
#pragma unroll
    for (int q = 0; q < kProbeChains; ++q) a[q] = __fmaf_rn(a[q], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < kProbeChains; ++q) s += a[q];
  out[blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) k_fma_packed(float* out, float b, float c) {
  float2 a[kProbeChains];
  const float2 bb = make_float2(b, b), cc = make_float2(c, c);
#pragma unroll
  for (int q = 0; q < kProbeChains; ++q)
    a[q] = make_float2((float)(threadIdx.x + q) * 1e-3f, (float)(threadIdx.x - q) * 1e-3f);
  for (int i = 0; i < kProbeIters; ++i) {
#pragma unroll
    for (int q = 0; q < kProbeChains; ++q) a[q] = __ffma2_rn(a[q], bb, cc);
  }
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < kProbeChains; ++q) s += a[q].x + a[q].y;
  out[blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

}  // namespace
}  // namespace dkm

using namespace dkm;

extern "C" DKM_API dkm_status dkm_device_peaks(dkm_peaks* out, void* stream) {
  if (!out) {
    dkm_set_last_error("dkm_device_peaks: null argument");
    return DKM_EINVAL;
  }
  *out = dkm_peaks{};
  int dev = 0, sms = 0, clk_khz = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
  cudaStream_t st = (cudaStream_t)stream;
  const int blocks = std::max(1, sms) * 8;
  float* buf = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&buf, sizeof(float) * blocks * kProbeThreads, st);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms_s = 0.f, ms_p = 0.f;
  if (e == cudaSuccess) {
    // a warm-up launch of each, then one timed launch of each
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
      if (rep) cudaEventRecord(e0, st);
      k_fma_scalar<<<blocks, kProbeThreads, 0, st>>>(buf, 0.999f, 1e-4f);
      if (rep) {
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_s, e0, e1);
      }
    }
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
      if (rep) cudaEventRecord(e0, st);
      k_fma_packed<<<blocks, kProbeThreads, 0, st>>>(buf, 0.999f, 1e-4f);
      if (rep) {
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_p, e0, e1);
      }
    }
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (buf) cudaFreeAsync(buf, st);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    std::string m = std::string("dkm_device_peaks: ") + cudaGetErrorString(e);
    dkm_set_last_error(m.c_str());
    return DKM_ECUDA;
  }
  const double fmas = (double)blocks * kProbeThreads * kProbeIters * kProbeChains;
  out->sm_count = sms;
  out->sm_clock_mhz = clk_khz / 1000;
  out->fp32_fma_tflops = ms_s > 0.f ? 2.0 * fmas / (ms_s * 1e-3) / 1e12 : 0.0;
  out->fp32x2_fma_tflops = ms_p > 0.f ? 4.0 * fmas / (ms_p * 1e-3) / 1e12 : 0.0;
  out->scalar_ms = ms_s;
  out->packed_ms = ms_p;
  return DKM_OK;
}
