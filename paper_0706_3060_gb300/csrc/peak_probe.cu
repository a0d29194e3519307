// peak_probe.cu -- throughput microbenchmarks for the units that bound the
// all-pairs kernels: FP32 FFMA (scalar and packed f32x2) and MUFU rsqrt. Each
// thread runs 16 independent dependency chains; per-SM cycles come from
// clock64, so the result (operations per SM per clock) does not depend on the
// clock the GPU happened to run at.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "api_common.h"

namespace {

constexpr int kChains = 16;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) probe_ffma(float *sink, int iters,
                                                       long long *cycles) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = threadIdx.x * 1e-3f + k;
  const float b = 0.9999999f, c = 1e-7f;
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
  }
  __syncthreads();
  const long long t1 = clock64();
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == 1234.5f) sink[blockIdx.x] = s;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

__global__ void __launch_bounds__(kThreads) probe_ffma2(float *sink, int iters,
                                                        long long *cycles) {
  float2 a[kChains / 2];
#pragma unroll
  for (int k = 0; k < kChains / 2; ++k) a[k] = make_float2(threadIdx.x * 1e-3f + k, k + 0.5f);
  const float2 b = make_float2(0.9999999f, 0.9999998f), c = make_float2(1e-7f, 2e-7f);
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains / 2; ++k) a[k] = __ffma2_rn(a[k], b, c);
  }
  __syncthreads();
  const long long t1 = clock64();
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains / 2; ++k) s += a[k].x + a[k].y;
  if (s == 1234.5f) sink[blockIdx.x] = s;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

__global__ void __launch_bounds__(kThreads) probe_mufu(float *sink, int iters,
                                                       long long *cycles) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1.0f + threadIdx.x * 1e-4f + k;
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      float y;
      asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[k]));
      a[k] = y;
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == 1234.5f) sink[blockIdx.x] = s;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace

using namespace nbody;

extern "C" int nbody_peak_probe(int32_t kind, int32_t iters, double *ops_per_clk_sm,
                                double *ops_per_s) {
  clear_error();
  if (kind < 0 || kind > 2) return set_error_msg(NBODY_EINVAL, "kind must be 0, 1 or 2");
  if (iters < 1 || iters > (1 << 24)) return set_error_msg(NBODY_EINVAL, "iters out of range");
  int dev = 0, sms = 0;
  NB_TRY(check_device(&dev, &sms));
  const int per_sm = 8;  // 8 x 256 threads = 2048 = the SM's thread limit
  const int blocks = sms * per_sm;
  float *sink = nullptr;
  long long *cyc = nullptr;
  NB_CUDA(cudaMalloc(&sink, sizeof(float) * blocks));
  NB_CUDA(cudaMalloc(&cyc, sizeof(long long) * blocks));
  cudaEvent_t e0, e1;
  NB_CUDA(cudaEventCreate(&e0));
  NB_CUDA(cudaEventCreate(&e1));
  auto launch = [&](int it) {
    if (kind == 0) probe_ffma<<<blocks, kThreads>>>(sink, it, cyc);
    else if (kind == 1) probe_ffma2<<<blocks, kThreads>>>(sink, it, cyc);
    else probe_mufu<<<blocks, kThreads>>>(sink, it, cyc);
  };
  launch(std::max(1, iters / 8));  // warm-up
  NB_CUDA(cudaEventRecord(e0));
  launch(iters);
  NB_CUDA(cudaEventRecord(e1));
  NB_CUDA(cudaEventSynchronize(e1));
  NB_CUDA(cudaGetLastError());
  float ms = 0.f;
  NB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  std::vector<long long> h(blocks);
  NB_CUDA(cudaMemcpy(h.data(), cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost));
  cudaFree(sink);
  cudaFree(cyc);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // lane operations per instruction: FFMA 1, FFMA2 2 (per thread), MUFU 1
  const double per_iter = double(kChains);
  const double total = double(blocks) * kThreads * per_iter * iters;
  long long cmax = *std::max_element(h.begin(), h.end());
  // all 8 blocks of an SM run concurrently, so an SM's cycle count is one block's
  if (ops_per_clk_sm) *ops_per_clk_sm = total / sms / double(cmax);
  if (ops_per_s) *ops_per_s = total / (ms * 1e-3);
  return NBODY_OK;
}
