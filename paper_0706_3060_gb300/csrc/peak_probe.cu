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

// A quarter of the chains packed (FFMA2, 8 lane ops), the rest scalar (FFMA, 8 lane
// ops): 16 lane ops per iteration.
__global__ void __launch_bounds__(kThreads) probe_mixed(float *sink, int iters,
                                                        long long *cycles) {
  float2 a[kChains / 4];
  float b[kChains / 2];
#pragma unroll
  for (int k = 0; k < kChains / 4; ++k) a[k] = make_float2(threadIdx.x * 1e-3f + k, k + 0.5f);
#pragma unroll
  for (int k = 0; k < kChains / 2; ++k) b[k] = threadIdx.x * 2e-3f + k;
  const float2 m2 = make_float2(0.9999999f, 0.9999998f), c2 = make_float2(1e-7f, 2e-7f);
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains / 4; ++k) a[k] = __ffma2_rn(a[k], m2, c2);
#pragma unroll
    for (int k = 0; k < kChains / 2; ++k) b[k] = fmaf(b[k], 0.9999997f, 3e-7f);
  }
  __syncthreads();
  const long long t1 = clock64();
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains / 4; ++k) s += a[k].x + a[k].y;
#pragma unroll
  for (int k = 0; k < kChains / 2; ++k) s += b[k];
  if (s == 1234.5f) sink[blockIdx.x] = s;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// The gravity pair loop alone (no pipeline, no compensation): 2 targets per
// thread against 512 sources broadcast from shared memory, packed (PK) or
// scalar arithmetic. Reports 12 lane ops per pair.
template <bool PK>
__global__ void __launch_bounds__(kThreads) probe_pairs(float *sink, int iters,
                                                        long long *cycles) {
  __shared__ float4 src[512];
  for (int j = threadIdx.x; j < 512; j += kThreads)
    src[j] = make_float4(j * 1e-3f, 1.0f - j * 2e-3f, 0.5f + j * 1e-3f, 1e-3f);
  __syncthreads();
  const float xi[2] = {threadIdx.x * 1e-4f, 0.3f}, yi[2] = {0.1f, -0.2f}, zi[2] = {0.7f, 0.2f};
  float4 acc[2] = {make_float4(0, 0, 0, 0), make_float4(0, 0, 0, 0)};
  const float eps2 = 1e-4f;
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
    if (PK) {
      float2 ax[2], ay[2], az[2];
#pragma unroll
      for (int r = 0; r < 2; ++r) ax[r] = ay[r] = az[r] = make_float2(0.f, 0.f);
#pragma unroll 2
      for (int p = 0; p < 256; ++p) {
        const float4 A = src[2 * p], B = src[2 * p + 1];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const float2 dx = __fadd2_rn(make_float2(A.x, A.y), make_float2(-xi[r], -xi[r]));
          const float2 dy = __fadd2_rn(make_float2(A.z, A.w), make_float2(-yi[r], -yi[r]));
          const float2 dz = __fadd2_rn(make_float2(B.x, B.y), make_float2(-zi[r], -zi[r]));
          float2 s2 = __ffma2_rn(dz, dz, make_float2(eps2, eps2));
          s2 = __ffma2_rn(dy, dy, s2);
          s2 = __ffma2_rn(dx, dx, s2);
          float2 y;
          asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y.x) : "f"(s2.x));
          asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y.y) : "f"(s2.y));
          const float2 my = __fmul2_rn(make_float2(B.z, B.w), y);
          const float2 w = __fmul2_rn(my, __fmul2_rn(y, y));
          ax[r] = __ffma2_rn(w, dx, ax[r]);
          ay[r] = __ffma2_rn(w, dy, ay[r]);
          az[r] = __ffma2_rn(w, dz, az[r]);
        }
      }
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        acc[r].x += ax[r].x + ax[r].y;
        acc[r].y += ay[r].x + ay[r].y;
        acc[r].z += az[r].x + az[r].y;
      }
    } else {
#pragma unroll 4
      for (int j = 0; j < 512; ++j) {
        const float4 pj = src[j];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const float dx = pj.x - xi[r], dy = pj.y - yi[r], dz = pj.z - zi[r];
          const float s2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
          float y;
          asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(s2));
          const float my = pj.w * y;
          const float w = my * (y * y);
          acc[r].x = fmaf(w, dx, acc[r].x);
          acc[r].y = fmaf(w, dy, acc[r].y);
          acc[r].z = fmaf(w, dz, acc[r].z);
        }
      }
    }
  }
  const long long t1 = clock64();
  const float s = acc[0].x + acc[0].y + acc[0].z + acc[1].x + acc[1].y + acc[1].z;
  if (s == 1234.5f) sink[blockIdx.x] = s;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// A wait that nothing completes: one thread initialises an mbarrier that expects
// one arrival, never arrives, and waits on it with a short bound. The bounded
// wait gives up after `limit` cycles, records the timeout in the error word and
// the kernel returns -- the path every pipeline wait takes if a producer stalls.
__global__ void expired_wait_kernel(long long limit, int *err) {
  __shared__ __align__(8) uint64_t bar;
  nbody::mbar_init(&bar, 1);
  nbody::mbar_fence_init();
  nbody::mbar_wait(&bar, 0, err, limit);
}

}  // namespace

using namespace nbody;

extern "C" int nbody_selftest_timeout(int64_t limit_cycles, nbody_stream_t stream) {
  clear_error();
  if (limit_cycles < 1 || limit_cycles > 100000000LL)
    return set_error_msg(NBODY_EINVAL, "limit_cycles must be in [1, 1e8]");
  NB_TRY(check_device(nullptr, nullptr));
  int *err = nullptr;
  NB_TRY(error_word(&err));
  expired_wait_kernel<<<1, 1, 0, reinterpret_cast<cudaStream_t>(stream)>>>(limit_cycles, err);
  NB_CUDA(cudaGetLastError());
  return NBODY_OK;
}

extern "C" int nbody_peak_probe(int32_t kind, int32_t iters, double *ops_per_clk_sm,
                                double *ops_per_s) {
  clear_error();
  if (kind < 0 || kind > 5) return set_error_msg(NBODY_EINVAL, "kind must be 0 .. 5");
  if (iters < 1 || iters > (1 << 24)) return set_error_msg(NBODY_EINVAL, "iters out of range");
  int dev = 0, sms = 0;
  NB_TRY(check_device(&dev, &sms));
  // As many 256-thread blocks per SM as can be resident at once (at most 8 =
  // the SM's 2048-thread limit), so all blocks of an SM run concurrently.
  int per_sm = 8;
  {
    cudaError_t oe = cudaSuccess;
    if (kind == 4)
      oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, probe_pairs<true>, kThreads, 0);
    else if (kind == 5)
      oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, probe_pairs<false>, kThreads, 0);
    if (oe != cudaSuccess) return set_error_msg(NBODY_ECUDA, "occupancy query failed");
    per_sm = std::max(1, std::min(per_sm, 8));
  }
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
    else if (kind == 2) probe_mufu<<<blocks, kThreads>>>(sink, it, cyc);
    else if (kind == 3) probe_mixed<<<blocks, kThreads>>>(sink, it, cyc);
    else if (kind == 4) probe_pairs<true><<<blocks, kThreads>>>(sink, it, cyc);
    else probe_pairs<false><<<blocks, kThreads>>>(sink, it, cyc);
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
  // lane operations per iteration and thread: 16 (16 FFMA or MUFU chains, 8
  // FFMA2 chains of 2 lanes, or 4 FFMA2 + 8 FFMA chains), 12 x 2 targets x 512
  // sources for the pair loops
  const double per_iter = kind >= 4 ? 12.0 * 2 * 512 : double(kChains);
  const double total = double(blocks) * kThreads * per_iter * iters;
  long long cmax = *std::max_element(h.begin(), h.end());
  // all 8 blocks of an SM run concurrently, so an SM's cycle count is one block's
  if (ops_per_clk_sm) *ops_per_clk_sm = total / sms / double(cmax);
  if (ops_per_s) *ops_per_s = total / (ms * 1e-3);
  return NBODY_OK;
}
