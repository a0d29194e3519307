// device_common.cuh -- sm_103a device primitives shared by the all-pairs kernels:
// mbarriers, 1-D TMA bulk copies, bounded waits, the hardware rsqrt and
// error-free transformations for compensated sums.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace nbody {

// Device error codes written to the error word (first error wins).
enum : int {
  kDevOk = 0,
  kDevTimeout = 1,   // a bounded mbarrier wait ran out
  kDevBadItem = 2,   // a work item failed its bounds check
};

// ~2 s at 2 GHz: no legitimate wait in these kernels comes near it.
constexpr long long kWaitLimitCycles = 4000000000LL;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void set_error(int *err, int code) {
  if (err) atomicCAS(err, 0, code);
}

// ---- mbarrier (shared::cta) -------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
      "r"(bytes)
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity to complete, for at most `limit`
// cycles (kWaitLimitCycles by default). Returns false (and records kDevTimeout)
// if it ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err,
                                          long long limit = kWaitLimitCycles) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) {
      set_error(err, kDevTimeout);
      return false;
    }
  }
  return true;
}

// ---- TMA: 1-D bulk copy global -> shared, completing on an mbarrier -----------
// dst and src 16-byte aligned, bytes a multiple of 16 (checked by callers).
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// ---- arithmetic ---------------------------------------------------------------
// Hardware reciprocal square root (MUFU.RSQ); s > 0 in every caller.
__device__ __forceinline__ float rsqrt_hw(float s) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(s));
  return y;
}

// One Newton-Raphson step for 1/sqrt(s): y <- y (3 - s y^2) / 2 (textbook).
__device__ __forceinline__ float rsqrt_newton(float y, float s) {
  const float hs = -0.5f * s;
  const float yy = y * y;
  return y * fmaf(hs, yy, 1.5f);
}

// Programmatic dependent launch: returns once the grid this one depends on has
// completed and its writes are visible (a no-op for a grid launched without the
// programmatic-serialization attribute). Called first thing by every kernel of
// the force / step chain, before it touches global memory. No kernel triggers
// its dependents early: the next grid is launched as this one's last CTAs exit,
// so its CTAs are placed on an idle GPU (placed while the previous grid still
// held the SMs, the CTAs of a grid under one wave bunch up on a few SMs).
__device__ __forceinline__ void griddep_start() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Knuth's TwoSum: s + e == a + b exactly, s = fl(a + b).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Add b into the compensated pair (hi, lo).
__device__ __forceinline__ void comp_add(float &hi, float &lo, float b) {
  float s, e;
  two_sum(hi, b, s, e);
  hi = s;
  lo = __fadd_rn(lo, e);
}

// Scale of the 64-bit fixed-point accumulation of softened gravity: the largest
// power of two 2^S for which every sum a target can reach, |sum_j m_j d / s^3| <=
// M 2 / (3 sqrt(3) eps^2) and |sum_j m_j / s| <= M / eps (M = sum |m_j|, the
// maximum of r / (r^2 + eps^2)^(3/2) being 2 / (3 sqrt(3) eps^2)), stays below 2^62.
// Writes 2^S and 2^-S.
__device__ __forceinline__ void fixed_scale_of(double M, float eps2, float *scale, double *inv) {
  const double e2 = double(eps2);
  const double bound = fmax(M * 0.3849001794597505 / e2, M / sqrt(e2)) + 1e-300;
  int S = int(floor(62.0 - log2(bound)));
  S = S > 126 ? 126 : (S < -126 ? -126 : S);
  *scale = ldexpf(1.0f, S);
  *inv = ldexp(1.0, -S);
}

}  // namespace nbody
