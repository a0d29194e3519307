// fixed_point.cuh -- exact fixed-point accumulation of FP32 partial sums with
// 64-bit integer atomics (the GRAPE-6 scheme of Sec. 3.2), shared by the
// Newton-symmetric force and VJP kernels.
#pragma once

#include <cuda_runtime.h>

namespace nbody {

// Add the FP32 partial v, scaled by sc = 2^S (a power of two, so v sc is exact),
// to component c of one particle's accumulator: the integer part of v sc to word
// p[c st] and its fraction, in units of 2^-32, to word p[(4 + c) st]. Both are
// exact for an FP32 value (to 2^-(S+32)), so the integer sums are exact in any
// order whatever the scale makes of the grid spacing 2^-S; the fraction word is
// touched only when the fraction is nonzero (from 2^24 on an FP32 value has none).
// The scale keeps |v sc| below 2^62 for every sum a particle can reach.
__device__ __forceinline__ void fixed_add(unsigned long long *p, long long st, int c, float v,
                                          float sc) {
  const float t = v * sc;
  const float h = truncf(t);
  atomicAdd(p + c * st, static_cast<unsigned long long>(static_cast<long long>(h)));
  if (fabsf(t) < 16777216.0f) {
    const long long lo = __float2ll_rn((t - h) * 4294967296.0f);  // t - h is exact
    if (lo != 0) atomicAdd(p + (4 + c) * st, static_cast<unsigned long long>(lo));
  }
}

// The value of one component of a fixed-point accumulator: integer part hi and
// fraction fr (units of 2^-32) times inv = 2^-S, in FP64.
__device__ __forceinline__ double fixed_value(long long hi, long long fr, double inv) {
  return fma(double(fr), inv * 0x1p-32, double(hi) * inv);
}

}  // namespace nbody
