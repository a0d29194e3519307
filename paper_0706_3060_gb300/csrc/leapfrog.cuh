// leapfrog.cuh -- per-particle leapfrog updates shared by the finalize, the
// kick-drift kernel and the pair-interleave kernels that apply a fused first
// half-kick and drift.
#pragma once

#include <cuda_runtime.h>

#include "device_common.cuh"

namespace nbody {

// Two-float state update (hi, lo) += c * d on xyz: the increment and the old
// low part are added first, then TwoSum splits the new value into the nearest
// float and its exact residual, so rounding does not accumulate over steps.
__device__ __forceinline__ void comp_axpy(float4 &hi, float4 &lo, float c, const float4 d) {
  float e;
  two_sum(hi.x, fmaf(c, d.x, lo.x), hi.x, e);
  lo.x = e;
  two_sum(hi.y, fmaf(c, d.y, lo.y), hi.y, e);
  lo.y = e;
  two_sum(hi.z, fmaf(c, d.z, lo.z), hi.z, e);
  lo.z = e;
}

// First half-kick and drift of particle i from a known acceleration (leapfrog,
// Sec. 2): v += dt/2 a, x += dt v, in place (with the two-float state when x_lo
// is given); writes the drifted position to trace1 (if given) and returns it.
__device__ __forceinline__ float4 kick_drift_at(float4 *pos, float4 *vel, const float4 *acc,
                                                float dt, float4 *trace1, float4 *x_lo,
                                                float4 *v_lo, int i) {
  float4 x = pos[i], v = vel[i];
  const float4 a = acc[i];
  const float h = 0.5f * dt;
  if (x_lo) {
    float4 xl = x_lo[i], vl = v_lo[i];
    comp_axpy(v, vl, h, a);
    const float4 vv = make_float4(v.x + vl.x, v.y + vl.y, v.z + vl.z, 0.f);
    comp_axpy(x, xl, dt, vv);
    x_lo[i] = xl;
    v_lo[i] = vl;
  } else {
    v.x = fmaf(h, a.x, v.x);
    v.y = fmaf(h, a.y, v.y);
    v.z = fmaf(h, a.z, v.z);
    x.x = fmaf(dt, v.x, x.x);
    x.y = fmaf(dt, v.y, x.y);
    x.z = fmaf(dt, v.z, x.z);
  }
  pos[i] = x;
  vel[i] = v;
  if (trace1) trace1[i] = x;
  return x;
}

}  // namespace nbody
