// aux_kernels.cuh -- O(N) kernels around the all-pairs force kernel:
//   packing (caller SoA doubles -> float4 streams),
//   finalize (fixed-order compensated sum of the per-slice partials, law
//         scaling, leapfrog kick/drift, position trace),
//   FP64 diagnostics (block partials, then one deterministic final sum).
#pragma once

#include <cstdint>

#include "aux_types.h"
#include "device_common.cuh"
#include "fixed_point.cuh"
#include "leapfrog.cuh"

namespace nbody {

// Sum of 8 doubles over the block in a fixed order; thread 0 gets the result.
__device__ __forceinline__ void block_sum8(double v[kDiagFields], double *out) {
  __shared__ double red[kFinThreads / 32][kDiagFields];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kDiagFields; ++k) {
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
    if (lane == 0) red[warp][k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x < kDiagFields) {
    double s = 0.0;
    for (int w = 0; w < kFinThreads / 32; ++w) s += red[w][threadIdx.x];
    out[threadIdx.x] = s;
  }
}

__global__ void __launch_bounds__(kFinThreads) finalize_kernel(const FinalizeArgs f) {
  griddep_start();
  const int i = blockIdx.x * kFinThreads + threadIdx.x;
  double dv[kDiagFields] = {0, 0, 0, 0, 0, 0, 0, 0};
  float4 xn = make_float4(1e18f, 1e18f, 1e18f, 0.0f);  // drifted position (pad: far away)
  if (i < f.n) {
    int law = f.law, slices = f.slices;
    float G = f.G, dt = f.dt;
    bool live = true;
    if (f.sys_of) {
      const int s = f.sys_of[i];
      if (s < 0) {
        live = false;
      } else {
        const SysInfo si = f.sys[s];
        law = si.law;
        slices = si.slices;
        G = si.G;
        dt = si.dt;
      }
    }
    if (live) {
      float4 t, r;
      // The slots that count, in index order: with the symmetric tiles' source
      // split (sp parts per block) a particle of block own_b and part own_s gets,
      // below its own block, only its part's slot of each block (kb * sp + own_s),
      // and from its own block on every slot; without a split, every slot.
      const int sp = f.sym_split > 1 ? f.sym_split : 1;
      const int own_b = sp > 1 ? i / f.sym_block : 0;
      const int own_s = sp > 1 ? ((i - own_b * f.sym_block) >> 1) / (f.sym_block / 2 / sp) : 0;
      const int k_all = own_b * sp;  // first slot from which every slot counts
      if (f.fx_inv) {
        // 64-bit fixed-point partials: exact integer sum, one rounding at the end
        long long sx = 0, sy = 0, sz = 0, sw = 0;
        // atomic plans: integer parts in words 0-3, fractions (units of 2^-32) in 4-7
        long long fr[4] = {0, 0, 0, 0};
        if (f.acc64) {  // already summed by the force kernel's integer atomics
          const long long st = f.stride;
          sx = f.acc64[i];
          sy = f.acc64[st + i];
          sz = f.acc64[2 * st + i];
          sw = f.acc64[3 * st + i];
#pragma unroll
          for (int c = 0; c < 4; ++c) fr[c] = f.acc64[(4 + c) * st + i];
          if (f.rezero) {  // ready for the next evaluation of this call
#pragma unroll
            for (int c = 0; c < 8; ++c) f.acc64[c * st + i] = 0;
          }
        }
        auto take = [&](int k) {
          const long long *ph = reinterpret_cast<const long long *>(f.part_hi) +
                                2 * ((long long)k * f.stride + i);
          const long long *pl = reinterpret_cast<const long long *>(f.part_lo) +
                                2 * ((long long)k * f.stride + i);
          sx += ph[0];
          sy += ph[1];
          sz += pl[0];
          sw += pl[1];
        };
        if (!f.acc64) {
          for (int kb = 0; kb < own_b; ++kb) take(kb * sp + own_s);
          for (int k = k_all; k < slices; ++k) take(k);
        }
        const double inv = *f.fx_inv;
        const double dx = fixed_value(sx, fr[0], inv), dy = fixed_value(sy, fr[1], inv),
                     dz = fixed_value(sz, fr[2], inv), dw = fixed_value(sw, fr[3], inv);
        t = make_float4(float(dx), float(dy), float(dz), float(dw));
        r = make_float4(float(dx - double(t.x)), float(dy - double(t.y)),
                        float(dz - double(t.z)), float(dw - double(t.w)));
      } else {
        // part_lo == nullptr: partials without low parts (symmetric tiles)
        const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 hi = zero, lo = zero;
        const bool plain = f.plain != 0;
        auto add = [&](const float4 &h, const float4 &l) {
          if (plain) {
            hi.x = __fadd_rn(hi.x, h.x);
            hi.y = __fadd_rn(hi.y, h.y);
            hi.z = __fadd_rn(hi.z, h.z);
            hi.w = __fadd_rn(hi.w, h.w);
          } else {
            comp_add(hi.x, lo.x, h.x);
            comp_add(hi.y, lo.y, h.y);
            comp_add(hi.z, lo.z, h.z);
            comp_add(hi.w, lo.w, h.w);
          }
          lo.x = __fadd_rn(lo.x, l.x);
          lo.y = __fadd_rn(lo.y, l.y);
          lo.z = __fadd_rn(lo.z, l.z);
          lo.w = __fadd_rn(lo.w, l.w);
        };
        // `count` slots k0, k0 + step, ...; loads issued eight slots ahead of the
        // adds (the symmetric tiles leave one slot per block and source part: a
        // hundred or more per particle, read by few CTAs at small N)
        auto run = [&](int k0, int count, int step) {
          constexpr int U = 8;
          int c = 0;
          for (; c + U <= count; c += U) {
            float4 h[U], l[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const long long o = (long long)(k0 + (c + u) * step) * f.stride + i;
              h[u] = f.part_hi[o];
              l[u] = f.part_lo ? f.part_lo[o] : zero;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) add(h[u], l[u]);
          }
          for (; c < count; ++c) {
            const long long o = (long long)(k0 + c * step) * f.stride + i;
            add(f.part_hi[o], f.part_lo ? f.part_lo[o] : zero);
          }
        };
        run(own_s, own_b, sp);
        run(k_all, slices - k_all, 1);
        // Round hi + lo to FP32 and keep the residual (Fast2Sum, |hi| >= |lo|).
        t.x = __fadd_rn(hi.x, lo.x);
        r.x = __fsub_rn(lo.x, __fsub_rn(t.x, hi.x));
        t.y = __fadd_rn(hi.y, lo.y);
        r.y = __fsub_rn(lo.y, __fsub_rn(t.y, hi.y));
        t.z = __fadd_rn(hi.z, lo.z);
        r.z = __fsub_rn(lo.z, __fsub_rn(t.z, hi.z));
        t.w = __fadd_rn(hi.w, lo.w);
        r.w = __fsub_rn(lo.w, __fsub_rn(t.w, hi.w));
      }
      float4 x = f.pos[i];
      float4 a, alo;
      if (law == 0) {  // gravity: a = G sum m_j y^3 d, phi = -G sum m_j y
        a = make_float4(G * t.x, G * t.y, G * t.z, -G * t.w);
        alo = make_float4(G * r.x, G * r.y, G * r.z, -G * r.w);
      } else {  // LJC: F = -sum f d, a = F / m; phi = sum of pair energies
        const float inv_m = 1.0f / x.w;
        a = make_float4(-t.x * inv_m, -t.y * inv_m, -t.z * inv_m, t.w);
        alo = make_float4(-r.x * inv_m, -r.y * inv_m, -r.z * inv_m, r.w);
      }
      if (f.mode & kFinWriteAcc) {
        f.acc[i] = a;
        if (f.acc_lo) f.acc_lo[i] = alo;
      }
      if (f.mode & (kFinKickSync | kFinDiag | kFinKickDrift)) {
        float4 v = f.vel[i];
        const float h = 0.5f * dt;
        const bool two = f.x_lo != nullptr;
        float4 xl = two ? f.x_lo[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 vl = two ? f.v_lo[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        if (f.mode & kFinKickSync) {
          if (two) {
            comp_axpy(v, vl, h, a);
          } else {
            v.x = fmaf(h, a.x, v.x);
            v.y = fmaf(h, a.y, v.y);
            v.z = fmaf(h, a.z, v.z);
          }
        }
        if (f.mode & kFinDiag) {
          const double m = x.w;
          const double vx = v.x, vy = v.y, vz = v.z;
          const double px = x.x, py = x.y, pz = x.z;
          dv[0] = 0.5 * m * (vx * vx + vy * vy + vz * vz);
          dv[1] = (law == 0) ? 0.5 * m * (double)a.w : 0.5 * (double)a.w;
          dv[2] = m * vx;
          dv[3] = m * vy;
          dv[4] = m * vz;
          dv[5] = m * (py * vz - pz * vy);
          dv[6] = m * (pz * vx - px * vz);
          dv[7] = m * (px * vy - py * vx);
        }
        if (f.mode & kFinKickDrift) {
          if (two) {
            comp_axpy(v, vl, h, a);
            // drift with the full two-float velocity
            const float4 vv = make_float4(v.x + vl.x, v.y + vl.y, v.z + vl.z, 0.f);
            comp_axpy(x, xl, dt, vv);
          } else {
            v.x = fmaf(h, a.x, v.x);
            v.y = fmaf(h, a.y, v.y);
            v.z = fmaf(h, a.z, v.z);
            x.x = fmaf(dt, v.x, x.x);
            x.y = fmaf(dt, v.y, x.y);
            x.z = fmaf(dt, v.z, x.z);
          }
          f.pos[i] = x;
          xn = x;
          if (f.trace_next) f.trace_next[i] = x;
        }
        f.vel[i] = v;
        if (two) {
          f.x_lo[i] = xl;
          f.v_lo[i] = vl;
        }
      }
    }
  }
  if (f.jnext) {  // the same for every thread of the launch
    // particles 2p and 2p + 1 are neighbouring lanes: exchange positions, then the
    // even lane writes the pair's (x x y y) word and the odd lane the (z z) half of
    // its second word (the even lane as well when its partner is the pad past n)
    const float px = __shfl_xor_sync(0xffffffffu, xn.x, 1);
    const float py = __shfl_xor_sync(0xffffffffu, xn.y, 1);
    const float pz = __shfl_xor_sync(0xffffffffu, xn.z, 1);
    if (i < f.n) {
      const int p = i >> 1;
      long long q0, q1;
      if (f.jn_block > 0) {
        const int half = f.jn_block / 2, blk = p / half, pp = p - blk * half;
        q0 = (long long)blk * f.jn_words * half + pp;
        q1 = q0 + half;
      } else {
        q0 = (long long)f.jn_words * p;
        q1 = q0 + 1;
      }
      if ((i & 1) == 0) {
        f.jnext[q0] = make_float4(xn.x, px, xn.y, py);
        if (i + 1 >= f.n) *reinterpret_cast<float2 *>(f.jnext + q1) = make_float2(xn.z, pz);
      } else {
        *reinterpret_cast<float2 *>(f.jnext + q1) = make_float2(pz, xn.z);
      }
    }
  }
  if (!(f.mode & kFinDiag)) return;
  block_sum8(dv, f.diag_part + (size_t)blockIdx.x * kDiagFields);
  if (!f.diag_out) return;  // the same for every thread of the launch
  // The block that finishes last (atomicInc ticket, which wraps back to zero) adds
  // the block rows: thread t the rows t, t + kFinThreads, ... in order, then the
  // fixed tree of block_sum8 -- the same bits whichever block it is.
  __shared__ bool last;
  __threadfence();  // this block's row is visible before its ticket is taken
  __syncthreads();
  if (threadIdx.x == 0) last = atomicInc(f.diag_ticket, gridDim.x - 1) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  double v[kDiagFields] = {0, 0, 0, 0, 0, 0, 0, 0};
  const volatile double *rows = f.diag_part;
  for (int b = threadIdx.x; b < int(gridDim.x); b += kFinThreads)
#pragma unroll
    for (int k = 0; k < kDiagFields; ++k) v[k] += rows[(size_t)b * kDiagFields + k];
  block_sum8(v, f.diag_out);
}

// Scale of the fixed-point mode (fixed_scale_of) for the one-sided fixed-point
// tiles: one block; the mass sum runs in FP64 in a fixed order.
__global__ void __launch_bounds__(256) fixed_scale_kernel(const float4 *pos, int n, float eps2,
                                                          float *scale, double *inv) {
  __shared__ double part[256];
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) m += fabs(double(pos[i].w));
  part[threadIdx.x] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double M = 0.0;
    for (int k = 0; k < 256; ++k) M += part[k];
    fixed_scale_of(M, eps2, scale, inv);
  }
}

// First half-kick and drift from a caller-supplied acceleration (NBODY_ACC_VALID).
// Batched runs pass sys_of / sys for the per-system step size.
__global__ void kick_drift_kernel(float4 *pos, float4 *vel, const float4 *acc, int n, float dt,
                                  float4 *trace1, const int *sys_of, const SysInfo *sys,
                                  float4 *x_lo, float4 *v_lo) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (sys_of) {
    const int s = sys_of[i];
    if (s < 0) return;
    dt = sys[s].dt;
  }
  kick_drift_at(pos, vel, acc, dt, trace1, x_lo, v_lo, i);
}

// Packing: caller SoA doubles -> (x, y, z, m) float4.
__global__ void pack_grav_kernel(const double *x, const double *y, const double *z,
                                 const double *m, float4 *out, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_float4((float)x[i], (float)y[i], (float)z[i], (float)m[i]);
}

// Packing: LJC parameters (q~, s~, e~, type) with q~ = q sqrt(kq), s~ = sigma / 2,
// e~ = sqrt(24 eps); computed in FP64 and rounded once.
__global__ void pack_ljc_kernel(const double *q, const double *sig, const double *eps,
                                const int32_t *type, double sqrt_kq, float4 *out, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n)
    out[i] = make_float4((float)(q[i] * sqrt_kq), (float)(0.5 * sig[i]),
                         (float)sqrt(24.0 * eps[i]), (float)type[i]);
}

}  // namespace nbody
