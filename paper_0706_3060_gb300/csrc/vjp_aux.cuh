// vjp_aux.cuh -- the O(N) kernels of the reverse sweep and of the jerk path
// (finalize of the per-slice partials, per-type reduction, layout kernels).
// Non-template kernels: included by exactly one translation unit (api_adjoint.cu).
#pragma once

#include "nbody.h"
#include "fixed_point.cuh"
#include "vjp_kernel.cuh"

namespace nbody {

// ---- O(N) kernels of the reverse sweep -------------------------------------------
struct VjpFinalizeArgs {
  const float4 *part_hi;
  const float4 *part_lo;
  long long stride;
  long long bstride;
  int slices;
  int n;
  int law;
  float G;
  float alpha;        // weight of this VJP (h or dt in the reverse sweep)
  const float4 *pos;
  const float4 *prm;
  const float4 *lam;  // gravity: lam; LJC: u
  float4 *grad_x;     // += alpha g (or = when !accumulate)
  float *grad_m;      // may be null
  int accumulate;
  double *type_part;  // [gridDim.x][8] or null
  float4 *lam_v;      // if non-null: lam_v += dt_next * grad_x afterwards
  float dt_next;
  // symmetric gravity VJP with the source split (block size, parts per block):
  // the slots a particle receives are its own part's slot of each lower block and
  // every slot from its own block on (sym_split <= 1: every slot)
  int sym_block;
  int sym_split;
  // exact fixed-point accumulators of the symmetric gravity VJP (eight int64
  // arrays of stride `stride`, see VjpArgs) and the word holding 2^-S; null: slots
  const long long *acc64;
  const double *fx_inv;
};

__global__ void __launch_bounds__(256) vjp_finalize_kernel(const VjpFinalizeArgs f) {
  griddep_start();
  const int i = blockIdx.x * 256 + threadIdx.x;
  double tv[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (i < f.n) {
    // part_lo == nullptr: partials without low parts (Newton-symmetric gravity tiles)
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 hA = zero, oA = zero, hB = zero, oB = zero;
    const bool lj = (f.law == NBODY_LAW_LJC || f.law == NBODY_LAW_LJC_LINEAR);
    const int sp = f.sym_split > 1 ? f.sym_split : 1;
    const int own_b = sp > 1 ? i / f.sym_block : 0;
    const int own_s = sp > 1 ? ((i - own_b * f.sym_block) >> 1) / (f.sym_block / 2 / sp) : 0;
    const int below = own_b;        // slots own_s, own_s + sp, ... below the own block
    const int k_all = own_b * sp;   // every slot from here on
    const int count = f.acc64 ? 0 : below + (f.slices - k_all);
    auto offset = [&](int c) {
      const int k = c < below ? c * sp + own_s : k_all + (c - below);
      return (long long)k * f.stride + i;
    };
    auto add = [&](float4 &h, float4 &o, const float4 &a, const float4 &l) {
      comp_add(h.x, o.x, a.x);
      comp_add(h.y, o.y, a.y);
      comp_add(h.z, o.z, a.z);
      comp_add(h.w, o.w, a.w);
      o.x += l.x;
      o.y += l.y;
      o.z += l.z;
      o.w += l.w;
    };
    // slots in the same order as one at a time, with the loads of eight slots
    // issued before their adds (the symmetric tiles leave dozens per particle)
    constexpr int U = 8;
    int c = 0;
    for (; c + U <= count; c += U) {
      float4 h[U], l[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const long long o = offset(c + u);
        h[u] = f.part_hi[o];
        l[u] = f.part_lo ? f.part_lo[o] : zero;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) add(hA, oA, h[u], l[u]);
      if (lj) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const long long o = f.bstride + offset(c + u);
          h[u] = f.part_hi[o];
          l[u] = f.part_lo ? f.part_lo[o] : zero;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) add(hB, oB, h[u], l[u]);
      }
    }
    for (; c < count; ++c) {
      const long long o = offset(c);
      add(hA, oA, f.part_hi[o], f.part_lo ? f.part_lo[o] : zero);
      if (lj)
        add(hB, oB, f.part_hi[f.bstride + o], f.part_lo ? f.part_lo[f.bstride + o] : zero);
    }
    float ax = hA.x + oA.x, ay = hA.y + oA.y, az = hA.z + oA.z, aw = hA.w + oA.w;
    if (f.acc64) {  // the exact sums, rounded once
      const long long st = f.stride;
      const double inv = *f.fx_inv;
      ax = float(fixed_value(f.acc64[i], f.acc64[4 * st + i], inv));
      ay = float(fixed_value(f.acc64[st + i], f.acc64[5 * st + i], inv));
      az = float(fixed_value(f.acc64[2 * st + i], f.acc64[6 * st + i], inv));
      aw = float(fixed_value(f.acc64[3 * st + i], f.acc64[7 * st + i], inv));
    }
    float gx, gy, gz, gm;
    if (!lj) {
      gx = f.G * ax;
      gy = f.G * ay;
      gz = f.G * az;
      gm = -f.G * aw;
    } else {
      const float4 x = f.pos[i];
      const float4 u = f.lam[i];
      const float bx = hB.x + oB.x, by = hB.y + oB.y, bz = hB.z + oB.z, bw = hB.w + oB.w;
      gx = ax;
      gy = ay;
      gz = az;
      gm = (u.x * bx + u.y * by + u.z * bz) / x.w;
      const float4 q = f.prm[i];
      const int t = int(q.w);
      if (f.type_part && t >= 0 && t < 4) {
        const double e2 = double(q.z) * double(q.z);  // 24 eps_k
        tv[t] = -3.0 * double(aw) * f.alpha;
        tv[4 + t] = -12.0 / e2 * double(bw) * f.alpha;
      }
    }
    float4 gxo = f.accumulate ? f.grad_x[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    gxo.x = fmaf(f.alpha, gx, gxo.x);
    gxo.y = fmaf(f.alpha, gy, gxo.y);
    gxo.z = fmaf(f.alpha, gz, gxo.z);
    gxo.w = 0.0f;
    f.grad_x[i] = gxo;
    if (f.grad_m) {
      const float gmo = f.accumulate ? f.grad_m[i] : 0.0f;
      f.grad_m[i] = fmaf(f.alpha, gm, gmo);
    }
    if (f.lam_v) {
      float4 v = f.lam_v[i];
      v.x = fmaf(f.dt_next, gxo.x, v.x);
      v.y = fmaf(f.dt_next, gxo.y, v.y);
      v.z = fmaf(f.dt_next, gxo.z, v.z);
      f.lam_v[i] = v;
    }
  }
  if (f.type_part) {
    // fixed-order block sum of the 8 per-type fields
    __shared__ double red[8][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) tv[k] += __shfl_down_sync(0xffffffffu, tv[k], off);
      if (lane == 0) red[warp][k] = tv[k];
    }
    __syncthreads();
    if (threadIdx.x < 8) {
      double s = 0.0;
      for (int w = 0; w < 8; ++w) s += red[w][threadIdx.x];
      f.type_part[(size_t)blockIdx.x * 8 + threadIdx.x] = s;
    }
  }
}

// GAJ: fixed-order compensated sum of the per-slice partials of A (acceleration)
// and B (jerk), scaled by G.
// acc64 (with inv = 2^-S): the exact fixed-point sums of the Newton-symmetric
// tiles, sixteen int64 arrays of stride `stride` (acceleration x, y, z, -, their
// fractions, then the same four and four for the jerk), rounded once; else null.
__global__ void __launch_bounds__(256) gaj_finalize_kernel(const float4 *part_hi,
                                                           const float4 *part_lo,
                                                           long long stride, long long bstride,
                                                           int slices, int n, float G,
                                                           float4 *acc, float4 *jerk,
                                                           const long long *acc64,
                                                           const double *inv) {
  const int i = blockIdx.x * 256 + threadIdx.x;
  if (i >= n) return;
  if (acc64) {
    const double iv = *inv;
    auto v = [&](int c) {
      return G * float(fixed_value(acc64[c * stride + i], acc64[(4 + c) * stride + i], iv));
    };
    auto w = [&](int c) {
      return G * float(fixed_value(acc64[(8 + c) * stride + i], acc64[(12 + c) * stride + i],
                                   iv));
    };
    acc[i] = make_float4(v(0), v(1), v(2), 0.0f);
    jerk[i] = make_float4(w(0), w(1), w(2), 0.0f);
    return;
  }
  // part_lo == nullptr: partials without low parts (Newton-symmetric tiles)
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 hA = part_hi[i], oA = part_lo ? part_lo[i] : zero;
  float4 hB = part_hi[bstride + i], oB = part_lo ? part_lo[bstride + i] : zero;
  for (int k = 1; k < slices; ++k) {
    const long long o = (long long)k * stride + i;
    const float4 a = part_hi[o], la = part_lo ? part_lo[o] : zero, b = part_hi[bstride + o],
                 lb = part_lo ? part_lo[bstride + o] : zero;
    comp_add(hA.x, oA.x, a.x);
    comp_add(hA.y, oA.y, a.y);
    comp_add(hA.z, oA.z, a.z);
    comp_add(hB.x, oB.x, b.x);
    comp_add(hB.y, oB.y, b.y);
    comp_add(hB.z, oB.z, b.z);
    oA.x += la.x;
    oA.y += la.y;
    oA.z += la.z;
    oB.x += lb.x;
    oB.y += lb.y;
    oB.z += lb.z;
  }
  acc[i] = make_float4(G * (hA.x + oA.x), G * (hA.y + oA.y), G * (hA.z + oA.z), 0.0f);
  jerk[i] = make_float4(G * (hB.x + oB.x), G * (hB.y + oB.y), G * (hB.z + oB.z), 0.0f);
}

// Sum per-block type partials in order and add them into out[0..2*ntypes).
__global__ void type_reduce_kernel(const double *part, int nblk, int ntypes, double *out) {
  griddep_start();
  const int k = threadIdx.x;
  if (k >= 8) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[(size_t)b * 8 + k];
  const int t = k & 3, which = k >> 2;  // 0: sigma, 1: eps
  if (t < ntypes) out[which * ntypes + t] += s;
}

// Fixed-point accumulation of the symmetric gravity VJP: the accumulators that
// the interleave launch zeroes, and the words from which it forms the scale.
struct VjpAtomicPrep {
  long long *acc64;  // nwords x n accumulators, or null (slots: nothing to prepare)
  double *part;      // four doubles per interleave block: sum |m|, max |m|, sum |lam|, max |lam|
  unsigned *ticket;  // zero before the launch; zero again after it
  float eps2;
  float *scale;      // out: 2^S, read by the VJP kernel
  double *inv;       // out: 2^-S, read by vjp_finalize_kernel
  int kind;          // 0: the VJP's bound (lam); 1: acceleration + jerk (lam = velocities)
  int nwords;        // int64 arrays to zero: 8 (VJP), 16 (acceleration and jerk)
};

// Scale of the VJP's fixed-point sums. With y = 1/s <= 1/eps and the matrix
// I - 3 y^2 d d^T of norm at most 2 (its eigenvalues are 1 and 1 - 3 r^2 / s^2),
// a particle's J^T lambda sum obeys |g_k| <= 2 / eps^3 (m_max L + lam_max M), and
// its mass term |sum lam_j . d y^3| <= 2 / (3 sqrt(3) eps^2) L (the maximum of
// r / s^3), with M = sum |m| and L = sum |lam_j|. Writes the largest 2^S that keeps
// both below 2^62, and 2^-S.
__device__ __forceinline__ void vjp_scale_of(double M, double mmax, double L, double lmax,
                                             float eps2, float *scale, double *inv) {
  const double e2 = double(eps2), e = sqrt(e2);
  const double bound =
      fmax(2.0 * (mmax * L + lmax * M) / (e2 * e), 0.3849001794597505 * L / e2) + 1e-300;
  int S = int(floor(62.0 - log2(bound)));
  S = S > 126 ? 126 : (S < -126 ? -126 : S);
  *scale = ldexpf(1.0f, S);
  *inv = ldexp(1.0, -S);
}

// Scale of the fixed-point sums of acceleration + jerk. With |d| / s^3 at most
// 2 / (3 sqrt(3) eps^2), u = v_j - v_i of norm at most 2 v_max and
// |u - 3 y^2 (d.u) d| <= 4 |u|, a particle's acceleration sum obeys |a| <= M 2 /
// (3 sqrt(3) eps^2) and its jerk sum |j| <= 8 v_max M / eps^3 (M = sum |m|).
// Writes the largest 2^S that keeps both below 2^62, and 2^-S.
__device__ __forceinline__ void gaj_scale_of(double M, double vmax, float eps2, float *scale,
                                             double *inv) {
  const double e2 = double(eps2), e = sqrt(e2);
  const double bound = fmax(0.3849001794597505 * M / e2, 8.0 * vmax * M / (e2 * e)) + 1e-300;
  int S = int(floor(62.0 - log2(bound)));
  S = S > 126 ? 126 : (S < -126 ? -126 : S);
  *scale = ldexpf(1.0f, S);
  *inv = ldexp(1.0, -S);
}

// Gravity VJP sources of the Newton-symmetric tiles, block by block (B
// particles, 2B float4 per block): the B/2 pairs' (x0 x1 y0 y1), then their
// (z0 z1 m0 m1), (lx0 lx1 ly0 ly1) and (lz0 lz1 0 0). Pairs past n are not written
// (the kernel copies only the block's own pairs). With at.acc64 the launch also
// zeroes its particles' accumulators and forms the fixed-point scale: every block
// reduces |m| and |lam| of its particles in FP64 in a fixed order, and the block
// that finishes last (atomicInc ticket, which wraps back to zero) combines the
// block results in index order -- the same bits whichever block is last.
__global__ void __launch_bounds__(256) interleave_vjp_pairs_blocked_kernel(
    const float4 *pos, const float4 *lam, float4 *jp, int n, int B, VjpAtomicPrep at) {
  griddep_start();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  double v[4] = {0.0, 0.0, 0.0, 0.0};  // sum |m|, max |m|, sum |lam|, max |lam|
  if (2 * p < n) {
    const bool two = 2 * p + 1 < n;
    const float4 a = pos[2 * p], la = lam[2 * p];
    const float4 b = two ? pos[2 * p + 1] : make_float4(1e18f, 1e18f, 1e18f, 0.0f);
    const float4 lb = two ? lam[2 * p + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int blk = (2 * p) / B, P = B / 2, pp = p - blk * P;
    const long long q = (long long)blk * 2 * B + pp;
    jp[q] = make_float4(a.x, b.x, a.y, b.y);
    jp[q + P] = make_float4(a.z, b.z, a.w, b.w);
    jp[q + 2 * P] = make_float4(la.x, lb.x, la.y, lb.y);
    jp[q + 3 * P] = make_float4(la.z, lb.z, 0.f, 0.f);
    if (at.acc64) {
      const double ma = fabs(double(a.w)), mb = fabs(double(b.w));
      const double na = sqrt(double(la.x) * la.x + double(la.y) * la.y + double(la.z) * la.z);
      const double nb = sqrt(double(lb.x) * lb.x + double(lb.y) * lb.y + double(lb.z) * lb.z);
      v[0] = ma + mb;
      v[1] = fmax(ma, mb);
      v[2] = na + nb;
      v[3] = fmax(na, nb);
      for (int c = 0; c < at.nwords; ++c) {
        at.acc64[(long long)c * n + 2 * p] = 0;
        if (two) at.acc64[(long long)c * n + 2 * p + 1] = 0;
      }
    }
  }
  if (!at.acc64) return;  // the same for every thread of the launch
  __shared__ double red[8][4];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  auto warp_reduce = [&](double x[4]) {
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      x[0] += __shfl_down_sync(0xffffffffu, x[0], off);
      x[1] = fmax(x[1], __shfl_down_sync(0xffffffffu, x[1], off));
      x[2] += __shfl_down_sync(0xffffffffu, x[2], off);
      x[3] = fmax(x[3], __shfl_down_sync(0xffffffffu, x[3], off));
    }
  };
  warp_reduce(v);
  if (lane == 0)
    for (int k = 0; k < 4; ++k) red[warp][k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    double bs[4] = {0.0, 0.0, 0.0, 0.0};
    for (int w = 0; w < 8; ++w) {
      bs[0] += red[w][0];
      bs[1] = fmax(bs[1], red[w][1]);
      bs[2] += red[w][2];
      bs[3] = fmax(bs[3], red[w][3]);
    }
    for (int k = 0; k < 4; ++k) at.part[4 * blockIdx.x + k] = bs[k];
    __threadfence();  // the block result is visible before the ticket is taken
    last = atomicInc(at.ticket, gridDim.x - 1) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double t[4] = {0.0, 0.0, 0.0, 0.0};
  const volatile double *part = at.part;
  for (int k = threadIdx.x; k < int(gridDim.x); k += 256) {
    t[0] += part[4 * k];
    t[1] = fmax(t[1], part[4 * k + 1]);
    t[2] += part[4 * k + 2];
    t[3] = fmax(t[3], part[4 * k + 3]);
  }
  warp_reduce(t);
  __syncthreads();
  if (lane == 0)
    for (int k = 0; k < 4; ++k) red[warp][k] = t[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    double M = 0.0, mmax = 0.0, L = 0.0, lmax = 0.0;
    for (int w = 0; w < 8; ++w) {
      M += red[w][0];
      mmax = fmax(mmax, red[w][1]);
      L += red[w][2];
      lmax = fmax(lmax, red[w][3]);
    }
    if (at.kind == 1)
      gaj_scale_of(M, lmax, at.eps2, at.scale, at.inv);
    else
      vjp_scale_of(M, mmax, L, lmax, at.eps2, at.scale, at.inv);
  }
}

// Packed gravity VJP sources: per pair (x0 x1 y0 y1)(z0 z1 m0 m1)(lx0 lx1 ly0 ly1)
// (lz0 lz1 0 0); an odd count is padded with a massless particle far away.
__global__ void interleave_vjp_pairs_kernel(const float4 *pos, const float4 *lam, float4 *jp,
                                            int n) {
  griddep_start();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (2 * p >= n) return;
  const bool two = 2 * p + 1 < n;
  const float4 a = pos[2 * p], la = lam[2 * p];
  const float4 b = two ? pos[2 * p + 1] : make_float4(1e18f, 1e18f, 1e18f, 0.0f);
  const float4 lb = two ? lam[2 * p + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
  const long long q = 4LL * p;  // 64-bit: 4p passes 2^31 for n above ~1.07e9
  jp[q] = make_float4(a.x, b.x, a.y, b.y);
  jp[q + 1] = make_float4(a.z, b.z, a.w, b.w);
  jp[q + 2] = make_float4(la.x, lb.x, la.y, lb.y);
  jp[q + 3] = make_float4(la.z, lb.z, 0.f, 0.f);
}

// LJC VJP source pairs: (x x y y)(z z q q)(s s e e)(-ux -ux -uy -uy)(-uz -uz 0 0);
// an odd count ends with an uncharged, motionless pad at 1e18 with zero LJ terms.
__global__ void interleave_ljc_vjp_pairs_kernel(const float4 *pos, const float4 *u,
                                                const float4 *prm, float4 *jp, int n) {
  griddep_start();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (2 * p >= n) return;
  const bool two = 2 * p + 1 < n;
  const float4 a = pos[2 * p], ua = u[2 * p], qa = prm[2 * p];
  const float4 b = two ? pos[2 * p + 1] : make_float4(1e18f, 1e18f, 1e18f, 0.0f);
  const float4 ub = two ? u[2 * p + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 qb = two ? prm[2 * p + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
  const long long q = 5LL * p;  // 64-bit: 5p passes 2^31 for n above ~8.6e8
  jp[q] = make_float4(a.x, b.x, a.y, b.y);
  jp[q + 1] = make_float4(a.z, b.z, qa.x, qb.x);
  jp[q + 2] = make_float4(qa.y, qb.y, qa.z, qb.z);
  jp[q + 3] = make_float4(-ua.x, -ub.x, -ua.y, -ub.y);
  jp[q + 4] = make_float4(-ua.z, -ub.z, 0.f, 0.f);
}

// LJC VJP sources of the Newton-symmetric tiles, block by block (B particles,
// 5B/2 float4 per block): the B/2 pairs' (x x y y), then (z z q q), (s s e e),
// (-ux -ux -uy -uy) and (-uz -uz 0 0). Pairs past n are not written.
__global__ void interleave_ljc_vjp_pairs_blocked_kernel(const float4 *pos, const float4 *u,
                                                        const float4 *prm, float4 *jp, int n,
                                                        int B) {
  griddep_start();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (2 * p >= n) return;
  const bool two = 2 * p + 1 < n;
  const float4 a = pos[2 * p], ua = u[2 * p], qa = prm[2 * p];
  const float4 b = two ? pos[2 * p + 1] : make_float4(1e18f, 1e18f, 1e18f, 0.0f);
  const float4 ub = two ? u[2 * p + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 qb = two ? prm[2 * p + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
  const int blk = (2 * p) / B, P = B / 2, pp = p - blk * P;
  const long long q = (long long)blk * 5 * P + pp;
  jp[q] = make_float4(a.x, b.x, a.y, b.y);
  jp[q + P] = make_float4(a.z, b.z, qa.x, qb.x);
  jp[q + 2 * P] = make_float4(qa.y, qb.y, qa.z, qb.z);
  jp[q + 3 * P] = make_float4(-ua.x, -ub.x, -ua.y, -ub.y);
  jp[q + 4 * P] = make_float4(-ua.z, -ub.z, 0.f, 0.f);
}

// u = lam / m (LJC sources are weighted by 1 / m_j).
__global__ void lam_over_m_kernel(const float4 *lam, const float4 *pos, float4 *u, int n) {
  griddep_start();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 l = lam[i];
  const float inv = 1.0f / pos[i].w;
  u[i] = make_float4(l.x * inv, l.y * inv, l.z * inv, 0.0f);
}

// y += alpha * x on float4 xyz.
__global__ void axpy4_kernel(float alpha, const float4 *x, float4 *y, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 a = x[i];
  float4 b = y[i];
  b.x = fmaf(alpha, a.x, b.x);
  b.y = fmaf(alpha, a.y, b.y);
  b.z = fmaf(alpha, a.z, b.z);
  y[i] = b;
}

__global__ void zero_doubles_kernel(double *p, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = 0.0;
}

}  // namespace nbody
