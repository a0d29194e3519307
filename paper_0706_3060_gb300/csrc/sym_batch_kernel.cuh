// sym_batch_kernel.cuh -- batched ensembles (many independent systems of mixed
// law and uneven size) with each unordered pair of a system evaluated once and
// applied to both particles.
//
// The work list holds one item per block pair (bi <= bj) of each system, blocks
// of B = NT * I particles; persistent CTAs take items from an atomic counter,
// longest first. An item stages source block bj of its system with TMA bulk
// copies from the law's blocked pair buffer (gravity: (x x y y), (z z m m);
// LJC: (x x y y), (z z q q), (s s e e)), holds the targets of block bi in
// registers, and runs the pair schedule of sym_kernel.cuh (gravity) or
// sym_ljc_kernel.cuh (LJC, constant or linear dielectric): a diagonal item
// (bi == bj) one-sided with the self pair masked, an off-diagonal item adding
// the target-side sums to slot bj of its targets and the source-side sums to
// slot bi of its sources. WorkItem.slice carries bj in its low 16 bits and bi in
// the high bits. The finalize kernel adds each system's slots in index order.
#pragma once

#include "force_kernel.cuh"
#include "sym_kernel.cuh"
#include "sym_ljc_kernel.cuh"

namespace nbody {

template <int NT, int I>
struct SymMixedTile {
  static constexpr int kB = NT * I;
  static constexpr int kPairs = kB / 2;
  static constexpr int kWarps = NT / 32;
  static constexpr size_t kSrcBytes = size_t(kPairs) * 48;  // room for the LJC layout
  static constexpr size_t kSmemBytes = kSrcBytes + size_t(kWarps) * 6 * kPairs * sizeof(float);
};

// Gravity pair against one target (halves = two sources), target side only or
// both sides; the source side gets m_i y^3 d before its sign change.
template <bool PRECISE, bool JS, bool MASK>
__device__ __forceinline__ void sym_grav_pair2(float2 X, float2 Y, float2 Z, float2 M,
                                               float2 nx, float2 ny, float2 nz, float2 mi,
                                               float2 e2, float2 &ax, float2 &ay, float2 &az,
                                               float2 &jx, float2 &jy, float2 &jz,
                                               bool self0 = false, bool self1 = false) {
  const float2 dx = __fadd2_rn(X, nx);
  const float2 dy = __fadd2_rn(Y, ny);
  const float2 dz = __fadd2_rn(Z, nz);
  float2 s2 = __ffma2_rn(dz, dz, e2);
  s2 = __ffma2_rn(dy, dy, s2);
  s2 = __ffma2_rn(dx, dx, s2);
  float2 y = make_float2(rsqrt_hw(s2.x), rsqrt_hw(s2.y));
  if (PRECISE) {
    const float2 hs = __fmul2_rn(s2, make_float2(-0.5f, -0.5f));
    y = __fmul2_rn(y, __ffma2_rn(hs, __fmul2_rn(y, y), make_float2(1.5f, 1.5f)));
  }
  if (MASK) {
    y.x = self0 ? 0.0f : y.x;
    y.y = self1 ? 0.0f : y.y;
  }
  const float2 y3 = __fmul2_rn(__fmul2_rn(y, y), y);
  const float2 wi = __fmul2_rn(M, y3);
  ax = __ffma2_rn(wi, dx, ax);
  ay = __ffma2_rn(wi, dy, ay);
  az = __ffma2_rn(wi, dz, az);
  if (JS) {
    const float2 wj = __fmul2_rn(mi, y3);
    jx = __ffma2_rn(wj, dx, jx);
    jy = __ffma2_rn(wj, dy, jy);
    jz = __ffma2_rn(wj, dz, jz);
  }
}

// One work item of law LAW. Returns false when the wait for the source block ran
// out (the error word is set; the whole CTA leaves).
template <int LAW, int NT, int I, bool PRECISE>
__device__ __forceinline__ bool sym_batch_item(const ForceArgs &a, const WorkItem &w,
                                               float4 *src, float *jsum, uint64_t *bar,
                                               uint32_t phase) {
  using T = SymMixedTile<NT, I>;
  constexpr int P = T::kPairs;
  constexpr bool LJ = (LAW != kLawGrav);
  constexpr bool LIN = (LAW == kLawLJCLin);
  constexpr int NF4 = LJ ? 3 : 2;  // source arrays per block
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int bj = w.slice & 0xffff, bi = w.slice >> 16;
  const bool diag = (bi == bj);
  const int npairs = (w.nj + 1) >> 1;  // an odd system ends with its pad particle
  if (tid == 0) {
    const uint32_t bytes = uint32_t(npairs) * 16u;
    const float4 *blk = (LJ ? a.jpair2 : a.jpair) + size_t(w.pj0);
    mbar_arrive_expect_tx(bar, NF4 * bytes);
#pragma unroll
    for (int c = 0; c < NF4; ++c) tma_load_1d(src + c * P, blk + c * P, bytes, bar);
  }
  if (!diag)
    for (int k = tid; k < T::kWarps * 6 * P; k += NT) jsum[k] = 0.0f;

  float2 nx[I], ny[I], nz[I], t0[I], t1[I], t2[I], ax[I], ay[I], az[I];
  int ig[I];
#pragma unroll
  for (int r = 0; r < I; ++r) {
    const int il = r * NT + tid;
    const int g = w.i0 + min(il, w.ni - 1);
    ig[r] = il < w.ni ? g : -1;
    const float4 p = il < w.ni ? __ldg(a.pos + g) : make_float4(1e18f, 1e18f, 1e18f, 0.0f);
    nx[r] = make_float2(-p.x, -p.x);
    ny[r] = make_float2(-p.y, -p.y);
    nz[r] = make_float2(-p.z, -p.z);
    if (LJ) {
      const float4 q = il < w.ni ? __ldg(a.prm + g) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      t0[r] = make_float2(q.x, q.x);
      t1[r] = make_float2(q.y, q.y);
      t2[r] = make_float2(q.z, q.z);
    } else {
      t0[r] = make_float2(p.w, p.w);
      t1[r] = t2[r] = make_float2(0.0f, 0.0f);
    }
    ax[r] = ay[r] = az[r] = make_float2(0.0f, 0.0f);
  }
  __syncthreads();  // jsum cleared
  const bool ok = mbar_wait(bar, phase, a.err);
  if (!__syncthreads_and(ok)) {  // a copy may still be landing: bounded drain, then leave
    if (tid == 0) mbar_wait(bar, phase, a.err);
    return false;
  }
  const float4 *s0 = src, *s1 = src + P, *s2 = src + 2 * P;
  const float2 e2 = make_float2(w.eps2, w.eps2);
  float2 dummy = make_float2(0.0f, 0.0f);

  if (diag) {
    for (int pp = 0; pp < npairs; ++pp) {
      const float4 A = s0[pp], Bq = s1[pp];
      const int jg = w.j0 + 2 * pp;
      if (LJ) {
        const float4 C = s2[pp];
#pragma unroll
        for (int r = 0; r < I; ++r)
          ljc_pair2<false, PRECISE, LIN, true>(
              make_float2(A.x, A.y), make_float2(A.z, A.w), make_float2(Bq.x, Bq.y),
              make_float2(Bq.z, Bq.w), make_float2(C.x, C.y), make_float2(C.z, C.w), nx[r],
              ny[r], nz[r], t0[r], t1[r], t2[r], ax[r], ay[r], az[r], dummy, jg == ig[r],
              jg + 1 == ig[r]);
      } else {
#pragma unroll
        for (int r = 0; r < I; ++r)
          sym_grav_pair2<PRECISE, false, true>(
              make_float2(A.x, A.y), make_float2(A.z, A.w), make_float2(Bq.x, Bq.y),
              make_float2(Bq.z, Bq.w), nx[r], ny[r], nz[r], t0[r], e2, ax[r], ay[r], az[r],
              dummy, dummy, dummy, jg == ig[r], jg + 1 == ig[r]);
      }
    }
  } else {
    float *J = jsum + size_t(warp) * 6 * P;
    for (int g0 = 0; g0 < npairs; g0 += 32) {
#pragma unroll 1
      for (int st = 0; st < 32; ++st) {
        const int pp = g0 + ((lane + st) & 31);
        if (pp < npairs) {
          const float4 A = s0[pp], Bq = s1[pp];
          const float2 X = make_float2(A.x, A.y), Y = make_float2(A.z, A.w);
          const float2 Z = make_float2(Bq.x, Bq.y), W = make_float2(Bq.z, Bq.w);
          float2 jx = make_float2(0.0f, 0.0f), jy = jx, jz = jx;
          if (LJ) {
            const float4 C = s2[pp];
            const float2 S = make_float2(C.x, C.y), E = make_float2(C.z, C.w);
#pragma unroll
            for (int r = 0; r < I; ++r)
              sym_ljc_pair2<false, PRECISE, LIN>(X, Y, Z, W, S, E, nx[r], ny[r], nz[r], t0[r],
                                                 t1[r], t2[r], ax[r], ay[r], az[r], dummy, jx,
                                                 jy, jz, dummy);
          } else {
#pragma unroll
            for (int r = 0; r < I; ++r)
              sym_grav_pair2<PRECISE, true, false>(X, Y, Z, W, nx[r], ny[r], nz[r], t0[r], e2,
                                                   ax[r], ay[r], az[r], jx, jy, jz);
          }
          // the sources feel the opposite force
          J[0 * P + pp] -= jx.x;
          J[1 * P + pp] -= jx.y;
          J[2 * P + pp] -= jy.x;
          J[3 * P + pp] -= jy.y;
          J[4 * P + pp] -= jz.x;
          J[5 * P + pp] -= jz.y;
        }
        __syncwarp();  // at the next step lane l - 1 updates the slot lane l just wrote
      }
    }
  }

  const long long ibase = (long long)bj * a.stride;
#pragma unroll
  for (int r = 0; r < I; ++r)
    if (ig[r] >= 0)
      a.part_hi[ibase + ig[r]] =
          make_float4(ax[r].x + ax[r].y, ay[r].x + ay[r].y, az[r].x + az[r].y, 0.0f);
  if (!diag) {
    __syncthreads();
    const long long jbase = (long long)bi * a.stride + w.j0;
    for (int q = tid; q < w.nj; q += NT) {
      const int pp = q >> 1, h = q & 1;
      float vx = 0.0f, vy = 0.0f, vz = 0.0f;
      for (int wp = 0; wp < T::kWarps; ++wp) {
        const float *Jw = jsum + size_t(wp) * 6 * P;
        vx += Jw[(0 + h) * P + pp];
        vy += Jw[(2 + h) * P + pp];
        vz += Jw[(4 + h) * P + pp];
      }
      a.part_hi[jbase + q] = make_float4(vx, vy, vz, 0.0f);
    }
  }
  return true;
}

template <int NT, int I, bool PRECISE, int MINB = 1>
__global__ void __launch_bounds__(NT, MINB) sym_batch_kernel(const ForceArgs a) {
  griddep_start();
  using T = SymMixedTile<NT, I>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float4 *src = reinterpret_cast<float4 *>(smem_raw);
  float *jsum = reinterpret_cast<float *>(smem_raw + T::kSrcBytes);
  __shared__ __align__(8) uint64_t bar;
  __shared__ int s_item;
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  uint32_t phase = 0;
  for (;;) {
    __syncthreads();  // the previous item is done with s_item and shared memory
    if (tid == 0) s_item = atomicAdd(a.counter, 1);
    __syncthreads();
    const int k = s_item;
    if (k >= a.n_items) break;
    const WorkItem w = a.items[k];
    const int bj = w.slice & 0xffff, bi = w.slice >> 16;
    if (w.ni <= 0 || w.ni > T::kB || w.nj <= 0 || w.nj > T::kB || w.i0 < 0 || w.j0 < 0 ||
        bi > bj || (w.law != kLawGrav && w.law != kLawLJC && w.law != kLawLJCLin)) {
      if (tid == 0) set_error(a.err, kDevBadItem);
      continue;
    }
    bool ok;
    if (w.law == kLawGrav)
      ok = sym_batch_item<kLawGrav, NT, I, PRECISE>(a, w, src, jsum, &bar, phase);
    else if (w.law == kLawLJC)
      ok = sym_batch_item<kLawLJC, NT, I, PRECISE>(a, w, src, jsum, &bar, phase);
    else
      ok = sym_batch_item<kLawLJCLin, NT, I, PRECISE>(a, w, src, jsum, &bar, phase);
    if (!ok) return;
    phase ^= 1u;
  }
}

}  // namespace nbody
