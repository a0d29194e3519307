// sym_ljc_kernel.cuh -- Lennard-Jones plus Coulomb forces (Table 1, LJC constant
// and linear dielectric) with each unordered pair evaluated once and applied to
// both particles.
//
// The pair function f(r) of force_kernel.cuh depends on the pair only through
// q~_i q~_j, s~_i + s~_j and e~_i e~_j, all symmetric, so the force of j on i,
// f d (d = x_j - x_i), and that of i on j, -f d, come from one evaluation, and
// so does the pair energy, which both particles count. The partial sums hold
// sum f d (the finalize kernel turns them into -sum f d / m). Per unordered
// pair: 26 FP32 lane ops (27 for the linear dielectric) against 23 (24) per
// ordered pair one-sided.
//
// Blocks, block pairs, the per-block partial slots, the source split (S parts
// per block at small N), the rotating lane schedule of the source-side sums and
// the diagonal blocks (one-sided, self pair masked) follow sym_kernel.cuh.
// Sources come in the blocked layout of
// interleave_ljc_pairs_blocked_kernel: per block of B particles the B/2 pairs'
// (x x y y), then (z z q q), then (s s e e) words.
#pragma once

#include <type_traits>

#include "force_kernel.cuh"
#include "sym_kernel.cuh"

namespace nbody {

template <int NT, int I>
struct SymLjcTile {
  static constexpr int kB = NT * I;
  static constexpr int kPairs = kB / 2;
  static constexpr int kWarps = NT / 32;
  static constexpr size_t kSrcBytes = size_t(kPairs) * 48;  // three float4 per pair
  static constexpr size_t smem_bytes(bool pot) {
    return kSrcBytes + size_t(kWarps) * (pot ? 8 : 6) * kPairs * sizeof(float);
  }
};

// One target against one source pair (halves = the two sources): adds f d to the
// target's (ax, ay, az) and to the sources' (jx, jy, jz) (negated when stored),
// and with POT the pair energy to both aw and jw.
template <bool POT, bool PRECISE, bool LIN>
__device__ __forceinline__ void sym_ljc_pair2(float2 X, float2 Y, float2 Z, float2 Q, float2 S,
                                              float2 E, float2 nxi, float2 nyi, float2 nzi,
                                              float2 qi, float2 si, float2 ei, float2 &ax,
                                              float2 &ay, float2 &az, float2 &aw, float2 &jx,
                                              float2 &jy, float2 &jz, float2 &jw) {
  const float2 dx = __fadd2_rn(X, nxi);
  const float2 dy = __fadd2_rn(Y, nyi);
  const float2 dz = __fadd2_rn(Z, nzi);
  float2 r2 = __fmul2_rn(dz, dz);
  r2 = __ffma2_rn(dy, dy, r2);
  r2 = __ffma2_rn(dx, dx, r2);
  float2 y = make_float2(rsqrt_hw(r2.x), rsqrt_hw(r2.y));
  if (PRECISE) {
    const float2 hs = __fmul2_rn(r2, make_float2(-0.5f, -0.5f));
    y = __fmul2_rn(y, __ffma2_rn(hs, __fmul2_rn(y, y), make_float2(1.5f, 1.5f)));
  }
  const float2 y2 = __fmul2_rn(y, y);
  const float2 qq = __fmul2_rn(Q, qi);
  const float2 s = __fadd2_rn(S, si);
  const float2 t = __fmul2_rn(__fmul2_rn(s, s), y2);
  const float2 u = __fmul2_rn(__fmul2_rn(t, t), t);
  const float2 ee = __fmul2_rn(E, ei);
  const float2 fc = LIN ? __fmul2_rn(__fmul2_rn(qq, y2), __fadd2_rn(y2, y2))
                        : __fmul2_rn(__fmul2_rn(qq, y), y2);
  const float2 h = __fmul2_rn(__ffma2_rn(u, make_float2(2.0f, 2.0f), make_float2(-1.0f, -1.0f)), u);
  const float2 f = __ffma2_rn(__fmul2_rn(ee, y2), h, fc);
  ax = __ffma2_rn(f, dx, ax);
  ay = __ffma2_rn(f, dy, ay);
  az = __ffma2_rn(f, dz, az);
  jx = __ffma2_rn(f, dx, jx);
  jy = __ffma2_rn(f, dy, jy);
  jz = __ffma2_rn(f, dz, jz);
  if (POT) {
    float2 e = __fmul2_rn(qq, LIN ? y2 : y);
    e = __ffma2_rn(__fmul2_rn(ee, make_float2(1.0f / 6.0f, 1.0f / 6.0f)),
                   __ffma2_rn(u, u, make_float2(-u.x, -u.y)), e);
    aw = __fadd2_rn(aw, e);
    jw = __fadd2_rn(jw, e);
  }
}

template <int LAW, int NT, int I, bool POT, bool PRECISE, int MINB = 1>
__global__ void __launch_bounds__(NT, MINB) sym_ljc_kernel(const ForceArgs a) {
  griddep_start();
  static_assert(LAW == kLawLJC || LAW == kLawLJCLin, "LJC laws only");
  constexpr bool LIN = (LAW == kLawLJCLin);
  using T = SymLjcTile<NT, I>;
  constexpr int B = T::kB;
  constexpr int P = T::kPairs;
  constexpr int NC = POT ? 8 : 6;  // source-side float components per source pair
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float4 *s0 = reinterpret_cast<float4 *>(smem_raw);  // (x x y y)
  float4 *s1 = s0 + P;                                 // (z z q q)
  float4 *s2 = s1 + P;                                 // (s s e e)
  float *jsum = reinterpret_cast<float *>(smem_raw + T::kSrcBytes);
  __shared__ __align__(8) uint64_t bar;
  __shared__ int part_meta[3];  // (parts per block, part, first pair), read after the loop

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = a.n;
  const int nparts = B / a.slice_len;  // source parts per block
  const int nb = a.slices / nparts;
  const int t = int(blockIdx.x) / nparts, sp = int(blockIdx.x) - t * nparts;
  int bi, bj;
  sym_tile_of(t, nb, bi, bj);
  if (bj >= nb) {  // outside the triangle: a launch-shape error
    if (tid == 0) set_error(a.err, kDevBadItem);
    return;
  }
  const int j0 = bj * B;
  const int nsrc = min(B, n - j0);
  const int p0 = sp * (P / nparts);  // first source pair of this part
  const int npairs = max(0, min(P / nparts, ((nsrc + 1) >> 1) - p0));
  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
    part_meta[0] = nparts;  // kept in shared memory, not in registers, across the loop
    part_meta[1] = sp;
    part_meta[2] = p0;
  }
  __syncthreads();
  if (tid == 0) {
    const uint32_t bytes = uint32_t(npairs) * 16u;
    const float4 *blk = a.jpair + size_t(bj) * 3 * P + p0;  // three arrays of P per block
    mbar_arrive_expect_tx(&bar, 3 * bytes);
    if (npairs > 0) {
      tma_load_1d(s0, blk, bytes, &bar);
      tma_load_1d(s1, blk + P, bytes, &bar);
      tma_load_1d(s2, blk + 2 * P, bytes, &bar);
    }
  }
  const bool diag = (bi == bj);
  if (!diag)
    for (int k = tid; k < T::kWarps * NC * P; k += NT) jsum[k] = 0.0f;

  // targets of block bi; missing ones are uncharged, far away, without an LJ well
  float2 nx[I], ny[I], nz[I], qi[I], si[I], ei[I], ax[I], ay[I], az[I], aw[I];
  int ig[I];
#pragma unroll
  for (int r = 0; r < I; ++r) {
    const int g = bi * B + r * NT + tid;
    ig[r] = g < n ? g : -1;
    const float4 p = g < n ? __ldg(a.pos + g) : make_float4(1e18f, 1e18f, 1e18f, 0.0f);
    const float4 q = g < n ? __ldg(a.prm + g) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    nx[r] = make_float2(-p.x, -p.x);
    ny[r] = make_float2(-p.y, -p.y);
    nz[r] = make_float2(-p.z, -p.z);
    qi[r] = make_float2(q.x, q.x);
    si[r] = make_float2(q.y, q.y);
    ei[r] = make_float2(q.z, q.z);
    ax[r] = ay[r] = az[r] = aw[r] = make_float2(0.0f, 0.0f);
  }
  __syncthreads();  // jsum cleared
  const bool ok = mbar_wait(&bar, 0, a.err);
  if (!__syncthreads_and(ok)) {  // a copy may still be landing: bounded drain, then leave
    if (tid == 0) mbar_wait(&bar, 0, a.err);
    return;
  }

  if (diag) {
    for (int pp = 0; pp < npairs; ++pp) {
      const float4 A = s0[pp], Bq = s1[pp], C = s2[pp];
      const int jg = j0 + 2 * (p0 + pp);
#pragma unroll
      for (int r = 0; r < I; ++r)
        ljc_pair2<POT, PRECISE, LIN, true>(
            make_float2(A.x, A.y), make_float2(A.z, A.w), make_float2(Bq.x, Bq.y),
            make_float2(Bq.z, Bq.w), make_float2(C.x, C.y), make_float2(C.z, C.w), nx[r],
            ny[r], nz[r], qi[r], si[r], ei[r], ax[r], ay[r], az[r], aw[r], jg == ig[r],
            jg + 1 == ig[r]);
    }
  } else {
    // this warp's source-side sums: one float2 (both halves of a source pair) per
    // component and pair, added with one packed read-modify-write per component;
    // they hold +sum f d (negated when the warps are added) and +sum of energies
    float2 *J = reinterpret_cast<float2 *>(jsum) + size_t(warp) * (NC / 2) * P;
    for (int g0 = 0; g0 < npairs; g0 += 32) {
#pragma unroll 1
      for (int st = 0; st < 32; ++st) {
        const int pp = g0 + ((lane + st) & 31);
        if (pp < npairs) {
          const float4 A = s0[pp], Bq = s1[pp], C = s2[pp];
          const float2 X = make_float2(A.x, A.y), Y = make_float2(A.z, A.w);
          const float2 Z = make_float2(Bq.x, Bq.y), Q = make_float2(Bq.z, Bq.w);
          const float2 S = make_float2(C.x, C.y), E = make_float2(C.z, C.w);
          float2 jx = make_float2(0.0f, 0.0f), jy = jx, jz = jx, jw = jx;
#pragma unroll
          for (int r = 0; r < I; ++r)
            sym_ljc_pair2<POT, PRECISE, LIN>(X, Y, Z, Q, S, E, nx[r], ny[r], nz[r], qi[r], si[r],
                                             ei[r], ax[r], ay[r], az[r], aw[r], jx, jy, jz, jw);
          J[0 * P + pp] = __fadd2_rn(J[0 * P + pp], jx);
          J[1 * P + pp] = __fadd2_rn(J[1 * P + pp], jy);
          J[2 * P + pp] = __fadd2_rn(J[2 * P + pp], jz);
          if (POT) J[3 * P + pp] = __fadd2_rn(J[3 * P + pp], jw);
        }
        __syncwarp();  // at the next step lane l - 1 updates the slot lane l just wrote
      }
    }
  }

  const int np_ = part_meta[0], s_ = part_meta[1], p0_ = part_meta[2];
  const long long ibase = (long long)(bj * np_ + s_) * a.stride;
#pragma unroll
  for (int r = 0; r < I; ++r)
    if (ig[r] >= 0)
      a.part_hi[ibase + ig[r]] = make_float4(ax[r].x + ax[r].y, ay[r].x + ay[r].y,
                                             az[r].x + az[r].y, aw[r].x + aw[r].y);
  if (diag) return;
  __syncthreads();
  const long long jbase = (long long)(bi * np_ + s_) * a.stride + j0 + 2 * p0_;
  const int nq = min(2 * npairs, nsrc - 2 * p0_);
  for (int q = tid; q < nq; q += NT) {
    const int pp = q >> 1, h = q & 1;
    float vx = 0.0f, vy = 0.0f, vz = 0.0f, vw = 0.0f;
    for (int w = 0; w < T::kWarps; ++w) {
      const float *Jw = jsum + size_t(w) * NC * P;  // float view of the float2 sums
      vx += Jw[2 * (0 * P + pp) + h];
      vy += Jw[2 * (1 * P + pp) + h];
      vz += Jw[2 * (2 * P + pp) + h];
      if (POT) vw += Jw[2 * (3 * P + pp) + h];
    }
    // the sources feel -f d; the pair energy counts for both
    a.part_hi[jbase + q] = make_float4(-vx, -vy, -vz, vw);
  }
}

}  // namespace nbody
