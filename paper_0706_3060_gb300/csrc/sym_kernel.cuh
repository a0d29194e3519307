// sym_kernel.cuh -- softened gravity (Eq. 1) with each unordered pair evaluated
// once and applied to both particles (Newton's third law).
//
// The paper's kernels evaluate every ordered pair (i, j) and use no symmetry.
// Here the particles are cut into blocks of B = NT * I, and one CTA handles one
// block pair (bi, bj) with bi <= bj:
//   * targets of block bi sit in registers, I per thread (packed f32x2 math over
//     source pairs as in force_kernel.cuh); the sources of block bj are loaded
//     into shared memory with two 1-D TMA bulk copies, the (x x y y) words of
//     its pairs and then their (z z m m) words (the blocked layout written by
//     interleave_pairs_blocked_kernel), so that lanes reading consecutive pairs
//     read consecutive 16-byte words without bank conflicts;
//   * for bi < bj every pair term m y^3 d is added to the target (i side) and,
//     with the target's mass, subtracted for the source (j side). The j side
//     needs a sum over all targets for each source: at step s of a group of 32
//     source pairs, lane l takes pair (l + s) mod 32, so the 32 lanes of a warp
//     work on distinct sources and add their sums (over the lane's I targets) to
//     distinct shared-memory slots, one slot set per warp, without atomics or
//     shuffles;
//   * for bi == bj the block is summed one-sided over all ordered pairs, the self
//     pair dropped by index.
// Every particle p of block b receives one partial per block ob: from the
// diagonal tile when ob == b, from the i side of tile (b, ob) when ob > b and
// from the j side of tile (ob, b) when ob < b. Partial ob goes to slot ob of
// part_hi; the finalize kernel adds the slots in index order (compensated), so
// the result is bitwise reproducible. Per-tile sums are plain FP32 over B terms.
// Source split (small N, more CTAs than block pairs): each block's B/2 source
// pairs are cut into S equal parts, a.slice_len = B / S sources each, and CTA
// t * S + s takes part s of block pair t. Its target-side partial goes to slot
// bj * S + s, its source-side partial to slot bi * S + s, so a particle of block
// b and part s_p receives every slot k with k / S >= b and, below that, those with
// k % S == s_p; the finalize kernel skips the rest. S = 1 is the plain scheme.
// Atomic accumulation (a.acc64 set; gravity with eps > 0, Sec. 3.2's GRAPE-6
// scheme): each partial, scaled by 2^S (S from *a.fscale, chosen from an a-priori
// bound on every sum), is added with integer atomics as an integer part and a
// fraction in units of 2^-32 into two int64 words per component and particle;
// integer addition is associative, so the result does not depend on the order of
// the CTAs, and the scratch is 64 bytes per particle instead of one partial per
// particle and block.
// FX without a.acc64: each partial is stored as four int64 in its slot, (x, y)
// in part_hi and (z, w) in part_lo, which the finalize adds as integers.
#pragma once

#include <cmath>

#include "fixed_point.cuh"
#include "force_kernel.cuh"

namespace nbody {

template <int NT, int I>
struct SymTile {
  static constexpr int kB = NT * I;          // particles per block
  static constexpr int kPairs = kB / 2;      // source pairs per block
  static constexpr int kWarps = NT / 32;
  static constexpr size_t kSrcBytes = size_t(kPairs) * 32;  // (x x y y), (z z m m) per pair
  // j-side sums per warp: components x, y, z (and w with the potential) of
  // both halves of every source pair
  static constexpr size_t smem_bytes(bool pot) {
    return kSrcBytes + size_t(kWarps) * (pot ? 8 : 6) * kPairs * sizeof(float);
  }
};

// Block pair (bi, bj), bi <= bj < nb, of the t-th CTA in row-major order of the
// upper triangle: row bi starts at bi * nb - bi (bi - 1) / 2.
__device__ __forceinline__ void sym_tile_of(long long t, int nb, int &bi, int &bj) {
  const double a = 2.0 * nb + 1.0;
  int b = int((a - sqrt(a * a - 8.0 * double(t))) * 0.5);
  b = max(0, min(b, nb - 1));
  auto start = [nb](long long r) { return r * nb - r * (r - 1) / 2; };
  while (b > 0 && start(b) > t) --b;
  while (b + 1 < nb && start(b + 1) <= t) ++b;
  bi = b;
  bj = b + int(t - start(b));
}

// Store one partial of `particle`: with a.acc64, add it, rounded onto the 64-bit
// fixed-point grid, to the particle's accumulator with integer atomics (exact,
// so the order in which CTAs arrive does not change the sum); otherwise write it
// to element `particle` of the slot starting at `slot_base` (FP32, or four int64
// with FX).
template <bool FX, bool POT>
__device__ __forceinline__ void sym_store(const ForceArgs &a, long long slot_base, int particle,
                                          float x, float y, float z, float w) {
  if (a.acc64) {
    const float sc = __ldg(a.fscale);
    unsigned long long *p = reinterpret_cast<unsigned long long *>(a.acc64) + particle;
    fixed_add(p, a.stride, 0, x, sc);
    fixed_add(p, a.stride, 1, y, sc);
    fixed_add(p, a.stride, 2, z, sc);
    if (POT) fixed_add(p, a.stride, 3, w, sc);
    return;
  }
  const long long idx = slot_base + particle;
  if constexpr (FX) {
    const float sc = __ldg(a.fscale);
    long long *ph = reinterpret_cast<long long *>(a.part_hi) + 2 * idx;
    long long *pl = reinterpret_cast<long long *>(a.part_lo) + 2 * idx;
    ph[0] = __float2ll_rn(x * sc);
    ph[1] = __float2ll_rn(y * sc);
    pl[0] = __float2ll_rn(z * sc);
    pl[1] = __float2ll_rn(w * sc);
  } else {
    a.part_hi[idx] = make_float4(x, y, z, w);
  }
}

template <int NT, int I, bool POT, bool PRECISE, int MINB = 1, bool FX = false>
__global__ void __launch_bounds__(NT, MINB) sym_grav_kernel(const ForceArgs a) {
  griddep_start();
  using T = SymTile<NT, I>;
  constexpr int B = T::kB;
  constexpr int NC = POT ? 8 : 6;  // j-side float components per source pair
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float4 *src0 = reinterpret_cast<float4 *>(smem_raw);  // (x x y y) of each pair
  float4 *src1 = src0 + T::kPairs;                       // (z z m m) of each pair
  float *jsum = reinterpret_cast<float *>(smem_raw + T::kSrcBytes);
  __shared__ __align__(8) uint64_t bar;
  __shared__ int part_meta[3];  // (parts per block, part, first pair), read after the loop

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = a.n;
  const int nparts = B / a.slice_len;  // source parts per block
  const int nb = a.slices / nparts;
  const int t = int(blockIdx.x) / nparts, s = int(blockIdx.x) - t * nparts;
  int bi, bj;
  sym_tile_of(t, nb, bi, bj);
  if (bj >= nb) {  // outside the triangle: a launch-shape error
    if (tid == 0) set_error(a.err, kDevBadItem);
    return;
  }
  const int j0 = bj * B;
  const int nsrc = min(B, n - j0);
  const int p0 = s * (T::kPairs / nparts);  // first source pair of this part
  // an odd count ends with the pad particle; the last block's late parts may be empty
  const int npairs = max(0, min(T::kPairs / nparts, ((nsrc + 1) >> 1) - p0));
  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
    part_meta[0] = nparts;  // kept in shared memory, not in registers, across the loop
    part_meta[1] = s;
    part_meta[2] = p0;
  }
  __syncthreads();
  if (tid == 0) {
    const uint32_t bytes = uint32_t(npairs) * 16u;
    const float4 *blk = a.jpair + size_t(bj) * B + p0;  // blocked layout: B float4 per block
    mbar_arrive_expect_tx(&bar, 2 * bytes);
    if (npairs > 0) {
      tma_load_1d(src0, blk, bytes, &bar);
      tma_load_1d(src1, blk + T::kPairs, bytes, &bar);
    }
  }
  const bool diag = (bi == bj);
  if (!diag)
    for (int k = tid; k < T::kWarps * NC * T::kPairs; k += NT) jsum[k] = 0.0f;

  // targets: block bi, I per thread; missing ones are massless and far away
  float2 nx[I], ny[I], nz[I], mi[I], ax[I], ay[I], az[I], aw[I];
  int ig[I];
#pragma unroll
  for (int r = 0; r < I; ++r) {
    const int g = bi * B + r * NT + tid;
    ig[r] = g < n ? g : -1;
    const float4 p = g < n ? __ldg(a.pos + g) : make_float4(1e18f, 1e18f, 1e18f, 0.0f);
    nx[r] = make_float2(-p.x, -p.x);
    ny[r] = make_float2(-p.y, -p.y);
    nz[r] = make_float2(-p.z, -p.z);
    mi[r] = make_float2(p.w, p.w);
    ax[r] = ay[r] = az[r] = aw[r] = make_float2(0.0f, 0.0f);
  }
  __syncthreads();  // jsum cleared
  // bounded wait for the source block; the CTA leaves together if any wait ran out
  const bool ok = mbar_wait(&bar, 0, a.err);
  if (!__syncthreads_and(ok)) {  // a copy may still be landing: bounded drain, then leave
    if (tid == 0) mbar_wait(&bar, 0, a.err);
    return;
  }
  const float2 e2 = make_float2(a.eps2, a.eps2);

  if (diag) {
    // one-sided over all ordered pairs of the block, self pair dropped
    for (int pp = 0; pp < npairs; ++pp) {
      const float4 A = src0[pp], Bq = src1[pp];
      const int jg = j0 + 2 * (p0 + pp);
#pragma unroll
      for (int r = 0; r < I; ++r)
        grav_pair2<POT, PRECISE, true>(make_float2(A.x, A.y), make_float2(A.z, A.w),
                                       make_float2(Bq.x, Bq.y), make_float2(Bq.z, Bq.w), nx[r],
                                       ny[r], nz[r], e2, ax[r], ay[r], az[r], aw[r], jg == ig[r],
                                       jg + 1 == ig[r]);
    }
  } else {
    float *J = jsum + size_t(warp) * NC * T::kPairs;
    for (int g0 = 0; g0 < npairs; g0 += 32) {
#pragma unroll 2
      for (int st = 0; st < 32; ++st) {
        const int pp = g0 + ((lane + st) & 31);
        if (pp < npairs) {
          const float4 A = src0[pp], Bq = src1[pp];
          const float2 X = make_float2(A.x, A.y), Y = make_float2(A.z, A.w);
          const float2 Z = make_float2(Bq.x, Bq.y), M = make_float2(Bq.z, Bq.w);
          float2 jx = make_float2(0.0f, 0.0f), jy = jx, jz = jx, jw = jx;
#pragma unroll
          for (int r = 0; r < I; ++r) {
            const float2 dx = __fadd2_rn(X, nx[r]);
            const float2 dy = __fadd2_rn(Y, ny[r]);
            const float2 dz = __fadd2_rn(Z, nz[r]);
            float2 s2 = __ffma2_rn(dz, dz, e2);
            s2 = __ffma2_rn(dy, dy, s2);
            s2 = __ffma2_rn(dx, dx, s2);
            float2 y = make_float2(rsqrt_hw(s2.x), rsqrt_hw(s2.y));
            if (PRECISE) {
              const float2 hs = __fmul2_rn(s2, make_float2(-0.5f, -0.5f));
              y = __fmul2_rn(y, __ffma2_rn(hs, __fmul2_rn(y, y), make_float2(1.5f, 1.5f)));
            }
            const float2 y3 = __fmul2_rn(__fmul2_rn(y, y), y);
            const float2 wi = __fmul2_rn(M, y3);      // source mass: pull on the target
            const float2 wj = __fmul2_rn(mi[r], y3);  // target mass: pull on the source
            ax[r] = __ffma2_rn(wi, dx, ax[r]);
            ay[r] = __ffma2_rn(wi, dy, ay[r]);
            az[r] = __ffma2_rn(wi, dz, az[r]);
            jx = __ffma2_rn(wj, dx, jx);
            jy = __ffma2_rn(wj, dy, jy);
            jz = __ffma2_rn(wj, dz, jz);
            if (POT) {
              aw[r] = __ffma2_rn(M, y, aw[r]);
              jw = __ffma2_rn(mi[r], y, jw);
            }
          }
          // d points from the target to the source: the source feels -d
          J[0 * T::kPairs + pp] -= jx.x;
          J[1 * T::kPairs + pp] -= jx.y;
          J[2 * T::kPairs + pp] -= jy.x;
          J[3 * T::kPairs + pp] -= jy.y;
          J[4 * T::kPairs + pp] -= jz.x;
          J[5 * T::kPairs + pp] -= jz.y;
          if (POT) {
            J[6 * T::kPairs + pp] += jw.x;
            J[7 * T::kPairs + pp] += jw.y;
          }
        }
        __syncwarp();  // at the next step lane l - 1 updates the slot lane l just wrote
      }
    }
  }

  // i side: slot bj (part s) of every target of block bi
  const int np_ = part_meta[0], s_ = part_meta[1], p0_ = part_meta[2];
  const long long ibase = (long long)(bj * np_ + s_) * a.stride;
#pragma unroll
  for (int r = 0; r < I; ++r)
    if (ig[r] >= 0)
      sym_store<FX, POT>(a, ibase, ig[r], ax[r].x + ax[r].y, ay[r].x + ay[r].y,
                         az[r].x + az[r].y, aw[r].x + aw[r].y);
  if (diag) return;
  // j side: slot bi (part s) of every source of the part, warps added in index order
  __syncthreads();
  const long long jbase = (long long)(bi * np_ + s_) * a.stride;
  const int jfirst = j0 + 2 * p0_;
  const int nq = min(2 * npairs, nsrc - 2 * p0_);
  for (int q = tid; q < nq; q += NT) {
    const int pp = q >> 1, h = q & 1;
    float vx = 0.0f, vy = 0.0f, vz = 0.0f, vw = 0.0f;
    for (int w = 0; w < T::kWarps; ++w) {
      const float *Jw = jsum + size_t(w) * NC * T::kPairs;
      vx += Jw[(0 + h) * T::kPairs + pp];
      vy += Jw[(2 + h) * T::kPairs + pp];
      vz += Jw[(4 + h) * T::kPairs + pp];
      if (POT) vw += Jw[(6 + h) * T::kPairs + pp];
    }
    sym_store<FX, POT>(a, jbase, jfirst + q, vx, vy, vz, vw);
  }
}

}  // namespace nbody
