// sym_vjp_kernel.cuh -- gravity force VJP (J^T lambda and the mass derivative)
// and acceleration + jerk (Table 1 "Gravity (accel & jerk)"), each with every
// unordered pair evaluated once and applied to both particles.
//
// For target k and source j (d = x_j - x_k, y = 1/s, w = m_k lam_j - m_j lam_k)
// the J^T lambda term y^3 [w - 3 y^2 (d.w) d] changes sign when k and j swap
// (d and w both do), so the source receives the negated term. The mass term
// (lam_j . d) y^3 of the target becomes (lam_k . (-d)) y^3 for the source. With
// ldj = lam_j . d and ldk = lam_k . d, d.w = m_k ldj - m_j ldk, so the pair costs
// 35 FP32 lane ops for both particles (29 for one in vjp_kernel.cuh).
//
// Blocks, block pairs, the per-block partial slots, the rotating lane schedule
// of the source-side sums and the diagonal blocks (one-sided, self pair masked)
// follow sym_kernel.cuh. Sources come in the blocked layout of
// interleave_vjp_pairs_blocked_kernel: per block of B particles the B/2 pairs'
// (x x y y), then (z z m m), (lx lx ly ly) and (lz lz 0 0) words.
#pragma once

#include "fixed_point.cuh"
#include "sym_kernel.cuh"
#include "vjp_kernel.cuh"

namespace nbody {

template <int NT, int I>
struct SymVjpTile {
  static constexpr int kB = NT * I;
  static constexpr int kPairs = kB / 2;
  static constexpr int kWarps = NT / 32;
  static constexpr size_t kSrcBytes = size_t(kPairs) * 64;  // four float4 per pair
  // source-side sums per warp: g.x, g.y, g.z and the mass term of both halves
  static constexpr size_t kSmemBytes = kSrcBytes + size_t(kWarps) * 8 * kPairs * sizeof(float);
};

// One target against one source pair (the halves of the f32x2 values are the
// two sources). nM = -m_j. Adds the target's terms to (ax, ay, az, aw); with JS
// also adds the terms the sources receive, before their sign change, to
// (jx, jy, jz, jw). MASK drops a source half equal to the target (y = 0).
template <bool JS, bool MASK>
__device__ __forceinline__ void sym_gvjp_pair2(float2 X, float2 Y, float2 Z, float2 nM,
                                               float2 LX, float2 LY, float2 LZ, float2 nx,
                                               float2 ny, float2 nz, float2 mk, float2 lkx,
                                               float2 lky, float2 lkz, float2 e2, float2 &ax,
                                               float2 &ay, float2 &az, float2 &aw, float2 &jx,
                                               float2 &jy, float2 &jz, float2 &jw,
                                               bool self0 = false, bool self1 = false) {
  const float2 dx = __fadd2_rn(X, nx);
  const float2 dy = __fadd2_rn(Y, ny);
  const float2 dz = __fadd2_rn(Z, nz);
  float2 s2 = __ffma2_rn(dz, dz, e2);
  s2 = __ffma2_rn(dy, dy, s2);
  s2 = __ffma2_rn(dx, dx, s2);
  float2 y = make_float2(rsqrt_hw(s2.x), rsqrt_hw(s2.y));
  if (MASK) {
    y.x = self0 ? 0.0f : y.x;
    y.y = self1 ? 0.0f : y.y;
  }
  const float2 y2 = __fmul2_rn(y, y);
  const float2 y3 = __fmul2_rn(y2, y);
  const float2 wx = __ffma2_rn(mk, LX, __fmul2_rn(nM, lkx));
  const float2 wy = __ffma2_rn(mk, LY, __fmul2_rn(nM, lky));
  const float2 wz = __ffma2_rn(mk, LZ, __fmul2_rn(nM, lkz));
  const float2 ldj = __ffma2_rn(LX, dx, __ffma2_rn(LY, dy, __fmul2_rn(LZ, dz)));
  const float2 ldk = __ffma2_rn(lkx, dx, __ffma2_rn(lky, dy, __fmul2_rn(lkz, dz)));
  const float2 dw = __ffma2_rn(mk, ldj, __fmul2_rn(nM, ldk));
  const float2 c = __fmul2_rn(dw, __fmul2_rn(y2, make_float2(-3.0f, -3.0f)));
  const float2 vx = __ffma2_rn(c, dx, wx);
  const float2 vy = __ffma2_rn(c, dy, wy);
  const float2 vz = __ffma2_rn(c, dz, wz);
  ax = __ffma2_rn(y3, vx, ax);
  ay = __ffma2_rn(y3, vy, ay);
  az = __ffma2_rn(y3, vz, az);
  aw = __ffma2_rn(ldj, y3, aw);
  if (JS) {
    jx = __ffma2_rn(y3, vx, jx);
    jy = __ffma2_rn(y3, vy, jy);
    jz = __ffma2_rn(y3, vz, jz);
    jw = __ffma2_rn(ldk, y3, jw);
  }
}

// One particle's (g.x, g.y, g.z, mass term) partial of one CTA: added exactly in
// fixed point to the particle's accumulator (a.acc64), or stored to element
// `particle` of the slot that starts at slot_base.
__device__ __forceinline__ void vjp_store(const VjpArgs &a, long long slot_base, int particle,
                                          float x, float y, float z, float w) {
  if (a.acc64) {
    const float sc = __ldg(a.fscale);
    unsigned long long *p = reinterpret_cast<unsigned long long *>(a.acc64) + particle;
    fixed_add(p, a.stride, 0, x, sc);
    fixed_add(p, a.stride, 1, y, sc);
    fixed_add(p, a.stride, 2, z, sc);
    fixed_add(p, a.stride, 3, w, sc);
    return;
  }
  a.part_hi[slot_base + particle] = make_float4(x, y, z, w);
}

// Partials: slot ob of part_hi holds (g.x, g.y, g.z, mass term) of block ob's
// contribution, before the G scaling of vjp_finalize_kernel; with a.acc64 every
// CTA adds its partials to the particles' fixed-point accumulators instead.
template <int NT, int I, int MINB = 1>
__global__ void __launch_bounds__(NT, MINB) sym_gvjp_kernel(const VjpArgs a) {
  griddep_start();
  using T = SymVjpTile<NT, I>;
  constexpr int B = T::kB;
  constexpr int P = T::kPairs;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float4 *s0 = reinterpret_cast<float4 *>(smem_raw);  // (x x y y)
  float4 *s1 = s0 + P;                                 // (z z m m)
  float4 *s2 = s1 + P;                                 // (lx lx ly ly)
  float4 *s3 = s2 + P;                                 // (lz lz 0 0)
  float *jsum = reinterpret_cast<float *>(smem_raw + T::kSrcBytes);
  __shared__ __align__(8) uint64_t bar;
  __shared__ int part_meta[3];  // (parts per block, part, first pair), read after the loop

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = a.n;
  // source split as in sym_kernel.cuh: a.slice_len sources per part
  const int nparts = B / a.slice_len;
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
    part_meta[0] = nparts;
    part_meta[1] = sp;
    part_meta[2] = p0;
  }
  __syncthreads();
  if (tid == 0) {
    const uint32_t bytes = uint32_t(npairs) * 16u;
    const float4 *blk = a.jpair + size_t(bj) * 2 * B + p0;  // four arrays of P per block
    mbar_arrive_expect_tx(&bar, 4 * bytes);
    if (npairs > 0) {
      tma_load_1d(s0, blk, bytes, &bar);
      tma_load_1d(s1, blk + P, bytes, &bar);
      tma_load_1d(s2, blk + 2 * P, bytes, &bar);
      tma_load_1d(s3, blk + 3 * P, bytes, &bar);
    }
  }
  const bool diag = (bi == bj);
  if (!diag)
    for (int k = tid; k < T::kWarps * 8 * P; k += NT) jsum[k] = 0.0f;

  // targets of block bi; missing ones are massless, far away and carry no lambda
  float2 nx[I], ny[I], nz[I], mk[I], lkx[I], lky[I], lkz[I], ax[I], ay[I], az[I], aw[I];
  int ig[I];
#pragma unroll
  for (int r = 0; r < I; ++r) {
    const int g = bi * B + r * NT + tid;
    ig[r] = g < n ? g : -1;
    const float4 p = g < n ? __ldg(a.pos + g) : make_float4(1e18f, 1e18f, 1e18f, 0.0f);
    const float4 l = g < n ? __ldg(a.lam + g) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    nx[r] = make_float2(-p.x, -p.x);
    ny[r] = make_float2(-p.y, -p.y);
    nz[r] = make_float2(-p.z, -p.z);
    mk[r] = make_float2(p.w, p.w);
    lkx[r] = make_float2(l.x, l.x);
    lky[r] = make_float2(l.y, l.y);
    lkz[r] = make_float2(l.z, l.z);
    ax[r] = ay[r] = az[r] = aw[r] = make_float2(0.0f, 0.0f);
  }
  __syncthreads();  // jsum cleared
  const bool ok = mbar_wait(&bar, 0, a.err);
  if (!__syncthreads_and(ok)) {  // a copy may still be landing: bounded drain, then leave
    if (tid == 0) mbar_wait(&bar, 0, a.err);
    return;
  }
  const float2 e2 = make_float2(a.eps2, a.eps2);

  if (diag) {
    float2 dummy = make_float2(0.0f, 0.0f);
    for (int pp = 0; pp < npairs; ++pp) {
      const float4 A = s0[pp], Bq = s1[pp], C = s2[pp], D = s3[pp];
      const float2 nM = make_float2(-Bq.z, -Bq.w);
      const int jg = j0 + 2 * (p0 + pp);
#pragma unroll
      for (int r = 0; r < I; ++r)
        sym_gvjp_pair2<false, true>(make_float2(A.x, A.y), make_float2(A.z, A.w),
                                    make_float2(Bq.x, Bq.y), nM, make_float2(C.x, C.y),
                                    make_float2(C.z, C.w), make_float2(D.x, D.y), nx[r], ny[r],
                                    nz[r], mk[r], lkx[r], lky[r], lkz[r], e2, ax[r], ay[r], az[r],
                                    aw[r], dummy, dummy, dummy, dummy, jg == ig[r],
                                    jg + 1 == ig[r]);
    }
  } else {
    // this warp's source-side sums: one float2 (both halves of a source pair) per
    // component and pair, one packed read-modify-write per component; they hold
    // the terms before the sources' sign change (negated when the warps are added)
    float2 *J = reinterpret_cast<float2 *>(jsum) + size_t(warp) * 4 * P;
    for (int g0 = 0; g0 < npairs; g0 += 32) {
#pragma unroll 1
      for (int st = 0; st < 32; ++st) {
        const int pp = g0 + ((lane + st) & 31);
        if (pp < npairs) {
          const float4 A = s0[pp], Bq = s1[pp], C = s2[pp], D = s3[pp];
          const float2 X = make_float2(A.x, A.y), Y = make_float2(A.z, A.w);
          const float2 Z = make_float2(Bq.x, Bq.y), nM = make_float2(-Bq.z, -Bq.w);
          const float2 LX = make_float2(C.x, C.y), LY = make_float2(C.z, C.w);
          const float2 LZ = make_float2(D.x, D.y);
          float2 jx = make_float2(0.0f, 0.0f), jy = jx, jz = jx, jw = jx;
#pragma unroll
          for (int r = 0; r < I; ++r)
            sym_gvjp_pair2<true, false>(X, Y, Z, nM, LX, LY, LZ, nx[r], ny[r], nz[r], mk[r],
                                        lkx[r], lky[r], lkz[r], e2, ax[r], ay[r], az[r], aw[r],
                                        jx, jy, jz, jw);
          J[0 * P + pp] = __fadd2_rn(J[0 * P + pp], jx);
          J[1 * P + pp] = __fadd2_rn(J[1 * P + pp], jy);
          J[2 * P + pp] = __fadd2_rn(J[2 * P + pp], jz);
          J[3 * P + pp] = __fadd2_rn(J[3 * P + pp], jw);
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
      vjp_store(a, ibase, ig[r], ax[r].x + ax[r].y, ay[r].x + ay[r].y, az[r].x + az[r].y,
                aw[r].x + aw[r].y);
  if (diag) return;
  __syncthreads();
  const long long jbase = (long long)(bi * np_ + s_) * a.stride;
  const int jfirst = j0 + 2 * p0_;
  const int nq = min(2 * npairs, nsrc - 2 * p0_);
  for (int q = tid; q < nq; q += NT) {
    const int pp = q >> 1, h = q & 1;
    float vx = 0.0f, vy = 0.0f, vz = 0.0f, vw = 0.0f;
    for (int w = 0; w < T::kWarps; ++w) {
      const float *Jw = jsum + size_t(w) * 8 * P;  // float view of the float2 sums
      vx += Jw[2 * (0 * P + pp) + h];
      vy += Jw[2 * (1 * P + pp) + h];
      vz += Jw[2 * (2 * P + pp) + h];
      vw += Jw[2 * (3 * P + pp) + h];
    }
    // the sources receive the negated terms
    vjp_store(a, jbase, jfirst + q, -vx, -vy, -vz, -vw);
  }
}

// Acceleration + jerk. For target i and source j (d = x_j - x_i, u = v_j - v_i,
// y = 1/s, c = -3 y^2 (d.u)) the target gets m_j y^3 d and m_j y^3 (u + c d);
// swapping the pair flips d and u and keeps c, so the source gets -m_i y^3 d and
// -m_i y^3 (u + c d): 33 FP32 lane ops per unordered pair against 26 per ordered
// pair one-sided. Sources in the four-array blocked layout with velocities in
// place of lambda; partial block A holds the accelerations, block B (bstride
// further) the jerks.
template <int NT, int I>
struct SymGajTile {
  static constexpr int kB = NT * I;
  static constexpr int kPairs = kB / 2;
  static constexpr int kWarps = NT / 32;
  static constexpr size_t kSrcBytes = size_t(kPairs) * 64;
  // source-side sums per warp: a and jerk components of both halves
  static constexpr size_t kSmemBytes = kSrcBytes + size_t(kWarps) * 12 * kPairs * sizeof(float);
};

template <bool JS, bool MASK>
__device__ __forceinline__ void sym_gaj_pair2(float2 X, float2 Y, float2 Z, float2 M, float2 VX,
                                              float2 VY, float2 VZ, float2 nx, float2 ny,
                                              float2 nz, float2 nvx, float2 nvy, float2 nvz,
                                              float2 mi, float2 e2, float2 &ax, float2 &ay,
                                              float2 &az, float2 &bx, float2 &by, float2 &bz,
                                              float2 *J, bool self0 = false,
                                              bool self1 = false) {
  const float2 dx = __fadd2_rn(X, nx);
  const float2 dy = __fadd2_rn(Y, ny);
  const float2 dz = __fadd2_rn(Z, nz);
  const float2 ux = __fadd2_rn(VX, nvx);
  const float2 uy = __fadd2_rn(VY, nvy);
  const float2 uz = __fadd2_rn(VZ, nvz);
  float2 s2 = __ffma2_rn(dz, dz, e2);
  s2 = __ffma2_rn(dy, dy, s2);
  s2 = __ffma2_rn(dx, dx, s2);
  float2 y = make_float2(rsqrt_hw(s2.x), rsqrt_hw(s2.y));
  if (MASK) {
    y.x = self0 ? 0.0f : y.x;
    y.y = self1 ? 0.0f : y.y;
  }
  const float2 y2 = __fmul2_rn(y, y);
  const float2 y3 = __fmul2_rn(y2, y);
  const float2 wi = __fmul2_rn(M, y3);
  const float2 du = __ffma2_rn(dx, ux, __ffma2_rn(dy, uy, __fmul2_rn(dz, uz)));
  const float2 c = __fmul2_rn(du, __fmul2_rn(y2, make_float2(-3.0f, -3.0f)));
  const float2 tx = __ffma2_rn(c, dx, ux);
  const float2 ty = __ffma2_rn(c, dy, uy);
  const float2 tz = __ffma2_rn(c, dz, uz);
  ax = __ffma2_rn(wi, dx, ax);
  ay = __ffma2_rn(wi, dy, ay);
  az = __ffma2_rn(wi, dz, az);
  bx = __ffma2_rn(wi, tx, bx);
  by = __ffma2_rn(wi, ty, by);
  bz = __ffma2_rn(wi, tz, bz);
  if (JS) {  // J[0..5]: source-side a and jerk before their sign change
    const float2 wj = __fmul2_rn(mi, y3);
    J[0] = __ffma2_rn(wj, dx, J[0]);
    J[1] = __ffma2_rn(wj, dy, J[1]);
    J[2] = __ffma2_rn(wj, dz, J[2]);
    J[3] = __ffma2_rn(wj, tx, J[3]);
    J[4] = __ffma2_rn(wj, ty, J[4]);
    J[5] = __ffma2_rn(wj, tz, J[5]);
  }
}

// One particle's acceleration and jerk partial of one CTA: added exactly in fixed
// point (a.acc64: eight int64 arrays for the acceleration, eight more for the
// jerk, each set laid out as in fixed_add), or stored to element `particle` of
// the slot at slot_base of partial blocks A (acceleration) and B (jerk).
__device__ __forceinline__ void gaj_store(const VjpArgs &a, long long slot_base, int particle,
                                          float ax, float ay, float az, float jx, float jy,
                                          float jz) {
  if (a.acc64) {
    const float sc = __ldg(a.fscale);
    const long long st = a.stride;
    unsigned long long *pa = reinterpret_cast<unsigned long long *>(a.acc64) + particle;
    unsigned long long *pj = pa + 8 * st;
    fixed_add(pa, st, 0, ax, sc);
    fixed_add(pa, st, 1, ay, sc);
    fixed_add(pa, st, 2, az, sc);
    fixed_add(pj, st, 0, jx, sc);
    fixed_add(pj, st, 1, jy, sc);
    fixed_add(pj, st, 2, jz, sc);
    return;
  }
  a.part_hi[slot_base + particle] = make_float4(ax, ay, az, 0.0f);
  a.part_hi[a.bstride + slot_base + particle] = make_float4(jx, jy, jz, 0.0f);
}

template <int NT, int I, int MINB = 1>
__global__ void __launch_bounds__(NT, MINB) sym_gaj_kernel(const VjpArgs a) {
  griddep_start();
  using T = SymGajTile<NT, I>;
  constexpr int B = T::kB;
  constexpr int P = T::kPairs;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float4 *s0 = reinterpret_cast<float4 *>(smem_raw);  // (x x y y)
  float4 *s1 = s0 + P;                                 // (z z m m)
  float4 *s2 = s1 + P;                                 // (vx vx vy vy)
  float4 *s3 = s2 + P;                                 // (vz vz 0 0)
  float *jsum = reinterpret_cast<float *>(smem_raw + T::kSrcBytes);
  __shared__ __align__(8) uint64_t bar;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = a.n;
  const int nb = a.slices;
  int bi, bj;
  sym_tile_of(blockIdx.x, nb, bi, bj);
  if (bj >= nb) {  // outside the triangle: a launch-shape error
    if (tid == 0) set_error(a.err, kDevBadItem);
    return;
  }
  const int j0 = bj * B;
  const int nsrc = min(B, n - j0);
  const int npairs = (nsrc + 1) >> 1;
  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (tid == 0) {
    const uint32_t bytes = uint32_t(npairs) * 16u;
    const float4 *blk = a.jpair + size_t(bj) * 2 * B;
    mbar_arrive_expect_tx(&bar, 4 * bytes);
    tma_load_1d(s0, blk, bytes, &bar);
    tma_load_1d(s1, blk + P, bytes, &bar);
    tma_load_1d(s2, blk + 2 * P, bytes, &bar);
    tma_load_1d(s3, blk + 3 * P, bytes, &bar);
  }
  const bool diag = (bi == bj);
  if (!diag)
    for (int k = tid; k < T::kWarps * 12 * P; k += NT) jsum[k] = 0.0f;

  // targets of block bi (a.lam holds the velocities); missing ones are massless
  float2 nx[I], ny[I], nz[I], nvx[I], nvy[I], nvz[I], mi[I];
  float2 ax[I], ay[I], az[I], bx[I], by[I], bz[I];
  int ig[I];
#pragma unroll
  for (int r = 0; r < I; ++r) {
    const int g = bi * B + r * NT + tid;
    ig[r] = g < n ? g : -1;
    const float4 p = g < n ? __ldg(a.pos + g) : make_float4(1e18f, 1e18f, 1e18f, 0.0f);
    const float4 v = g < n ? __ldg(a.lam + g) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    nx[r] = make_float2(-p.x, -p.x);
    ny[r] = make_float2(-p.y, -p.y);
    nz[r] = make_float2(-p.z, -p.z);
    nvx[r] = make_float2(-v.x, -v.x);
    nvy[r] = make_float2(-v.y, -v.y);
    nvz[r] = make_float2(-v.z, -v.z);
    mi[r] = make_float2(p.w, p.w);
    ax[r] = ay[r] = az[r] = bx[r] = by[r] = bz[r] = make_float2(0.0f, 0.0f);
  }
  __syncthreads();  // jsum cleared
  const bool ok = mbar_wait(&bar, 0, a.err);
  if (!__syncthreads_and(ok)) {  // a copy may still be landing: bounded drain, then leave
    if (tid == 0) mbar_wait(&bar, 0, a.err);
    return;
  }
  const float2 e2 = make_float2(a.eps2, a.eps2);

  if (diag) {
    for (int pp = 0; pp < npairs; ++pp) {
      const float4 A = s0[pp], Bq = s1[pp], C = s2[pp], D = s3[pp];
      const int jg = j0 + 2 * pp;
#pragma unroll
      for (int r = 0; r < I; ++r)
        sym_gaj_pair2<false, true>(make_float2(A.x, A.y), make_float2(A.z, A.w),
                                   make_float2(Bq.x, Bq.y), make_float2(Bq.z, Bq.w),
                                   make_float2(C.x, C.y), make_float2(C.z, C.w),
                                   make_float2(D.x, D.y), nx[r], ny[r], nz[r], nvx[r], nvy[r],
                                   nvz[r], mi[r], e2, ax[r], ay[r], az[r], bx[r], by[r], bz[r],
                                   nullptr, jg == ig[r], jg + 1 == ig[r]);
    }
  } else {
    float *J = jsum + size_t(warp) * 12 * P;
    for (int g0 = 0; g0 < npairs; g0 += 32) {
#pragma unroll 1
      for (int st = 0; st < 32; ++st) {
        const int pp = g0 + ((lane + st) & 31);
        if (pp < npairs) {
          const float4 A = s0[pp], Bq = s1[pp], C = s2[pp], D = s3[pp];
          const float2 X = make_float2(A.x, A.y), Y = make_float2(A.z, A.w);
          const float2 Z = make_float2(Bq.x, Bq.y), M = make_float2(Bq.z, Bq.w);
          const float2 VX = make_float2(C.x, C.y), VY = make_float2(C.z, C.w);
          const float2 VZ = make_float2(D.x, D.y);
          float2 js[6];
#pragma unroll
          for (int c = 0; c < 6; ++c) js[c] = make_float2(0.0f, 0.0f);
#pragma unroll
          for (int r = 0; r < I; ++r)
            sym_gaj_pair2<true, false>(X, Y, Z, M, VX, VY, VZ, nx[r], ny[r], nz[r], nvx[r],
                                       nvy[r], nvz[r], mi[r], e2, ax[r], ay[r], az[r], bx[r],
                                       by[r], bz[r], js);
          // the sources receive the negated terms
#pragma unroll
          for (int c = 0; c < 6; ++c) {
            J[(2 * c) * P + pp] -= js[c].x;
            J[(2 * c + 1) * P + pp] -= js[c].y;
          }
        }
        __syncwarp();  // at the next step lane l - 1 updates the slot lane l just wrote
      }
    }
  }

  const long long ibase = (long long)bj * a.stride;
#pragma unroll
  for (int r = 0; r < I; ++r)
    if (ig[r] >= 0)
      gaj_store(a, ibase, ig[r], ax[r].x + ax[r].y, ay[r].x + ay[r].y, az[r].x + az[r].y,
                bx[r].x + bx[r].y, by[r].x + by[r].y, bz[r].x + bz[r].y);
  if (diag) return;
  __syncthreads();
  const long long jbase = (long long)bi * a.stride;
  for (int q = tid; q < nsrc; q += NT) {
    const int pp = q >> 1, h = q & 1;
    float v[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    for (int w = 0; w < T::kWarps; ++w) {
      const float *Jw = jsum + size_t(w) * 12 * P;
#pragma unroll
      for (int c = 0; c < 6; ++c) v[c] += Jw[(2 * c + h) * P + pp];
    }
    gaj_store(a, jbase, j0 + q, v[0], v[1], v[2], v[3], v[4], v[5]);
  }
}

// LJC VJP (constant or linear dielectric). With u = lam / m, w = u_k - u_j and the
// pair quantities of vjp_kernel.cuh (phi, 2 phi' = tp, c = tp (d.w)), target k
// gets g += c d + phi w, F += phi d, D += (d.w) e~e~ y^2 (4 u6^2 - u6) / sigma and
// E += (d.w) phi_lj. Swapping the pair flips d and w and keeps d.w, phi and tp,
// so the source gets -(c d + phi w) and -phi d and the same D and E terms:
// 59 FP32 lane ops per unordered pair against 48 (49) per ordered pair one-sided.
// Sources in a five-array blocked layout (x x y y), (z z q q), (s s e e),
// (-ux -ux -uy -uy), (-uz -uz 0 0); partial block A holds (g, D), block B (F, E).
template <int NT, int I>
struct SymLjcVjpTile {
  static constexpr int kB = NT * I;
  static constexpr int kPairs = kB / 2;
  static constexpr int kWarps = NT / 32;
  static constexpr size_t kSrcBytes = size_t(kPairs) * 80;  // five float4 per pair
  // source-side sums per warp: g, D, F, E components of both halves
  static constexpr size_t kSmemBytes = kSrcBytes + size_t(kWarps) * 16 * kPairs * sizeof(float);
};

// One target against one source pair. J (JS) receives the source-side terms in
// the order g.x, g.y, g.z, D, F.x, F.y, F.z, E, before the sign change of g and F.
template <bool LIN, bool JS, bool MASK>
__device__ __forceinline__ void sym_ljc_vjp_pair2(const float4 F0, const float4 F1,
                                                  const float4 F2, const float4 F3,
                                                  const float4 F4, float2 nxk, float2 nyk,
                                                  float2 nzk, float2 ukx, float2 uky, float2 ukz,
                                                  float2 qk, float2 sk, float2 ek,
                                                  float2 (&A)[4], float2 (&B)[4], float2 *J,
                                                  bool self0 = false, bool self1 = false) {
  const float2 dx = __fadd2_rn(make_float2(F0.x, F0.y), nxk);
  const float2 dy = __fadd2_rn(make_float2(F0.z, F0.w), nyk);
  const float2 dz = __fadd2_rn(make_float2(F1.x, F1.y), nzk);
  const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
  float2 y = make_float2(rsqrt_hw(r2.x), rsqrt_hw(r2.y));
  if (MASK) {
    y.x = self0 ? 0.0f : y.x;
    y.y = self1 ? 0.0f : y.y;
  }
  const float2 y2 = __fmul2_rn(y, y);
  const float2 qq = __fmul2_rn(qk, make_float2(F1.z, F1.w));
  const float2 s = __fadd2_rn(sk, make_float2(F2.x, F2.y));
  const float2 ee = __fmul2_rn(ek, make_float2(F2.z, F2.w));
  const float2 t = __fmul2_rn(__fmul2_rn(s, s), y2);
  const float2 u = __fmul2_rn(__fmul2_rn(t, t), t);
  const float2 qy3 = LIN ? __fmul2_rn(__fmul2_rn(qq, y2), __fadd2_rn(y2, y2))
                         : __fmul2_rn(qq, __fmul2_rn(y, y2));
  const float2 eey2 = __fmul2_rn(ee, y2);
  const float2 h = __fmul2_rn(__ffma2_rn(u, make_float2(2.0f, 2.0f), make_float2(-1.0f, -1.0f)), u);
  const float2 phi_lj = __fmul2_rn(eey2, h);
  const float2 phi = __fadd2_rn(phi_lj, qy3);
  const float2 k1 =
      __fmul2_rn(__ffma2_rn(u, make_float2(-28.0f, -28.0f), make_float2(8.0f, 8.0f)), u);
  const float kc = LIN ? -4.0f : -3.0f;
  const float2 tp = __fmul2_rn(y2, __ffma2_rn(eey2, k1, __fmul2_rn(make_float2(kc, kc), qy3)));
  const float2 wx = __fadd2_rn(ukx, make_float2(F3.x, F3.y));
  const float2 wy = __fadd2_rn(uky, make_float2(F3.z, F3.w));
  const float2 wz = __fadd2_rn(ukz, make_float2(F4.x, F4.y));
  const float2 dw = __ffma2_rn(dx, wx, __ffma2_rn(dy, wy, __fmul2_rn(dz, wz)));
  const float2 c = __fmul2_rn(tp, dw);
  const float2 k2 = __fmul2_rn(__ffma2_rn(u, make_float2(4.0f, 4.0f), make_float2(-1.0f, -1.0f)), u);
  const float2 rs = make_float2(rcp_hw(s.x), rcp_hw(s.y));
  const float2 dterm = __fmul2_rn(dw, __fmul2_rn(__fmul2_rn(eey2, k2), rs));
  const float2 eterm = __fmul2_rn(dw, phi_lj);
  A[0] = __ffma2_rn(c, dx, __ffma2_rn(phi, wx, A[0]));
  A[1] = __ffma2_rn(c, dy, __ffma2_rn(phi, wy, A[1]));
  A[2] = __ffma2_rn(c, dz, __ffma2_rn(phi, wz, A[2]));
  A[3] = __fadd2_rn(A[3], dterm);
  B[0] = __ffma2_rn(phi, dx, B[0]);
  B[1] = __ffma2_rn(phi, dy, B[1]);
  B[2] = __ffma2_rn(phi, dz, B[2]);
  B[3] = __fadd2_rn(B[3], eterm);
  if (JS) {
    J[0] = __ffma2_rn(c, dx, __ffma2_rn(phi, wx, J[0]));
    J[1] = __ffma2_rn(c, dy, __ffma2_rn(phi, wy, J[1]));
    J[2] = __ffma2_rn(c, dz, __ffma2_rn(phi, wz, J[2]));
    J[3] = __fadd2_rn(J[3], dterm);
    J[4] = __ffma2_rn(phi, dx, J[4]);
    J[5] = __ffma2_rn(phi, dy, J[5]);
    J[6] = __ffma2_rn(phi, dz, J[6]);
    J[7] = __fadd2_rn(J[7], eterm);
  }
}

template <int NT, int I, bool LIN, int MINB = 1>
__global__ void __launch_bounds__(NT, MINB) sym_ljc_vjp_kernel(const VjpArgs a) {
  griddep_start();
  using T = SymLjcVjpTile<NT, I>;
  constexpr int B = T::kB;
  constexpr int P = T::kPairs;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float4 *src = reinterpret_cast<float4 *>(smem_raw);  // five arrays of P float4
  float *jsum = reinterpret_cast<float *>(smem_raw + T::kSrcBytes);
  __shared__ __align__(8) uint64_t bar;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = a.n;
  const int nb = a.slices;
  int bi, bj;
  sym_tile_of(blockIdx.x, nb, bi, bj);
  if (bj >= nb) {  // outside the triangle: a launch-shape error
    if (tid == 0) set_error(a.err, kDevBadItem);
    return;
  }
  const int j0 = bj * B;
  const int nsrc = min(B, n - j0);
  const int npairs = (nsrc + 1) >> 1;
  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (tid == 0) {
    const uint32_t bytes = uint32_t(npairs) * 16u;
    const float4 *blk = a.jpair + size_t(bj) * 5 * P;
    mbar_arrive_expect_tx(&bar, 5 * bytes);
#pragma unroll
    for (int c = 0; c < 5; ++c) tma_load_1d(src + c * P, blk + c * P, bytes, &bar);
  }
  const bool diag = (bi == bj);
  if (!diag)
    for (int k = tid; k < T::kWarps * 16 * P; k += NT) jsum[k] = 0.0f;

  // targets of block bi (a.lam holds u = lam / m); missing ones have no charge, well or u
  float2 nx[I], ny[I], nz[I], ux[I], uy[I], uz[I], qk[I], sk[I], ek[I];
  float2 A[I][4], Bv[I][4];
  int ig[I];
#pragma unroll
  for (int r = 0; r < I; ++r) {
    const int g = bi * B + r * NT + tid;
    ig[r] = g < n ? g : -1;
    const float4 p = g < n ? __ldg(a.pos + g) : make_float4(1e18f, 1e18f, 1e18f, 0.0f);
    const float4 l = g < n ? __ldg(a.lam + g) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    const float4 q = g < n ? __ldg(a.prm + g) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    nx[r] = make_float2(-p.x, -p.x);
    ny[r] = make_float2(-p.y, -p.y);
    nz[r] = make_float2(-p.z, -p.z);
    ux[r] = make_float2(l.x, l.x);
    uy[r] = make_float2(l.y, l.y);
    uz[r] = make_float2(l.z, l.z);
    qk[r] = make_float2(q.x, q.x);
    sk[r] = make_float2(q.y, q.y);
    ek[r] = make_float2(q.z, q.z);
#pragma unroll
    for (int c = 0; c < 4; ++c) A[r][c] = Bv[r][c] = make_float2(0.0f, 0.0f);
  }
  __syncthreads();  // jsum cleared
  const bool ok = mbar_wait(&bar, 0, a.err);
  if (!__syncthreads_and(ok)) {  // a copy may still be landing: bounded drain, then leave
    if (tid == 0) mbar_wait(&bar, 0, a.err);
    return;
  }
  const float4 *s0 = src, *s1 = src + P, *s2 = src + 2 * P, *s3 = src + 3 * P,
               *s4 = src + 4 * P;

  if (diag) {
    for (int pp = 0; pp < npairs; ++pp) {
      const float4 F0 = s0[pp], F1 = s1[pp], F2 = s2[pp], F3 = s3[pp], F4 = s4[pp];
      const int jg = j0 + 2 * pp;
#pragma unroll
      for (int r = 0; r < I; ++r)
        sym_ljc_vjp_pair2<LIN, false, true>(F0, F1, F2, F3, F4, nx[r], ny[r], nz[r], ux[r],
                                            uy[r], uz[r], qk[r], sk[r], ek[r], A[r], Bv[r],
                                            nullptr, jg == ig[r], jg + 1 == ig[r]);
    }
  } else {
    float *J = jsum + size_t(warp) * 16 * P;
    for (int g0 = 0; g0 < npairs; g0 += 32) {
#pragma unroll 1
      for (int st = 0; st < 32; ++st) {
        const int pp = g0 + ((lane + st) & 31);
        if (pp < npairs) {
          const float4 F0 = s0[pp], F1 = s1[pp], F2 = s2[pp], F3 = s3[pp], F4 = s4[pp];
          float2 js[8];
#pragma unroll
          for (int c = 0; c < 8; ++c) js[c] = make_float2(0.0f, 0.0f);
#pragma unroll
          for (int r = 0; r < I; ++r)
            sym_ljc_vjp_pair2<LIN, true, false>(F0, F1, F2, F3, F4, nx[r], ny[r], nz[r], ux[r],
                                                uy[r], uz[r], qk[r], sk[r], ek[r], A[r], Bv[r],
                                                js);
          // g and F change sign for the sources, D and E do not
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const bool sym = (c == 3 || c == 7);
            J[(2 * c) * P + pp] += sym ? js[c].x : -js[c].x;
            J[(2 * c + 1) * P + pp] += sym ? js[c].y : -js[c].y;
          }
        }
        __syncwarp();  // at the next step lane l - 1 updates the slot lane l just wrote
      }
    }
  }

  const long long ibase = (long long)bj * a.stride;
#pragma unroll
  for (int r = 0; r < I; ++r)
    if (ig[r] >= 0) {
      a.part_hi[ibase + ig[r]] = make_float4(A[r][0].x + A[r][0].y, A[r][1].x + A[r][1].y,
                                             A[r][2].x + A[r][2].y, A[r][3].x + A[r][3].y);
      a.part_hi[a.bstride + ibase + ig[r]] =
          make_float4(Bv[r][0].x + Bv[r][0].y, Bv[r][1].x + Bv[r][1].y,
                      Bv[r][2].x + Bv[r][2].y, Bv[r][3].x + Bv[r][3].y);
    }
  if (diag) return;
  __syncthreads();
  const long long jbase = (long long)bi * a.stride + j0;
  for (int q = tid; q < nsrc; q += NT) {
    const int pp = q >> 1, h = q & 1;
    float v[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    for (int w = 0; w < T::kWarps; ++w) {
      const float *Jw = jsum + size_t(w) * 16 * P;
#pragma unroll
      for (int c = 0; c < 8; ++c) v[c] += Jw[(2 * c + h) * P + pp];
    }
    a.part_hi[jbase + q] = make_float4(v[0], v[1], v[2], v[3]);
    a.part_hi[a.bstride + jbase + q] = make_float4(v[4], v[5], v[6], v[7]);
  }
}

}  // namespace nbody
