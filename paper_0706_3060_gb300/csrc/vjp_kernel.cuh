// vjp_kernel.cuh -- all-pairs vector-Jacobian product of the force laws for
// reverse-mode leapfrog. The paper has no adjoint; the pair terms below are the
// derivatives of Eq. 1 and of the Table 1 LJC(constant) law.
//
// Gravity, target k, source j, d = x_j - x_k, s^2 = |d|^2 + eps^2, y = 1/s,
// w = m_k lam_j - m_j lam_k:
//   g_k  = G sum_j y^3 [ w - 3 y^2 (d.w) d ]        (T = I/s^3 - 3 d d^T / s^5)
//   gm_k = -G sum_j (lam_j . d) y^3                   (d/dm_k of sum_i lam_i . a_i)
// LJC with u = lam / m, w = u_k - u_j, y = 1/r, sigma = s~k + s~j,
// u6 = (sigma y)^6, phi = q~q~ y^3 + e~e~ y^2 (2 u6^2 - u6) and
// 2 phi' = y^2 [ -3 q~q~ y^3 + e~e~ y^2 (8 u6 - 28 u6^2) ]:
//   g_k  = sum_j [ phi w + 2 phi' (d.w) d ]           (H = phi I + 2 phi' d d^T)
//   F_k  = -sum_j phi d                               (mass derivative -u_k.F_k / m_k)
//   D_k  = sum_j (d.w) e~e~ y^2 (4 u6^2 - u6) / sigma (sigma derivative, x -3 later)
//   E_k  = sum_j (d.w) e~e~ y^2 (2 u6^2 - u6)         (epsilon derivative, x -1/(2 eps_k))
// The pipeline (producer warp, TMA ring, compensated per-tile sums, j-lanes
// with shuffle reduction, per-slice partials) is the same as force_kernel.cuh.
#pragma once

#include "device_common.cuh"
#include "force_kernel.cuh"

namespace nbody {

// Table 1 "Gravity (accel & jerk)" runs on this kernel's two-accumulator pipeline.
constexpr int kLawGAJ = 3;

struct VjpArgs {
  const float4 *pos;   // (x, y, z, m)
  const float4 *lam;   // gravity: lam; LJC: u = lam / m; GAJ: velocities
  const float4 *prm;   // LJC parameters or null
  const float4 *jpair; // packed gravity: (x x y y)(z z m m)(lx lx ly ly)(lz lz 0 0) per pair
  float4 *part_hi;     // [2][slices][stride]: block A then block B (LJC)
  float4 *part_lo;
  long long stride;
  long long bstride;   // offset of block B (slices * stride)
  int *err;
  int n;
  int slices;
  int slice_len;
  float eps2;
  int comp;
  int pdl;  // host side: launch with programmatic dependent launch (griddep_start)
  // Newton-symmetric gravity VJP with exact fixed-point accumulation: eight int64
  // arrays of stride `stride` (integer parts of g.x, g.y, g.z and the mass term
  // scaled by *fscale, then their fractions in units of 2^-32), zeroed before the
  // launch; null: per-block partial slots in part_hi
  long long *acc64;
  const float *fscale;
};

__device__ __forceinline__ float rcp_hw(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

template <bool MASK>
__device__ __forceinline__ void grav_vjp_pair(const float4 pj, const float4 lj, float xk,
                                              float yk, float zk, float mk, float lkx, float lky,
                                              float lkz, float eps2, float4 &A, bool self) {
  const float dx = pj.x - xk;
  const float dy = pj.y - yk;
  const float dz = pj.z - zk;
  const float s2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
  float y = rsqrt_hw(s2);
  if (MASK) y = self ? 0.0f : y;
  const float y2 = y * y;
  const float y3 = y2 * y;
  const float mj = pj.w;
  const float wx = fmaf(mk, lj.x, -(mj * lkx));
  const float wy = fmaf(mk, lj.y, -(mj * lky));
  const float wz = fmaf(mk, lj.z, -(mj * lkz));
  const float dw = fmaf(dx, wx, fmaf(dy, wy, dz * wz));
  const float c = dw * (-3.0f * y2);
  A.x = fmaf(y3, fmaf(c, dx, wx), A.x);
  A.y = fmaf(y3, fmaf(c, dy, wy), A.y);
  A.z = fmaf(y3, fmaf(c, dz, wz), A.z);
  const float ld = fmaf(lj.x, dx, fmaf(lj.y, dy, lj.z * dz));
  A.w = fmaf(ld, y3, A.w);
}

// The gravity VJP pair for two sources at once (f32x2); A holds (g.x, g.y, g.z,
// mass term) as even/odd-source halves.
__device__ __forceinline__ void grav_vjp_pair2(float2 X, float2 Y, float2 Z, float2 Mj, float2 LX,
                                               float2 LY, float2 LZ, float2 nxk, float2 nyk,
                                               float2 nzk, float2 mk, float2 lkx, float2 lky,
                                               float2 lkz, float2 e2, float2 &ax, float2 &ay,
                                               float2 &az, float2 &aw) {
  const float2 dx = __fadd2_rn(X, nxk);
  const float2 dy = __fadd2_rn(Y, nyk);
  const float2 dz = __fadd2_rn(Z, nzk);
  float2 s2 = __ffma2_rn(dz, dz, e2);
  s2 = __ffma2_rn(dy, dy, s2);
  s2 = __ffma2_rn(dx, dx, s2);
  const float2 y = make_float2(rsqrt_hw(s2.x), rsqrt_hw(s2.y));
  const float2 y2 = __fmul2_rn(y, y);
  const float2 y3 = __fmul2_rn(y2, y);
  const float2 nmj = make_float2(-Mj.x, -Mj.y);
  const float2 wx = __ffma2_rn(mk, LX, __fmul2_rn(nmj, lkx));
  const float2 wy = __ffma2_rn(mk, LY, __fmul2_rn(nmj, lky));
  const float2 wz = __ffma2_rn(mk, LZ, __fmul2_rn(nmj, lkz));
  const float2 dw = __ffma2_rn(dx, wx, __ffma2_rn(dy, wy, __fmul2_rn(dz, wz)));
  const float2 c = __fmul2_rn(dw, __fmul2_rn(y2, make_float2(-3.0f, -3.0f)));
  ax = __ffma2_rn(y3, __ffma2_rn(c, dx, wx), ax);
  ay = __ffma2_rn(y3, __ffma2_rn(c, dy, wy), ay);
  az = __ffma2_rn(y3, __ffma2_rn(c, dz, wz), az);
  const float2 ld = __ffma2_rn(LX, dx, __ffma2_rn(LY, dy, __fmul2_rn(LZ, dz)));
  aw = __ffma2_rn(ld, y3, aw);
}

// LIN: linear dielectric (Table 1 LJC(linear)): the Coulomb part of phi is
// 2 q~q~ y^4 instead of q~q~ y^3, and its share of 2 phi' is -4 y^2 times it
// instead of -3 y^2 times it.
template <bool MASK, bool LIN = false>
__device__ __forceinline__ void ljc_vjp_pair(const float4 pj, const float4 uj, const float4 qj,
                                             float xk, float yk, float zk, float ukx, float uky,
                                             float ukz, float qk, float sk, float ek, float4 &A,
                                             float4 &B, bool self) {
  const float dx = pj.x - xk;
  const float dy = pj.y - yk;
  const float dz = pj.z - zk;
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  float y = rsqrt_hw(r2);
  if (MASK) y = self ? 0.0f : y;
  const float y2 = y * y;
  const float qq = qk * qj.x;
  const float s = sk + qj.y;
  const float ee = ek * qj.z;
  const float t = (s * s) * y2;
  const float u = (t * t) * t;
  const float qy3 = LIN ? (qq * y2) * (y2 + y2) : qq * (y * y2);  // Coulomb part of phi
  const float eey2 = ee * y2;
  const float h = fmaf(u, 2.0f, -1.0f) * u;
  const float phi_lj = eey2 * h;
  const float phi = phi_lj + qy3;
  const float k1 = fmaf(u, -28.0f, 8.0f) * u;
  const float tp = y2 * fmaf(eey2, k1, (LIN ? -4.0f : -3.0f) * qy3);
  const float wx = ukx - uj.x;
  const float wy = uky - uj.y;
  const float wz = ukz - uj.z;
  const float dw = fmaf(dx, wx, fmaf(dy, wy, dz * wz));
  const float c = tp * dw;
  A.x = fmaf(c, dx, fmaf(phi, wx, A.x));
  A.y = fmaf(c, dy, fmaf(phi, wy, A.y));
  A.z = fmaf(c, dz, fmaf(phi, wz, A.z));
  B.x = fmaf(phi, dx, B.x);
  B.y = fmaf(phi, dy, B.y);
  B.z = fmaf(phi, dz, B.z);
  const float k2 = fmaf(u, 4.0f, -1.0f) * u;
  const float rs = MASK ? (self ? 0.0f : rcp_hw(s)) : rcp_hw(s);
  A.w = fmaf(dw, (eey2 * k2) * rs, A.w);
  B.w = fmaf(dw, phi_lj, B.w);
}

// The LJC VJP pair for two sources at once (f32x2), the same terms in the same
// order as ljc_vjp_pair. Sources arrive as (x x y y)(z z q q)(s s e e)
// (-ux -ux -uy -uy)(-uz -uz 0 0): the negated u_j makes w = u_k - u_j one add.
template <bool LIN = false>
__device__ __forceinline__ void ljc_vjp_pair2(const float4 F0, const float4 F1, const float4 F2,
                                              const float4 F3, const float4 F4, float2 nxk,
                                              float2 nyk, float2 nzk, float2 ukx, float2 uky,
                                              float2 ukz, float2 qk, float2 sk, float2 ek,
                                              float2 (&A)[4], float2 (&B)[4]) {
  const float2 dx = __fadd2_rn(make_float2(F0.x, F0.y), nxk);
  const float2 dy = __fadd2_rn(make_float2(F0.z, F0.w), nyk);
  const float2 dz = __fadd2_rn(make_float2(F1.x, F1.y), nzk);
  const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
  const float2 y = make_float2(rsqrt_hw(r2.x), rsqrt_hw(r2.y));
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
  A[0] = __ffma2_rn(c, dx, __ffma2_rn(phi, wx, A[0]));
  A[1] = __ffma2_rn(c, dy, __ffma2_rn(phi, wy, A[1]));
  A[2] = __ffma2_rn(c, dz, __ffma2_rn(phi, wz, A[2]));
  B[0] = __ffma2_rn(phi, dx, B[0]);
  B[1] = __ffma2_rn(phi, dy, B[1]);
  B[2] = __ffma2_rn(phi, dz, B[2]);
  const float2 k2 = __fmul2_rn(__ffma2_rn(u, make_float2(4.0f, 4.0f), make_float2(-1.0f, -1.0f)), u);
  const float2 rs = make_float2(rcp_hw(s.x), rcp_hw(s.y));
  A[3] = __ffma2_rn(dw, __fmul2_rn(__fmul2_rn(eey2, k2), rs), A[3]);
  B[3] = __ffma2_rn(dw, phi_lj, B[3]);
}

// Acceleration and jerk (Table 1 GAJ): d = x_j - x_k, u = v_j - v_k, y = 1/s,
// w = m_j y^3:  A += w d;  B += w (u - 3 (d.u) y^2 d).
template <bool MASK>
__device__ __forceinline__ void gaj_pair(const float4 pj, const float4 vj, float xk, float yk,
                                         float zk, float vxk, float vyk, float vzk, float eps2,
                                         float4 &A, float4 &B, bool self) {
  const float dx = pj.x - xk;
  const float dy = pj.y - yk;
  const float dz = pj.z - zk;
  const float ux = vj.x - vxk;
  const float uy = vj.y - vyk;
  const float uz = vj.z - vzk;
  const float s2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
  float y = rsqrt_hw(s2);
  if (MASK) y = self ? 0.0f : y;
  const float y2 = y * y;
  const float w = (pj.w * y) * y2;
  const float ru = fmaf(dx, ux, fmaf(dy, uy, dz * uz));
  const float c = ru * (3.0f * y2);
  A.x = fmaf(w, dx, A.x);
  A.y = fmaf(w, dy, A.y);
  A.z = fmaf(w, dz, A.z);
  B.x = fmaf(w, fmaf(-c, dx, ux), B.x);
  B.y = fmaf(w, fmaf(-c, dy, uy), B.y);
  B.z = fmaf(w, fmaf(-c, dz, uz), B.z);
}

// Acceleration and jerk for two sources at once (f32x2), the same terms as
// gaj_pair: A += w d, B += w (u - 3 y^2 (d.u) d), w = m_j y^3.
__device__ __forceinline__ void gaj_pair2(float2 X, float2 Y, float2 Z, float2 Mj, float2 VX,
                                          float2 VY, float2 VZ, float2 nxk, float2 nyk,
                                          float2 nzk, float2 nvx, float2 nvy, float2 nvz,
                                          float2 e2, float2 &ax, float2 &ay, float2 &az,
                                          float2 &bx, float2 &by, float2 &bz) {
  const float2 dx = __fadd2_rn(X, nxk);
  const float2 dy = __fadd2_rn(Y, nyk);
  const float2 dz = __fadd2_rn(Z, nzk);
  const float2 ux = __fadd2_rn(VX, nvx);
  const float2 uy = __fadd2_rn(VY, nvy);
  const float2 uz = __fadd2_rn(VZ, nvz);
  float2 s2 = __ffma2_rn(dz, dz, e2);
  s2 = __ffma2_rn(dy, dy, s2);
  s2 = __ffma2_rn(dx, dx, s2);
  const float2 y = make_float2(rsqrt_hw(s2.x), rsqrt_hw(s2.y));
  const float2 y2 = __fmul2_rn(y, y);
  const float2 w = __fmul2_rn(__fmul2_rn(Mj, y), y2);
  const float2 ru = __ffma2_rn(dx, ux, __ffma2_rn(dy, uy, __fmul2_rn(dz, uz)));
  const float2 c = __fmul2_rn(ru, __fmul2_rn(y2, make_float2(-3.0f, -3.0f)));
  ax = __ffma2_rn(w, dx, ax);
  ay = __ffma2_rn(w, dy, ay);
  az = __ffma2_rn(w, dz, az);
  bx = __ffma2_rn(w, __ffma2_rn(c, dx, ux), bx);
  by = __ffma2_rn(w, __ffma2_rn(c, dy, uy), by);
  bz = __ffma2_rn(w, __ffma2_rn(c, dz, uz), bz);
}

template <int LAW, int NT, int I, int SW, int JT, bool PK = false>
struct VjpTile {
  static constexpr int kThreads = NT + 32;
  static constexpr int kSlots = NT / SW;
  static constexpr int kTileI = kSlots * I;
  static constexpr int kStreams = is_ljc(LAW) ? 3 : 2;
  static constexpr size_t kSmemBytes = size_t(kStages) * JT * 16 * kStreams;
  // packed sources: float4s per source pair (gravity VJP and jerk 4, LJC VJP 5)
  static constexpr int kPairF4 = is_ljc(LAW) ? 5 : 4;
  static constexpr int kStageF4 = kPairF4 * JT / 2;  // float4s of one ring stage
  static_assert(!PK || kStageF4 <= JT * kStreams, "packed stage exceeds the ring");
};

__device__ __forceinline__ void comp_fold(float4 &hi, float4 &lo, float4 &p, int comp) {
  if (comp) {
    comp_add(hi.x, lo.x, p.x);
    comp_add(hi.y, lo.y, p.y);
    comp_add(hi.z, lo.z, p.z);
    comp_add(hi.w, lo.w, p.w);
  } else {
    hi.x += p.x;
    hi.y += p.y;
    hi.z += p.z;
    hi.w += p.w;
  }
  p = make_float4(0.f, 0.f, 0.f, 0.f);
}

__device__ __forceinline__ void shfl_combine(float4 &hi, float4 &lo, int off) {
  float4 oh, ol;
  oh.x = __shfl_xor_sync(0xffffffffu, hi.x, off);
  oh.y = __shfl_xor_sync(0xffffffffu, hi.y, off);
  oh.z = __shfl_xor_sync(0xffffffffu, hi.z, off);
  oh.w = __shfl_xor_sync(0xffffffffu, hi.w, off);
  ol.x = __shfl_xor_sync(0xffffffffu, lo.x, off);
  ol.y = __shfl_xor_sync(0xffffffffu, lo.y, off);
  ol.z = __shfl_xor_sync(0xffffffffu, lo.z, off);
  ol.w = __shfl_xor_sync(0xffffffffu, lo.w, off);
  float e;
  two_sum(hi.x, oh.x, hi.x, e);
  lo.x = __fadd_rn(__fadd_rn(lo.x, ol.x), e);
  two_sum(hi.y, oh.y, hi.y, e);
  lo.y = __fadd_rn(__fadd_rn(lo.y, ol.y), e);
  two_sum(hi.z, oh.z, hi.z, e);
  lo.z = __fadd_rn(__fadd_rn(lo.z, ol.z), e);
  two_sum(hi.w, oh.w, hi.w, e);
  lo.w = __fadd_rn(__fadd_rn(lo.w, ol.w), e);
}

template <int LAW, int NT, int I, int SW, int JT, bool PK = false, int PU = 2>
__global__ void __launch_bounds__(NT + 32) vjp_kernel(const VjpArgs a) {
  griddep_start();
  using T = VjpTile<LAW, NT, I, SW, JT, PK>;
  static_assert(!PK || SW == 1, "packed tiles: one j-lane");
  static_assert(JT % 2 == 0, "j-tiles hold whole source pairs");
  constexpr int NWARPS = NT / 32;
  constexpr int SLOTS = T::kSlots;
  constexpr int TI = T::kTileI;
  constexpr bool LJ = is_ljc(LAW);
  constexpr bool LIN = (LAW == kLawLJCLin);  // linear dielectric
  constexpr bool GJ = (LAW == kLawGAJ);
  constexpr bool TWO = LJ || GJ;  // second accumulator block in use

  extern __shared__ __align__(128) unsigned char smem_raw[];
  float4 *sm_pos = reinterpret_cast<float4 *>(smem_raw);
  float4 *sm_lam = sm_pos + kStages * JT;
  float4 *sm_prm = sm_lam + kStages * JT;
  __shared__ __align__(8) uint64_t full_bar[kStages];
  __shared__ __align__(8) uint64_t empty_bar[kStages];
  __shared__ int meta_len[kStages];
  __shared__ int meta_cj0[kStages];

  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], NWARPS);
    }
    mbar_fence_init();
  }
  __syncthreads();

  const int b = blockIdx.x;
  const int tile = b / a.slices, slice = b % a.slices;
  const int i0 = tile * TI;
  const int ni = min(TI, a.n - i0);
  const int j0 = slice * a.slice_len;
  const int jend = min(a.n, j0 + a.slice_len);
  const int nchunks = (jend - j0 + JT - 1) / JT;
  if (ni <= 0 || jend <= j0) {
    if (tid == 0) set_error(a.err, kDevBadItem);
    return;
  }

  if (tid >= NT) {  // producer
    if (tid != NT) return;
    int it = 0;
    for (; it < nchunks; ++it) {
      const int st = it % kStages;
      if (!mbar_wait(&empty_bar[st], ((it / kStages) & 1) ^ 1, a.err)) break;
      const int cj = j0 + it * JT;
      const int len = min(JT, jend - cj);
      meta_len[st] = len;
      meta_cj0[st] = cj;
      if (PK) {
        // pairs of sources, kPairF4 float4 each; stages of kStageF4 float4s
        const uint32_t bytes = uint32_t((len + 1) >> 1) * T::kPairF4 * 16u;
        mbar_arrive_expect_tx(&full_bar[st], bytes);
        tma_load_1d(sm_pos + st * T::kStageF4, a.jpair + size_t(cj >> 1) * T::kPairF4, bytes,
                    &full_bar[st]);
      } else {
        const uint32_t bytes = uint32_t(len) * 16u;
        mbar_arrive_expect_tx(&full_bar[st], bytes * T::kStreams);
        tma_load_1d(sm_pos + st * JT, a.pos + cj, bytes, &full_bar[st]);
        tma_load_1d(sm_lam + st * JT, a.lam + cj, bytes, &full_bar[st]);
        if (LJ) tma_load_1d(sm_prm + st * JT, a.prm + cj, bytes, &full_bar[st]);
      }
    }
    if (it < nchunks)  // timed out: bounded drain of copies in flight
      for (int k = max(0, it - kStages); k < it; ++k)
        mbar_wait(&full_bar[k % kStages], (k / kStages) & 1, a.err);
    return;
  }

  const int warp = tid >> 5, lane = tid & 31;
  const int jl = (SW > 1) ? (lane % SW) : 0;
  const int slot = warp * (32 / SW) + lane / SW;
  float xk[I], yk[I], zk[I], mk[I], lx[I], ly[I], lz[I], qk[I], sk[I], ek[I];
  int ig[I];
  float4 pA[I], hA[I], oA[I], pB[I], hB[I], oB[I];
#pragma unroll
  for (int r = 0; r < I; ++r) {
    const int il = r * SLOTS + slot;
    const int g = i0 + min(il, ni - 1);
    ig[r] = (il < ni) ? g : -1;
    const float4 p4 = __ldg(a.pos + g);
    const float4 l4 = __ldg(a.lam + g);
    xk[r] = p4.x;
    yk[r] = p4.y;
    zk[r] = p4.z;
    mk[r] = p4.w;
    lx[r] = l4.x;
    ly[r] = l4.y;
    lz[r] = l4.z;
    if (LJ) {
      const float4 q4 = __ldg(a.prm + g);
      qk[r] = q4.x;
      sk[r] = q4.y;
      ek[r] = q4.z;
    } else {
      qk[r] = sk[r] = ek[r] = 0.f;
    }
    pA[r] = hA[r] = oA[r] = make_float4(0.f, 0.f, 0.f, 0.f);
    pB[r] = hB[r] = oB[r] = make_float4(0.f, 0.f, 0.f, 0.f);
  }

  for (int it = 0; it < nchunks; ++it) {
    const int st = it % kStages;
    if (!mbar_wait(&full_bar[st], (it / kStages) & 1, a.err)) return;
    const int len = meta_len[st];
    const int cj0 = meta_cj0[st];
    const float4 *sp = sm_pos + st * JT;
    const float4 *sl = sm_lam + st * JT;
    const float4 *sq = sm_prm + st * JT;
    const bool masked = (cj0 < i0 + ni) && (i0 < cj0 + len);
    if (PK && GJ) {
      const float4 *pk = sm_pos + st * T::kStageF4;
      if (!masked) {
        const float2 e2 = make_float2(a.eps2, a.eps2);
        const int npairs = (len + 1) >> 1;
        float2 ax[I], ay[I], az[I], bx[I], by[I], bz[I];
#pragma unroll
        for (int r = 0; r < I; ++r)
          ax[r] = ay[r] = az[r] = bx[r] = by[r] = bz[r] = make_float2(0.f, 0.f);
#pragma unroll PU
        for (int pp = 0; pp < npairs; ++pp) {
          const float4 P0 = pk[4 * pp], P1 = pk[4 * pp + 1];
          const float4 V0 = pk[4 * pp + 2], V1 = pk[4 * pp + 3];
#pragma unroll
          for (int r = 0; r < I; ++r)
            gaj_pair2(make_float2(P0.x, P0.y), make_float2(P0.z, P0.w), make_float2(P1.x, P1.y),
                      make_float2(P1.z, P1.w), make_float2(V0.x, V0.y), make_float2(V0.z, V0.w),
                      make_float2(V1.x, V1.y), make_float2(-xk[r], -xk[r]),
                      make_float2(-yk[r], -yk[r]), make_float2(-zk[r], -zk[r]),
                      make_float2(-lx[r], -lx[r]), make_float2(-ly[r], -ly[r]),
                      make_float2(-lz[r], -lz[r]), e2, ax[r], ay[r], az[r], bx[r], by[r], bz[r]);
        }
#pragma unroll
        for (int r = 0; r < I; ++r) {
          pA[r].x += ax[r].x + ax[r].y;
          pA[r].y += ay[r].x + ay[r].y;
          pA[r].z += az[r].x + az[r].y;
          pB[r].x += bx[r].x + bx[r].y;
          pB[r].y += by[r].x + by[r].y;
          pB[r].z += bz[r].x + bz[r].y;
        }
      } else {
        for (int jj = 0; jj < len; ++jj) {
          const int q = 4 * (jj >> 1);
          const bool odd = jj & 1;
          const float4 P0 = pk[q], P1 = pk[q + 1], V0 = pk[q + 2], V1 = pk[q + 3];
          const float4 pj = make_float4(odd ? P0.y : P0.x, odd ? P0.w : P0.z, odd ? P1.y : P1.x,
                                        odd ? P1.w : P1.z);
          const float4 vj = make_float4(odd ? V0.y : V0.x, odd ? V0.w : V0.z, odd ? V1.y : V1.x,
                                        0.f);
          const int jg = cj0 + jj;
#pragma unroll
          for (int r = 0; r < I; ++r)
            gaj_pair<true>(pj, vj, xk[r], yk[r], zk[r], lx[r], ly[r], lz[r], a.eps2, pA[r], pB[r],
                           jg == ig[r]);
        }
      }
    } else if (PK && LJ) {
      const float4 *pk = sm_pos + st * T::kStageF4;
      if (!masked) {
        const int npairs = (len + 1) >> 1;
        float2 A2[I][4], B2[I][4];
#pragma unroll
        for (int r = 0; r < I; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) A2[r][c] = B2[r][c] = make_float2(0.f, 0.f);
#pragma unroll PU
        for (int pp = 0; pp < npairs; ++pp) {
          const float4 F0 = pk[5 * pp], F1 = pk[5 * pp + 1], F2 = pk[5 * pp + 2];
          const float4 F3 = pk[5 * pp + 3], F4 = pk[5 * pp + 4];
#pragma unroll
          for (int r = 0; r < I; ++r)
            ljc_vjp_pair2<LIN>(F0, F1, F2, F3, F4, make_float2(-xk[r], -xk[r]),
                          make_float2(-yk[r], -yk[r]), make_float2(-zk[r], -zk[r]),
                          make_float2(lx[r], lx[r]), make_float2(ly[r], ly[r]),
                          make_float2(lz[r], lz[r]), make_float2(qk[r], qk[r]),
                          make_float2(sk[r], sk[r]), make_float2(ek[r], ek[r]), A2[r], B2[r]);
        }
#pragma unroll
        for (int r = 0; r < I; ++r) {
          pA[r].x += A2[r][0].x + A2[r][0].y;
          pA[r].y += A2[r][1].x + A2[r][1].y;
          pA[r].z += A2[r][2].x + A2[r][2].y;
          pA[r].w += A2[r][3].x + A2[r][3].y;
          pB[r].x += B2[r][0].x + B2[r][0].y;
          pB[r].y += B2[r][1].x + B2[r][1].y;
          pB[r].z += B2[r][2].x + B2[r][2].y;
          pB[r].w += B2[r][3].x + B2[r][3].y;
        }
      } else {
        for (int jj = 0; jj < len; ++jj) {
          const int q = 5 * (jj >> 1);
          const bool odd = jj & 1;
          const float4 F0 = pk[q], F1 = pk[q + 1], F2 = pk[q + 2], F3 = pk[q + 3],
                       F4 = pk[q + 4];
          const float4 pj = make_float4(odd ? F0.y : F0.x, odd ? F0.w : F0.z, odd ? F1.y : F1.x,
                                        0.f);
          const float4 uj = make_float4(-(odd ? F3.y : F3.x), -(odd ? F3.w : F3.z),
                                        -(odd ? F4.y : F4.x), 0.f);
          const float4 qj = make_float4(odd ? F1.w : F1.z, odd ? F2.y : F2.x, odd ? F2.w : F2.z,
                                        0.f);
          const int jg = cj0 + jj;
#pragma unroll
          for (int r = 0; r < I; ++r)
            ljc_vjp_pair<true, LIN>(pj, uj, qj, xk[r], yk[r], zk[r], lx[r], ly[r], lz[r], qk[r],
                               sk[r], ek[r], pA[r], pB[r], jg == ig[r]);
        }
      }
    } else if (PK) {
      const float4 *pk = sm_pos + st * T::kStageF4;
      if (!masked) {
        const float2 e2 = make_float2(a.eps2, a.eps2);
        const int npairs = (len + 1) >> 1;
        float2 ax[PK ? I : 1], ay[PK ? I : 1], az[PK ? I : 1], aw[PK ? I : 1];
#pragma unroll
        for (int r = 0; r < I; ++r) ax[r] = ay[r] = az[r] = aw[r] = make_float2(0.f, 0.f);
#pragma unroll PU
        for (int pp = 0; pp < npairs; ++pp) {
          const float4 P0 = pk[4 * pp], P1 = pk[4 * pp + 1];
          const float4 L0 = pk[4 * pp + 2], L1 = pk[4 * pp + 3];
#pragma unroll
          for (int r = 0; r < I; ++r)
            grav_vjp_pair2(make_float2(P0.x, P0.y), make_float2(P0.z, P0.w),
                           make_float2(P1.x, P1.y), make_float2(P1.z, P1.w),
                           make_float2(L0.x, L0.y), make_float2(L0.z, L0.w),
                           make_float2(L1.x, L1.y), make_float2(-xk[r], -xk[r]),
                           make_float2(-yk[r], -yk[r]), make_float2(-zk[r], -zk[r]),
                           make_float2(mk[r], mk[r]), make_float2(lx[r], lx[r]),
                           make_float2(ly[r], ly[r]), make_float2(lz[r], lz[r]), e2, ax[r],
                           ay[r], az[r], aw[r]);
        }
#pragma unroll
        for (int r = 0; r < I; ++r) {
          pA[r].x += ax[r].x + ax[r].y;
          pA[r].y += ay[r].x + ay[r].y;
          pA[r].z += az[r].x + az[r].y;
          pA[r].w += aw[r].x + aw[r].y;
        }
      } else {
        for (int jj = 0; jj < len; ++jj) {
          const int q = 4 * (jj >> 1);
          const bool odd = jj & 1;
          const float4 P0 = pk[q], P1 = pk[q + 1], L0 = pk[q + 2], L1 = pk[q + 3];
          const float4 pj = make_float4(odd ? P0.y : P0.x, odd ? P0.w : P0.z, odd ? P1.y : P1.x,
                                        odd ? P1.w : P1.z);
          const float4 lj = make_float4(odd ? L0.y : L0.x, odd ? L0.w : L0.z, odd ? L1.y : L1.x,
                                        0.f);
          const int jg = cj0 + jj;
#pragma unroll
          for (int r = 0; r < I; ++r)
            grav_vjp_pair<true>(pj, lj, xk[r], yk[r], zk[r], mk[r], lx[r], ly[r], lz[r], a.eps2,
                                pA[r], jg == ig[r]);
        }
      }
    } else if (GJ) {
      if (!masked) {
#pragma unroll PU
        for (int jj = jl; jj < len; jj += SW) {
          const float4 pj = sp[jj];
          const float4 vj = sl[jj];
#pragma unroll
          for (int r = 0; r < I; ++r)
            gaj_pair<false>(pj, vj, xk[r], yk[r], zk[r], lx[r], ly[r], lz[r], a.eps2, pA[r], pB[r],
                            false);
        }
      } else {
        for (int jj = jl; jj < len; jj += SW) {
          const float4 pj = sp[jj];
          const float4 vj = sl[jj];
          const int jg = cj0 + jj;
#pragma unroll
          for (int r = 0; r < I; ++r)
            gaj_pair<true>(pj, vj, xk[r], yk[r], zk[r], lx[r], ly[r], lz[r], a.eps2, pA[r], pB[r],
                           jg == ig[r]);
        }
      }
    } else if (!LJ) {
      if (!masked) {
#pragma unroll PU
        for (int jj = jl; jj < len; jj += SW) {
          const float4 pj = sp[jj];
          const float4 lj = sl[jj];
#pragma unroll
          for (int r = 0; r < I; ++r)
            grav_vjp_pair<false>(pj, lj, xk[r], yk[r], zk[r], mk[r], lx[r], ly[r], lz[r], a.eps2,
                                 pA[r], false);
        }
      } else {
        for (int jj = jl; jj < len; jj += SW) {
          const float4 pj = sp[jj];
          const float4 lj = sl[jj];
          const int jg = cj0 + jj;
#pragma unroll
          for (int r = 0; r < I; ++r)
            grav_vjp_pair<true>(pj, lj, xk[r], yk[r], zk[r], mk[r], lx[r], ly[r], lz[r], a.eps2,
                                pA[r], jg == ig[r]);
        }
      }
    } else {
      if (!masked) {
        for (int jj = jl; jj < len; jj += SW) {
          const float4 pj = sp[jj];
          const float4 uj = sl[jj];
          const float4 qj = sq[jj];
#pragma unroll
          for (int r = 0; r < I; ++r)
            ljc_vjp_pair<false, LIN>(pj, uj, qj, xk[r], yk[r], zk[r], lx[r], ly[r], lz[r], qk[r],
                                sk[r], ek[r], pA[r], pB[r], false);
        }
      } else {
        for (int jj = jl; jj < len; jj += SW) {
          const float4 pj = sp[jj];
          const float4 uj = sl[jj];
          const float4 qj = sq[jj];
          const int jg = cj0 + jj;
#pragma unroll
          for (int r = 0; r < I; ++r)
            ljc_vjp_pair<true, LIN>(pj, uj, qj, xk[r], yk[r], zk[r], lx[r], ly[r], lz[r], qk[r],
                               sk[r], ek[r], pA[r], pB[r], jg == ig[r]);
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty_bar[st]);
#pragma unroll
    for (int r = 0; r < I; ++r) {
      comp_fold(hA[r], oA[r], pA[r], a.comp);
      if (TWO) comp_fold(hB[r], oB[r], pB[r], a.comp);
    }
  }

#pragma unroll
  for (int off = SW / 2; off >= 1; off >>= 1) {
#pragma unroll
    for (int r = 0; r < I; ++r) {
      shfl_combine(hA[r], oA[r], off);
      if (TWO) shfl_combine(hB[r], oB[r], off);
    }
  }
  if (jl == 0) {
    const long long base = (long long)slice * a.stride;
#pragma unroll
    for (int r = 0; r < I; ++r) {
      if (ig[r] < 0) continue;
      a.part_hi[base + ig[r]] = hA[r];
      a.part_lo[base + ig[r]] = oA[r];
      if (TWO) {
        a.part_hi[a.bstride + base + ig[r]] = hB[r];
        a.part_lo[a.bstride + base + ig[r]] = oB[r];
      }
    }
  }
}

}  // namespace nbody
