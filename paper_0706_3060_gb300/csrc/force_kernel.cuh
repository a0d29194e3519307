// force_kernel.cuh -- warp-specialized all-pairs force kernel for sm_103a.
//
// The computation is the direct sum of Sec. 2 (every target i accumulates the
// pair force of every source j), parallel over i, with the j-stream shared by
// every thread of a CTA, as in the paper's force kernel. GB300 mapping:
//   * one producer warp streams j-tiles of JT particles (16 B each, plus 16 B
//     of LJC parameters) from global memory into a STAGES-deep shared-memory
//     ring with 1-D TMA bulk copies completing on mbarriers;
//   * NT consumer threads each hold I target particles in registers -- the
//     i-side half of the paper's A x B unrolling (Sec. 3.3) -- and read
//     every staged j once per I interactions; the j-loop is unrolled;
//   * each j-tile's contribution is summed plainly in FP32 and then folded into
//     a (hi, lo) pair with TwoSum, so the compensation costs a few operations
//     per tile rather than per pair (the precision policy of Sec. 3.2);
//   * SW j-lanes per warp split the j-range inside a warp and are combined
//     with __shfl_xor in a fixed butterfly; several CTAs may split the
//     j-range of one i-tile ("replication", Sec. 3.4) and write per-slice
//     partials that the finalize kernel adds in a fixed order. Results
//     are therefore bitwise reproducible run to run.
// The self pair is excluded by index (an index comparison, as in the Appendix
// listing) only in tiles whose j-range overlaps the CTA's i-range.
#pragma once

#include <type_traits>

#include "device_common.cuh"

namespace nbody {

enum : int { kLawGrav = 0, kLawLJC = 1, kLawMixed = 2, kLawLJCLin = 4 };

// LJ + Coulomb laws (constant or linear dielectric) share data layout and code.
__host__ __device__ constexpr bool is_ljc(int law) { return law == kLawLJC || law == kLawLJCLin; }

constexpr int kStages = 4;

// One unit of work: targets [i0, i0+ni) against sources [j0, j0+nj) of the
// same system; results go to partial slot `slice`.
struct WorkItem {
  int i0;
  int ni;
  int j0;
  int nj;
  int law;
  int slice;
  float eps2;
  int pj0;  // packed kernels: index of the source pair that starts at j0
};

struct ForceArgs {
  const float4 *pos;   // (x, y, z, m)
  const float4 *prm;   // LJC (q~, s~, e~, type) or null
  const float4 *jpair; // packed kernels: source pairs, gravity (x0 x1 y0 y1)(z0 z1 m0 m1)
                       // or LJC (x0 x1 y0 y1)(z0 z1 q0 q1)(s0 s1 e0 e1)
  const float4 *jpair2;// batched packed kernels: the LJC pair buffer (jpair: gravity)
  float4 *part_hi;     // [slices][stride]
  float4 *part_lo;     // [slices][stride]
  long long stride;    // elements per slice
  int *err;            // device error word
  // targets: by default the sources themselves (tpos == pos, tprm == prm,
  // n_t == n); for a subset, a gathered copy plus the global index of each
  // target (tidx), which then drives the self-pair mask in every tile
  const float4 *tpos;
  const float4 *tprm;
  const int *tidx;
  int n_t;
  // single system: items are (i-tile, j-slice) pairs enumerated by blockIdx.x
  int n;
  int slices;
  int slice_len;       // multiple of JT
  float eps2;
  // work list (batched): items[k], k taken from *counter (persistent CTAs)
  const WorkItem *items;
  int n_items;
  int *counter;        // null: single-system mode
  int comp;            // 1: compensated (hi, lo) sums per j-tile
  const float *fscale; // fixed-point kernels: device word holding the scale 2^S
  // Newton-symmetric gravity with atomic accumulation: eight int64 arrays of
  // stride `stride` (integer parts of x, y, z, w scaled by *fscale, then their
  // fractions in units of 2^-32), zeroed before the launch, into which every CTA
  // adds its per-block partials; null: per-block partial slots in part_hi / part_lo
  long long *acc64;
  int pdl;  // host side: launch with programmatic dependent launch (griddep_start)
};

enum : int { kChunkFirst = 1, kChunkLast = 2, kChunkEnd = 4 };

struct ChunkMeta {
  WorkItem item;
  int cj0;
  int len;
  int flags;
  int pad;
};

// ---- pair interactions ---------------------------------------------------------
// Gravity (Eq. 1, Appendix listing): d = x_j - x_i, s2 = |d|^2 + eps^2,
// y = 1/sqrt(s2); acc += m_j y^3 d; pot += m_j y (scaled by G / -G later).
template <bool POT, bool PRECISE, bool MASK>
__device__ __forceinline__ void grav_pair(const float4 pj, float xi, float yi, float zi,
                                          float eps2, float4 &acc, bool self) {
  const float dx = pj.x - xi;
  const float dy = pj.y - yi;
  const float dz = pj.z - zi;
  const float s2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
  float y = rsqrt_hw(s2);
  if (PRECISE) y = rsqrt_newton(y, s2);
  if (MASK) y = self ? 0.0f : y;
  const float my = pj.w * y;
  const float w = my * (y * y);
  acc.x = fmaf(w, dx, acc.x);
  acc.y = fmaf(w, dy, acc.y);
  acc.z = fmaf(w, dz, acc.z);
  if (POT) acc.w += my;
}

// The same gravity pair for two sources at once with packed f32x2 arithmetic
// (FADD2/FFMA2/FMUL2 issue one instruction for two lanes of work); the two
// halves of each accumulator are the even and odd sources of the j-tile.
// MASK: s0 / s1 flag a source that is the target itself; its term is dropped
// (y = 0), the index exclusion of the scalar path.
template <bool POT, bool PRECISE, bool MASK = false>
__device__ __forceinline__ void grav_pair2(float2 X, float2 Y, float2 Z, float2 M, float2 nxi,
                                           float2 nyi, float2 nzi, float2 eps2, float2 &ax,
                                           float2 &ay, float2 &az, float2 &pot, bool s0 = false,
                                           bool s1 = false) {
  const float2 dx = __fadd2_rn(X, nxi);
  const float2 dy = __fadd2_rn(Y, nyi);
  const float2 dz = __fadd2_rn(Z, nzi);
  float2 s2 = __ffma2_rn(dz, dz, eps2);
  s2 = __ffma2_rn(dy, dy, s2);
  s2 = __ffma2_rn(dx, dx, s2);
  float2 y = make_float2(rsqrt_hw(s2.x), rsqrt_hw(s2.y));
  if (PRECISE) {
    const float2 hs = __fmul2_rn(s2, make_float2(-0.5f, -0.5f));
    const float2 t = __ffma2_rn(hs, __fmul2_rn(y, y), make_float2(1.5f, 1.5f));
    y = __fmul2_rn(y, t);
  }
  if (MASK) {
    y.x = s0 ? 0.0f : y.x;
    y.y = s1 ? 0.0f : y.y;
  }
  const float2 my = __fmul2_rn(M, y);
  const float2 w = __fmul2_rn(my, __fmul2_rn(y, y));
  ax = __ffma2_rn(w, dx, ax);
  ay = __ffma2_rn(w, dy, ay);
  az = __ffma2_rn(w, dz, az);
  if (POT) pot = __fadd2_rn(pot, my);
}

// LJ 12-6 + Coulomb (Table 1 LJC(constant)) with pre-scaled parameters:
// q~ = q sqrt(k/eps_r), s~ = sigma/2, e~ = sqrt(24 eps), so that
// q~i q~j = k qi qj / eps_r, s~i + s~j = sigma_ij, e~i e~j = 24 eps_ij.
// With d = x_j - x_i, y = 1/r, u = (sigma_ij y)^6:
//   f = q~q~ y^3 + e~e~ y^2 (2u^2 - u);  acc += f d  (force on i is -acc)
//   pot += q~q~ y + (e~e~ / 6)(u^2 - u)
//
// LIN (Table 1 LJC(linear), dielectric growing linearly with r): the Coulomb
// terms become 2 q~q~ y^4 in f and q~q~ y^2 in pot.
template <bool POT, bool PRECISE, bool MASK, bool LIN = false>
__device__ __forceinline__ void ljc_pair(const float4 pj, const float4 qj, float xi, float yi,
                                         float zi, float qi, float si, float ei, float4 &acc,
                                         bool self) {
  const float dx = pj.x - xi;
  const float dy = pj.y - yi;
  const float dz = pj.z - zi;
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  float y = rsqrt_hw(r2);
  if (PRECISE) y = rsqrt_newton(y, r2);
  if (MASK) y = self ? 0.0f : y;
  const float y2 = y * y;
  const float qq = qi * qj.x;
  const float s = si + qj.y;
  const float t = (s * s) * y2;
  const float u = (t * t) * t;
  const float ee = ei * qj.z;
  const float fc = LIN ? (qq * y2) * (y2 + y2) : (qq * y) * y2;
  const float h = fmaf(u, 2.0f, -1.0f) * u;
  const float f = fmaf(ee * y2, h, fc);
  acc.x = fmaf(f, dx, acc.x);
  acc.y = fmaf(f, dy, acc.y);
  acc.z = fmaf(f, dz, acc.z);
  if (POT) {
    acc.w = fmaf(qq, LIN ? y2 : y, acc.w);
    acc.w = fmaf(ee * (1.0f / 6.0f), fmaf(u, u, -u), acc.w);
  }
}

// LJC for two sources at once in f32x2 arithmetic (same terms as ljc_pair).
template <bool POT, bool PRECISE, bool LIN = false, bool MASK = false>
__device__ __forceinline__ void ljc_pair2(float2 X, float2 Y, float2 Z, float2 Q, float2 S,
                                          float2 E, float2 nxi, float2 nyi, float2 nzi,
                                          float2 qi, float2 si, float2 ei, float2 &ax, float2 &ay,
                                          float2 &az, float2 &pot, bool s0 = false,
                                          bool s1 = false) {
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
  if (MASK) {
    y.x = s0 ? 0.0f : y.x;
    y.y = s1 ? 0.0f : y.y;
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
  if (POT) {
    pot = __ffma2_rn(qq, LIN ? y2 : y, pot);
    pot = __ffma2_rn(__fmul2_rn(ee, make_float2(1.0f / 6.0f, 1.0f / 6.0f)),
                     __ffma2_rn(u, u, make_float2(-u.x, -u.y)), pot);
  }
}

// float4s per pair of sources in the packed layouts: gravity (x x y y)(z z m m),
// LJC (x x y y)(z z q q)(s s e e).
template <int LAW>
struct PairLayout {
  static constexpr int kF4 = (LAW == kLawGrav) ? 2 : 3;
};
// (is_ljc laws use the 3-float4 layout)

template <int LAW, int NT, int I, int SW, int JT>
struct ForceTile {
  static constexpr int kThreads = NT + 32;  // + producer warp
  static constexpr int kSlots = NT / SW;    // i-slots per CTA
  static constexpr int kTileI = kSlots * I; // targets per item
  static constexpr bool kPrm = (LAW != kLawGrav);
  static constexpr size_t kSmemBytes = size_t(kStages) * JT * 16 * (kPrm ? 2 : 1);
};

// ---- the kernel -------------------------------------------------------------------
// FX: each j-tile's FP32 partial is rounded onto a 64-bit fixed-point grid
// (scale 2^S from *a.fscale) and added as an integer, as GRAPE-6 accumulates
// (Sec. 3.2). Integer addition is associative, so the result does not depend on
// how the j-range is split across CTAs or lanes: bitwise the same for every
// j-split and slice boundary.
template <int LAW, int NT, int I, int SW, int JT, bool POT, bool PRECISE, bool PK = false,
          int PU = 2, int MINB = 1, bool FX = false>
__global__ void __launch_bounds__(NT + 32, MINB) force_kernel(const ForceArgs a) {
  griddep_start();
  using T = ForceTile<LAW, NT, I, SW, JT>;
  constexpr bool LIN = (LAW == kLawLJCLin);
  constexpr bool MIX = (LAW == kLawMixed);
  // float4s per source pair (the mixed kernel sizes its stages for the LJC layout)
  constexpr int PF4 = PairLayout<(is_ljc(LAW) || MIX) ? kLawLJC : kLawGrav>::kF4;
  constexpr int STAGE_F4 = PK ? PF4 * JT / 2 : JT;  // float4s per ring stage
  constexpr int NWARPS = NT / 32;
  constexpr int SLOTS = T::kSlots;
  constexpr int TI = T::kTileI;
  static_assert(NT % 32 == 0 && 32 % SW == 0, "bad tile");
  static_assert(JT % SW == 0, "bad j tile");

  extern __shared__ __align__(128) unsigned char smem_raw[];
  float4 *sm_pos = reinterpret_cast<float4 *>(smem_raw);
  float4 *sm_prm = sm_pos + kStages * JT;
  __shared__ __align__(8) uint64_t full_bar[kStages];
  __shared__ __align__(8) uint64_t empty_bar[kStages];
  __shared__ ChunkMeta meta[kStages];

  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], NWARPS);
    }
    mbar_fence_init();
  }
  __syncthreads();

  // ===================== producer warp: TMA j-tiles into the ring ================
  if (tid >= NT) {
    if (tid != NT) return;
    int it = 0;
    bool ok = true;
    auto push = [&](const WorkItem &w, int cj0, int len, int flags) {
      const int st = it % kStages;
      const uint32_t par = ((it / kStages) & 1) ^ 1;
      if (!mbar_wait(&empty_bar[st], par, a.err)) {
        ok = false;
        return;
      }
      meta[st].item = w;
      meta[st].cj0 = cj0;
      meta[st].len = len;
      meta[st].flags = flags;
      if (flags & kChunkEnd) {
        mbar_arrive(&full_bar[st]);
      } else {
        if (PK) {
          // Packed layout: a tile of len sources is ceil(len/2) pairs of pf4
          // float4; an odd tail reads the pad particle after the system's last source.
          const bool lj = is_ljc(LAW) || (MIX && w.law != kLawGrav);
          const int pf4 = lj ? 3 : 2;
          const float4 *src = (MIX && lj) ? a.jpair2 : a.jpair;
          const uint32_t bytes = uint32_t((len + 1) >> 1) * pf4 * 16u;
          mbar_arrive_expect_tx(&full_bar[st], bytes);
          tma_load_1d(sm_pos + st * STAGE_F4,
                      src + size_t(w.pj0 + ((cj0 - w.j0) >> 1)) * size_t(pf4), bytes,
                      &full_bar[st]);
        } else {
          const uint32_t bytes = uint32_t(len) * 16u;
          const bool with_prm = is_ljc(LAW) || (MIX && w.law != kLawGrav);
          mbar_arrive_expect_tx(&full_bar[st], with_prm ? 2u * bytes : bytes);
          tma_load_1d(sm_pos + st * JT, a.pos + cj0, bytes, &full_bar[st]);
          if (with_prm) tma_load_1d(sm_prm + st * JT, a.prm + cj0, bytes, &full_bar[st]);
        }
      }
      ++it;
    };
    auto push_item = [&](const WorkItem &w) {
      const int jend = w.j0 + w.nj;
      for (int cj = w.j0; cj < jend && ok; cj += JT) {
        const int len = min(JT, jend - cj);
        int flags = 0;
        if (cj == w.j0) flags |= kChunkFirst;
        if (cj + len >= jend) flags |= kChunkLast;
        push(w, cj, len, flags);
      }
    };
    if (a.counter == nullptr) {
      const int b = blockIdx.x;
      WorkItem w;
      const int t = b / a.slices, s = b % a.slices;
      w.i0 = t * TI;
      w.ni = min(TI, a.n_t - w.i0);
      w.j0 = s * a.slice_len;
      w.nj = min(a.slice_len, a.n - w.j0);
      w.law = is_ljc(LAW) ? kLawLJC : kLawGrav;
      w.slice = s;
      w.eps2 = a.eps2;
      w.pj0 = w.j0 >> 1;
      if (w.ni > 0 && w.nj > 0) push_item(w);
      else set_error(a.err, kDevBadItem);
    } else {
      while (ok) {
        const int k = atomicAdd(a.counter, 1);
        if (k >= a.n_items) break;
        const WorkItem w = a.items[k];
        if (w.ni <= 0 || w.ni > TI || w.nj <= 0 || w.i0 < 0 || w.j0 < 0) {
          set_error(a.err, kDevBadItem);
          continue;
        }
        push_item(w);
      }
    }
    if (ok) {
      WorkItem none{};
      push(none, 0, 0, kChunkEnd);
    }
    if (!ok) {
      // Bounded drain of copies still in flight before leaving.
      for (int k = max(0, it - kStages); k < it; ++k)
        mbar_wait(&full_bar[k % kStages], (k / kStages) & 1, a.err);
    }
    return;
  }

  // ===================== consumer warps ===========================================
  const int warp = tid >> 5, lane = tid & 31;
  const int jl = (SW > 1) ? (lane % SW) : 0;
  const int slot = warp * (32 / SW) + lane / SW;

  float xi[I], yi[I], zi[I];
  float qi[I], si[I], ei[I];
  int ig[I];      // global index of each target (self mask)
  int slot_g[I];  // output slot of each target (-1: padding)
  float4 p[I], hi[I], lo[I];
  float2 pax[PK ? I : 1], pay[PK ? I : 1], paz[PK ? I : 1], ppt[PK ? I : 1];
  long long fxa[FX ? I : 1][4];
  const float fsc = FX ? __ldg(a.fscale) : 0.0f;
  WorkItem cur{};
  int cur_law = is_ljc(LAW) ? kLawLJC : kLawGrav;

  for (int it = 0;; ++it) {
    const int st = it % kStages;
    if (!mbar_wait(&full_bar[st], (it / kStages) & 1, a.err)) return;
    const int flags = meta[st].flags;
    if (flags & kChunkEnd) break;
    const int cj0 = meta[st].cj0;
    const int len = meta[st].len;
    if (flags & kChunkFirst) {
      cur = meta[st].item;
      if (LAW == kLawMixed) cur_law = cur.law;
#pragma unroll
      for (int r = 0; r < I; ++r) {
        const int il = r * SLOTS + slot;
        const int g = cur.i0 + min(il, cur.ni - 1);
        ig[r] = (il < cur.ni) ? (a.tidx ? __ldg(a.tidx + g) : g) : -1;
        slot_g[r] = (il < cur.ni) ? g : -1;
        const float4 pi4 = __ldg(a.tpos + g);
        xi[r] = pi4.x;
        yi[r] = pi4.y;
        zi[r] = pi4.z;
        if (T::kPrm && cur_law != kLawGrav) {
          const float4 pr = __ldg(a.tprm + g);
          qi[r] = pr.x;
          si[r] = pr.y;
          ei[r] = pr.z;
        } else {
          qi[r] = si[r] = ei[r] = 0.0f;
        }
        hi[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        lo[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        p[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (PK) pax[r] = pay[r] = paz[r] = ppt[r] = make_float2(0.f, 0.f);
        if (FX) fxa[r][0] = fxa[r][1] = fxa[r][2] = fxa[r][3] = 0;
      }
    }
    const float4 *sp = sm_pos + st * STAGE_F4;
    const float4 *sq = sm_prm + st * JT;
    const float eps2 = cur.eps2;
    const bool masked = a.tidx != nullptr || ((cj0 < cur.i0 + cur.ni) && (cur.i0 < cj0 + len));

    if (PK && (is_ljc(LAW) || (MIX && cur_law != kLawGrav))) {
      // L: the linear dielectric (fixed by LAW, or per item in the mixed kernel)
      auto ljc_chunk = [&](auto lin_tag) {
        constexpr bool L = decltype(lin_tag)::value;
        if (!masked) {
          const int npairs = (len + 1) >> 1;
          float2 nx[PK ? I : 1], ny[PK ? I : 1], nz[PK ? I : 1];
          float2 q2[PK ? I : 1], s2[PK ? I : 1], e2[PK ? I : 1];
#pragma unroll
          for (int r = 0; r < I; ++r) {
            nx[r] = make_float2(-xi[r], -xi[r]);
            ny[r] = make_float2(-yi[r], -yi[r]);
            nz[r] = make_float2(-zi[r], -zi[r]);
            q2[r] = make_float2(qi[r], qi[r]);
            s2[r] = make_float2(si[r], si[r]);
            e2[r] = make_float2(ei[r], ei[r]);
          }
#pragma unroll PU
          for (int pp = jl; pp < npairs; pp += SW) {
            const float4 A = sp[3 * pp];
            const float4 B = sp[3 * pp + 1];
            const float4 C = sp[3 * pp + 2];
#pragma unroll
            for (int r = 0; r < I; ++r)
              ljc_pair2<POT, PRECISE, L>(make_float2(A.x, A.y), make_float2(A.z, A.w),
                                      make_float2(B.x, B.y), make_float2(B.z, B.w),
                                      make_float2(C.x, C.y), make_float2(C.z, C.w), nx[r], ny[r],
                                      nz[r], q2[r], s2[r], e2[r], pax[r], pay[r], paz[r], ppt[r]);
          }
        } else {
          // Diagonal tile (or subset targets): the same pair loop with the self
          // source's term dropped by index.
          const int npairs = (len + 1) >> 1;
          for (int pp = jl; pp < npairs; pp += SW) {
            const float4 A = sp[3 * pp];
            const float4 B = sp[3 * pp + 1];
            const float4 C = sp[3 * pp + 2];
            const int jg = cj0 + 2 * pp;
#pragma unroll
            for (int r = 0; r < I; ++r)
              ljc_pair2<POT, PRECISE, L, true>(
                  make_float2(A.x, A.y), make_float2(A.z, A.w), make_float2(B.x, B.y),
                  make_float2(B.z, B.w), make_float2(C.x, C.y), make_float2(C.z, C.w),
                  make_float2(-xi[r], -xi[r]), make_float2(-yi[r], -yi[r]),
                  make_float2(-zi[r], -zi[r]), make_float2(qi[r], qi[r]),
                  make_float2(si[r], si[r]), make_float2(ei[r], ei[r]), pax[r], pay[r], paz[r],
                  ppt[r], jg == ig[r], jg + 1 == ig[r]);
          }
        }
      };
      if constexpr (MIX) {
        if (cur_law == kLawLJCLin) ljc_chunk(std::true_type{});
        else ljc_chunk(std::false_type{});
      } else {
        ljc_chunk(std::integral_constant<bool, LIN>{});
      }
    } else if (PK) {
      if (!masked) {
        const float2 e2 = make_float2(eps2, eps2);
        const int npairs = (len + 1) >> 1;
        float2 nx[PK ? I : 1], ny[PK ? I : 1], nz[PK ? I : 1];
#pragma unroll
        for (int r = 0; r < I; ++r) {
          nx[r] = make_float2(-xi[r], -xi[r]);
          ny[r] = make_float2(-yi[r], -yi[r]);
          nz[r] = make_float2(-zi[r], -zi[r]);
        }
#pragma unroll PU
        for (int pp = jl; pp < npairs; pp += SW) {
          const float4 A = sp[2 * pp];
          const float4 B = sp[2 * pp + 1];
          const float2 X = make_float2(A.x, A.y), Y = make_float2(A.z, A.w);
          const float2 Z = make_float2(B.x, B.y), M = make_float2(B.z, B.w);
#pragma unroll
          for (int r = 0; r < I; ++r)
            grav_pair2<POT, PRECISE>(X, Y, Z, M, nx[r], ny[r], nz[r], e2, pax[r], pay[r],
                                     paz[r], ppt[r]);
        }
      } else {
        // Diagonal tile (or subset targets): the same pair loop with the self
        // source's term dropped by index.
        const float2 e2 = make_float2(eps2, eps2);
        const int npairs = (len + 1) >> 1;
        for (int pp = jl; pp < npairs; pp += SW) {
          const float4 A = sp[2 * pp];
          const float4 B = sp[2 * pp + 1];
          const int jg = cj0 + 2 * pp;
#pragma unroll
          for (int r = 0; r < I; ++r)
            grav_pair2<POT, PRECISE, true>(
                make_float2(A.x, A.y), make_float2(A.z, A.w), make_float2(B.x, B.y),
                make_float2(B.z, B.w), make_float2(-xi[r], -xi[r]), make_float2(-yi[r], -yi[r]),
                make_float2(-zi[r], -zi[r]), e2, pax[r], pay[r], paz[r], ppt[r], jg == ig[r],
                jg + 1 == ig[r]);
        }
      }
    } else if (!T::kPrm || cur_law == kLawGrav) {
      if (!masked && len == JT) {
#pragma unroll 4
        for (int jj = jl; jj < JT; jj += SW) {
          const float4 pj = sp[jj];
#pragma unroll
          for (int r = 0; r < I; ++r)
            grav_pair<POT, PRECISE, false>(pj, xi[r], yi[r], zi[r], eps2, p[r], false);
        }
      } else if (!masked) {
#pragma unroll 2
        for (int jj = jl; jj < len; jj += SW) {
          const float4 pj = sp[jj];
#pragma unroll
          for (int r = 0; r < I; ++r)
            grav_pair<POT, PRECISE, false>(pj, xi[r], yi[r], zi[r], eps2, p[r], false);
        }
      } else {
        for (int jj = jl; jj < len; jj += SW) {
          const float4 pj = sp[jj];
          const int jg = cj0 + jj;
#pragma unroll
          for (int r = 0; r < I; ++r)
            grav_pair<POT, PRECISE, true>(pj, xi[r], yi[r], zi[r], eps2, p[r], jg == ig[r]);
        }
      }
    } else {
      auto ljc_chunk = [&](auto lin_tag) {
        constexpr bool L = decltype(lin_tag)::value;
        if (!masked && len == JT) {
#pragma unroll 2
          for (int jj = jl; jj < JT; jj += SW) {
            const float4 pj = sp[jj];
            const float4 qj = sq[jj];
#pragma unroll
            for (int r = 0; r < I; ++r)
              ljc_pair<POT, PRECISE, false, L>(pj, qj, xi[r], yi[r], zi[r], qi[r], si[r], ei[r],
                                            p[r], false);
          }
        } else if (!masked) {
          for (int jj = jl; jj < len; jj += SW) {
            const float4 pj = sp[jj];
            const float4 qj = sq[jj];
#pragma unroll
            for (int r = 0; r < I; ++r)
              ljc_pair<POT, PRECISE, false, L>(pj, qj, xi[r], yi[r], zi[r], qi[r], si[r], ei[r],
                                            p[r], false);
          }
        } else {
          for (int jj = jl; jj < len; jj += SW) {
            const float4 pj = sp[jj];
            const float4 qj = sq[jj];
            const int jg = cj0 + jj;
#pragma unroll
            for (int r = 0; r < I; ++r)
              ljc_pair<POT, PRECISE, true, L>(pj, qj, xi[r], yi[r], zi[r], qi[r], si[r], ei[r],
                                           p[r], jg == ig[r]);
          }
        }
      };
      if constexpr (MIX) {
        if (cur_law == kLawLJCLin) ljc_chunk(std::true_type{});
        else ljc_chunk(std::false_type{});
      } else {
        ljc_chunk(std::integral_constant<bool, LIN>{});
      }
    }

    // The stage has been read: hand it back to the producer.
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty_bar[st]);

    // Fold this j-tile's plain FP32 partial into the compensated (hi, lo).
#pragma unroll
    for (int r = 0; r < I; ++r) {
      if (PK) {
        // packed partial sums (diagonal tiles included) into the tile partial p
        p[r].x += pax[r].x + pax[r].y;
        p[r].y += pay[r].x + pay[r].y;
        p[r].z += paz[r].x + paz[r].y;
        if (POT) p[r].w += ppt[r].x + ppt[r].y;
        pax[r] = pay[r] = paz[r] = ppt[r] = make_float2(0.f, 0.f);
      }
      if (FX) {
        fxa[r][0] += __float2ll_rn(p[r].x * fsc);
        fxa[r][1] += __float2ll_rn(p[r].y * fsc);
        fxa[r][2] += __float2ll_rn(p[r].z * fsc);
        if (POT) fxa[r][3] += __float2ll_rn(p[r].w * fsc);
      } else if (a.comp) {
        comp_add(hi[r].x, lo[r].x, p[r].x);
        comp_add(hi[r].y, lo[r].y, p[r].y);
        comp_add(hi[r].z, lo[r].z, p[r].z);
        if (POT) comp_add(hi[r].w, lo[r].w, p[r].w);
      } else {
        hi[r].x += p[r].x;
        hi[r].y += p[r].y;
        hi[r].z += p[r].z;
        if (POT) hi[r].w += p[r].w;
      }
      p[r] = make_float4(0.f, 0.f, 0.f, 0.f);
    }

    if (flags & kChunkLast) {
      // Combine the SW j-lanes of each target: fixed butterfly, identical on
      // both partners of every exchange.
#pragma unroll
      for (int off = SW / 2; off >= 1; off >>= 1) {
#pragma unroll
        for (int r = 0; r < I; ++r) {
          if (FX) {
#pragma unroll
            for (int c = 0; c < 4; ++c) fxa[r][c] += __shfl_xor_sync(0xffffffffu, fxa[r][c], off);
            continue;
          }
          float4 oh, ol;
          oh.x = __shfl_xor_sync(0xffffffffu, hi[r].x, off);
          oh.y = __shfl_xor_sync(0xffffffffu, hi[r].y, off);
          oh.z = __shfl_xor_sync(0xffffffffu, hi[r].z, off);
          oh.w = __shfl_xor_sync(0xffffffffu, hi[r].w, off);
          ol.x = __shfl_xor_sync(0xffffffffu, lo[r].x, off);
          ol.y = __shfl_xor_sync(0xffffffffu, lo[r].y, off);
          ol.z = __shfl_xor_sync(0xffffffffu, lo[r].z, off);
          ol.w = __shfl_xor_sync(0xffffffffu, lo[r].w, off);
          float e;
          two_sum(hi[r].x, oh.x, hi[r].x, e);
          lo[r].x = __fadd_rn(__fadd_rn(lo[r].x, ol.x), e);
          two_sum(hi[r].y, oh.y, hi[r].y, e);
          lo[r].y = __fadd_rn(__fadd_rn(lo[r].y, ol.y), e);
          two_sum(hi[r].z, oh.z, hi[r].z, e);
          lo[r].z = __fadd_rn(__fadd_rn(lo[r].z, ol.z), e);
          two_sum(hi[r].w, oh.w, hi[r].w, e);
          lo[r].w = __fadd_rn(__fadd_rn(lo[r].w, ol.w), e);
        }
      }
      if (jl == 0) {
        const long long base = (long long)cur.slice * a.stride;
#pragma unroll
        for (int r = 0; r < I; ++r) {
          if (slot_g[r] >= 0) {
            if (FX) {  // four int64 per target: (x, y) in part_hi, (z, w) in part_lo
              long long *ph = reinterpret_cast<long long *>(a.part_hi) + 2 * (base + slot_g[r]);
              long long *pl = reinterpret_cast<long long *>(a.part_lo) + 2 * (base + slot_g[r]);
              ph[0] = fxa[r][0];
              ph[1] = fxa[r][1];
              pl[0] = fxa[r][2];
              pl[1] = fxa[r][3];
            } else {
              a.part_hi[base + slot_g[r]] = hi[r];
              a.part_lo[base + slot_g[r]] = lo[r];
            }
          }
        }
      }
    }
  }
}

}  // namespace nbody
