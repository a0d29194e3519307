// api_adjoint.cu -- C-ABI entry points of the reverse-mode path: one force VJP
// (nbody_adjoint) and the reverse leapfrog sweep over stored positions
// (nbody_adjoint_leapfrog). Kernels in vjp_kernel.cuh and vjp_aux.cuh; tile
// tables in vjp_tiles.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <initializer_list>
#include <cmath>

#include "api_common.h"
#include "vjp_aux.cuh"
#include "vjp_kernel.cuh"
#include "vjp_tiles.h"

using namespace nbody;

namespace {

struct VjpScratch {
  float4 *part_hi, *part_lo, *u, *jp;
  char *extra;  // caller-requested extra bytes
  double *type_part;
  int slices, slice_len, grid, nblk;
  long long bstride;
  const VjpDesc *d;
  int sym_split;  // symmetric gravity VJP: source parts per block (1 otherwise)
  // symmetric gravity VJP in exact fixed point (null otherwise): eight int64
  // accumulators per particle, four doubles per interleave block for the scale's
  // reductions, and the arena header's ticket, scale and inverse-scale words
  long long *acc64;
  double *vpart;
  unsigned *ticket;
  float *fscale;
  double *finv;
};

// When the symmetric gravity VJP (and, with the same params, acceleration + jerk)
// adds its per-block partials in exact fixed point (its scale needs a bound:
// eps > 0): 2 always (NBODY_FIXED_POINT), 1 only where
// one partial per particle, block and part would pass the partial-sum cap (at
// N = 16384 and 65536 the slots measured 2-5% faster: eight integer atomics per
// particle and CTA cost more than the slot writes and their read-back), 0 never
// (no softening, or NBODY_NO_COMPENSATION without NBODY_FIXED_POINT).
int vjp_atomic_mode(const nbody_params &p) {
  if (p.law != NBODY_LAW_GRAV || !(p.eps2 > 0.0f)) return 0;
  if (p.flags & NBODY_FIXED_POINT) return 2;
  return (p.flags & NBODY_NO_COMPENSATION) ? 0 : 1;
}

// Tile table of a VJP-kernel law (gravity VJP, LJC VJP, acceleration + jerk).
int vjp_table(int law) {
  if (law == kLawGAJ) return kTableJerk;
  if (law == NBODY_LAW_LJC_LINEAR) return kTableVjpLJCLin;
  return law == NBODY_LAW_LJC ? kTableVjpLJC : kTableVjpGrav;
}

// Tile (params tile >= 0, else the tuned or default row of the law's table)
// and j-split (params jsplit > 0, else the tuned one, else the split whose
// items best fill whole waves of resident CTAs), then the scratch layout.
// atomic_mode (vjp_atomic_mode): whether a symmetric gravity VJP tile accumulates
// in exact fixed point; it then needs 64 B of scratch per particle instead of one
// slot per particle, block and part, and has no partial-sum cap.
int vjp_prepare(int law, int n, int tile, int jsplit, int sms, cudaStream_t s, VjpScratch *sc,
                size_t extra = 0, int atomic_mode = 0) {
  const int table = vjp_table(law);
  int count = 0;
  const VjpDesc *tiles = vjp_tiles(table, &count);
  int tj = 0;
  const bool tuned = tile < 0;
  if (tuned) get_config(table, n, &tile, &tj);
  if (jsplit <= 0) jsplit = tj;
  if (!tiles || tile < 0 || tile >= count)
    return set_error_msg(NBODY_EINVAL, "bad tile %d for table %d", tile, table);
  const bool atomic = (law == NBODY_LAW_GRAV || law == kLawGAJ) && tiles[tile].sym &&
                     (atomic_mode == 2 ||
                      (atomic_mode == 1 && !sym_fits(n, tiles[tile].tile_i)));
  if (tiles[tile].sym && !atomic && !sym_fits(n, tiles[tile].tile_i)) {
    if (tuned)  // a tuned symmetric entry above the cap: the default tile instead
      return vjp_prepare(law, n, default_tile(table, n), 0, sms, s, sc, extra, atomic_mode);
    return set_error_msg(NBODY_EINVAL, "n = %d too large for symmetric tile %d", n, tile);
  }
  const VjpDesc &d = tiles[tile];
  sc->acc64 = nullptr;
  sc->vpart = nullptr;
  if (d.sym) {  // one CTA per block pair (and source part), one slot per block (and part)
    const int nb = (n + d.tile_i - 1) / d.tile_i;
    const bool lj = (law == NBODY_LAW_LJC || law == NBODY_LAW_LJC_LINEAR);
    const int nblocks = (law == kLawGAJ || lj) ? 2 : 1;  // two partial blocks
    // the gravity VJP takes the source split of the force tiles (j-split rounded down
    // to a power of two of at most 8, parts of at least 32 source pairs)
    const int max_split = (law == NBODY_LAW_GRAV) ? std::min(8, std::max(1, d.tile_i / 64)) : 1;
    int S = 1;
    while (jsplit > 0 && S * 2 <= std::min(jsplit, max_split)) S *= 2;
    const long long pairs = (long long)nb * (nb + 1) / 2;
    if (pairs * S > 0x7fffffffLL)
      return set_error_msg(NBODY_EINVAL, "n = %d too large for symmetric tile %d split %d", n,
                           tile, S);
    // the partials: one float4 slot per particle, block and part, or the int64
    // fixed-point accumulators per particle (8 for the VJP, 16 for acceleration
    // and jerk)
    const size_t part =
        atomic ? round_up(size_t(8 * nblocks) * size_t(n) * sizeof(long long), 256)
               : round_up(size_t(nblocks) * size_t(nb) * S * size_t(n) * sizeof(float4), 256);
    const size_t ubytes = round_up(size_t(n) * sizeof(float4), 256);
    const int nblk = (n + 255) / 256;
    const size_t tbytes = round_up(size_t(nblk) * 8 * sizeof(double), 256);
    const int pair_f4 = lj ? 5 : 4;  // float4 per source pair in the blocked layout
    const size_t jbytes =
        round_up(size_t(nb) * (d.tile_i / 2) * pair_f4 * sizeof(float4), 256);
    const int pblocks = ((n + 1) / 2 + 255) / 256;  // interleave blocks
    const size_t vbytes = atomic ? round_up(size_t(pblocks) * 4 * sizeof(double), 256) : 0;
    void *base = nullptr;
    char *hdr = nullptr;
    NB_TRY(workspace(s, part + ubytes + tbytes + jbytes + vbytes + extra, &base, &hdr));
    char *b = static_cast<char *>(base);
    sc->part_hi = reinterpret_cast<float4 *>(b);
    sc->part_lo = nullptr;
    sc->u = reinterpret_cast<float4 *>(b + part);
    sc->type_part = reinterpret_cast<double *>(b + part + ubytes);
    sc->jp = reinterpret_cast<float4 *>(b + part + ubytes + tbytes);
    sc->extra = b + part + ubytes + tbytes + jbytes + vbytes;
    if (atomic) {  // header words 32-55 (the force path's are 0-23)
      sc->acc64 = reinterpret_cast<long long *>(b);
      sc->part_hi = nullptr;
      sc->vpart = reinterpret_cast<double *>(b + part + ubytes + tbytes + jbytes);
      sc->fscale = reinterpret_cast<float *>(hdr + 32);
      sc->finv = reinterpret_cast<double *>(hdr + 40);
      sc->ticket = reinterpret_cast<unsigned *>(hdr + 48);
    }
    sc->slices = nb * S;
    sc->slice_len = d.tile_i / S;
    sc->grid = int(pairs * S);
    sc->nblk = nblk;
    sc->bstride = (long long)nb * S * n;
    sc->d = &d;
    sc->sym_split = S;
    return NBODY_OK;
  }
  const int n_it = (n + d.tile_i - 1) / d.tile_i;
  const int cap = sms * d.occupancy();
  const int max_s = (n + d.jt - 1) / d.jt;
  int S = 1;
  if (jsplit > 0) {
    S = std::min(jsplit, max_s);
  } else {
    double best = -1.0;
    for (int k = 1; k <= 64 && k <= max_s; ++k) {
      const int len = int(round_up(size_t((n + k - 1) / k), size_t(d.jt)));
      const int kk = (n + len - 1) / len;
      const double waves = double(n_it) * kk / cap;
      const double score = waves / std::ceil(waves) - 0.002 * kk;
      if (score > best + 1e-12) {
        best = score;
        S = kk;
      }
    }
  }
  const int len = int(round_up(size_t((n + S - 1) / S), size_t(d.jt)));
  S = (n + len - 1) / len;
  const bool ljc = (law == NBODY_LAW_LJC || law == NBODY_LAW_LJC_LINEAR);
  const int blocks = (ljc || law == kLawGAJ) ? 2 : 1;
  const size_t part = round_up(size_t(blocks) * S * size_t(n) * sizeof(float4), 256);
  const size_t ubytes = round_up(size_t(n) * sizeof(float4), 256);
  const int nblk = (n + 255) / 256;
  const size_t tbytes = round_up(size_t(nblk) * 8 * sizeof(double), 256);
  const int pair_f4 = ljc ? 5 : 4;  // float4s per packed source pair
  const size_t jbytes =
      d.packed ? round_up(size_t((n + 1) / 2) * pair_f4 * sizeof(float4), 256) : 0;
  void *base = nullptr;
  NB_TRY(workspace(s, 2 * part + ubytes + tbytes + jbytes + extra, &base));
  char *b = static_cast<char *>(base);
  sc->extra = b + 2 * part + ubytes + tbytes + jbytes;
  sc->jp = d.packed ? reinterpret_cast<float4 *>(b + 2 * part + ubytes + tbytes) : nullptr;
  sc->part_hi = reinterpret_cast<float4 *>(b);
  sc->part_lo = reinterpret_cast<float4 *>(b + part);
  sc->u = reinterpret_cast<float4 *>(b + 2 * part);
  sc->type_part = reinterpret_cast<double *>(b + 2 * part + ubytes);
  sc->slices = S;
  sc->slice_len = len;
  sc->grid = n_it * S;
  sc->nblk = nblk;
  sc->bstride = (long long)S * n;
  sc->d = &d;
  sc->sym_split = 1;
  return NBODY_OK;
}

// One VJP: all-pairs kernel + finalize (+ type reduction). chained: the previous
// operation in `s` is a kernel of this library issued by the same call, so every
// launch here may be a programmatic dependent launch (otherwise all but the first).
int vjp_once(const float4 *pos, const float4 *prm, const float4 *lam, float4 *grad_x,
             float *grad_m, double *grad_types, int ntypes, float alpha, int accumulate, int n,
             const nbody_params &p, const VjpScratch &sc, float4 *lam_v, float dt_next,
             cudaStream_t s, bool chained) {
  int *err = nullptr;
  NB_TRY(error_word(&err));
  const float4 *src = lam;
  const bool ljc = (p.law == NBODY_LAW_LJC || p.law == NBODY_LAW_LJC_LINEAR);
  if (ljc) {
    NB_CUDA(launch_kernel(lam_over_m_kernel, (n + 255) / 256, 256, 0, s, chained, lam, pos,
                          sc.u, n));
    chained = true;
    src = sc.u;
  }
  if (sc.d->packed) {
    const int pblocks = ((n + 1) / 2 + 255) / 256;
    if (sc.d->sym && ljc)
      NB_CUDA(launch_kernel(interleave_ljc_vjp_pairs_blocked_kernel, pblocks, 256, 0, s, chained,
                            pos, src, prm, sc.jp, n, sc.d->tile_i));
    else if (sc.d->sym)
      NB_CUDA(launch_kernel(interleave_vjp_pairs_blocked_kernel, pblocks, 256, 0, s, chained,
                            pos, src, sc.jp, n, sc.d->tile_i,
                            VjpAtomicPrep{sc.acc64, sc.vpart, sc.ticket, p.eps2, sc.fscale,
                                          sc.finv, 0, 8}));
    else if (ljc)
      NB_CUDA(launch_kernel(interleave_ljc_vjp_pairs_kernel, pblocks, 256, 0, s, chained, pos,
                            src, prm, sc.jp, n));
    else
      NB_CUDA(launch_kernel(interleave_vjp_pairs_kernel, pblocks, 256, 0, s, chained, pos, src,
                            sc.jp, n));
    chained = true;
  }
  VjpArgs a{};
  a.pos = pos;
  a.lam = src;
  a.prm = prm;
  a.jpair = sc.jp;
  a.part_hi = sc.part_hi;
  a.part_lo = sc.part_lo;
  a.stride = n;
  a.bstride = sc.bstride;
  a.err = err;
  a.n = n;
  a.slices = sc.slices;
  a.slice_len = sc.slice_len;
  a.eps2 = p.eps2;
  a.comp = (p.flags & NBODY_NO_COMPENSATION) ? 0 : 1;
  a.pdl = chained ? 1 : 0;
  a.acc64 = sc.acc64;
  a.fscale = sc.acc64 ? sc.fscale : nullptr;
  const TimerMark tm = timer_begin(1, s);
  cudaError_t e = sc.d->launch(a, sc.grid, s);
  timer_end(tm, s);
  if (e != cudaSuccess)
    return set_error_msg(NBODY_ECUDA, "VJP kernel launch failed: %s", cudaGetErrorString(e));
  VjpFinalizeArgs f{};
  f.part_hi = sc.part_hi;
  f.part_lo = sc.part_lo;
  f.stride = n;
  f.bstride = sc.bstride;
  f.slices = sc.slices;
  f.sym_block = sc.d->sym ? sc.d->tile_i : 0;
  f.sym_split = sc.sym_split;
  f.n = n;
  f.law = p.law;
  f.G = p.G;
  f.alpha = alpha;
  f.pos = pos;
  f.prm = prm;
  f.lam = src;
  f.grad_x = grad_x;
  f.grad_m = grad_m;
  f.accumulate = accumulate;
  const bool types = grad_types && ljc;
  f.type_part = types ? sc.type_part : nullptr;
  f.lam_v = lam_v;
  f.dt_next = dt_next;
  f.acc64 = sc.acc64;
  f.fx_inv = sc.acc64 ? sc.finv : nullptr;
  NB_CUDA(launch_kernel(vjp_finalize_kernel, sc.nblk, 256, 0, s, true, f));
  if (types)
    NB_CUDA(launch_kernel(type_reduce_kernel, 1, 32, 0, s, true, sc.type_part, sc.nblk, ntypes,
                          grad_types));
  return NBODY_OK;
}

int check_common(const nbody_params *p, const void *pos, const void *prm, int64_t n,
                 int ntypes, const double *grad_types) {
  if (!p) return set_error_msg(NBODY_EINVAL, "params is NULL");
  if (p->law != NBODY_LAW_GRAV && p->law != NBODY_LAW_LJC && p->law != NBODY_LAW_LJC_LINEAR)
    return set_error_msg(NBODY_EINVAL, "unknown law %d", p->law);
  if (n < 0 || n > 0x7fffffffLL) return set_error_msg(NBODY_EINVAL, "n out of range");
  if (!pos) return set_error_msg(NBODY_EINVAL, "pos_m is NULL");
  if (p->law != NBODY_LAW_GRAV && !prm) return set_error_msg(NBODY_EINVAL, "LJC needs prm");
  if (grad_types && (ntypes < 1 || ntypes > 4))
    return set_error_msg(NBODY_EUNSUPPORTED, "per-type gradients support 1..4 types");
  if (!(p->eps2 >= 0.0f)) return set_error_msg(NBODY_EINVAL, "eps2 must be >= 0");
  if ((p->flags & NBODY_FIXED_POINT) && (p->law != NBODY_LAW_GRAV || !(p->eps2 > 0.0f)))
    return set_error_msg(NBODY_EINVAL, "fixed-point accumulation needs gravity with eps2 > 0");
  return NBODY_OK;
}

int check_dev(const void *q, const char *name, bool required) {
  if (!q) return required ? set_error_msg(NBODY_EINVAL, "%s is NULL", name) : NBODY_OK;
  if (!aligned16(q)) return set_error_msg(NBODY_EALIGN, "%s is not 16-byte aligned", name);
  return NBODY_OK;
}

int check_dev_ptrs(std::initializer_list<const void *> ptrs) {
  for (const void *q : ptrs)
    if (q && is_host_pointer(q)) return set_error_msg(NBODY_EINVAL, "device pointers only");
  return NBODY_OK;
}

// Hermite predictor: x_p = x + dt (v + dt (a/2 + dt j/6)), v_p = v + dt (a + dt j/2).
__global__ void hermite_predict_kernel(const float4 *pos, const float4 *vel, const float4 *acc,
                                       const float4 *jerk, float dt, int n, float4 *xp,
                                       float4 *vp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 x = pos[i], v = vel[i], a = acc[i], j = jerk[i];
  const float h2 = 0.5f * dt, h6 = dt * (1.0f / 6.0f);
  xp[i] = make_float4(fmaf(dt, fmaf(dt, fmaf(h6, j.x, 0.5f * a.x), v.x), x.x),
                      fmaf(dt, fmaf(dt, fmaf(h6, j.y, 0.5f * a.y), v.y), x.y),
                      fmaf(dt, fmaf(dt, fmaf(h6, j.z, 0.5f * a.z), v.z), x.z), x.w);
  vp[i] = make_float4(fmaf(dt, fmaf(h2, j.x, a.x), v.x), fmaf(dt, fmaf(h2, j.y, a.y), v.y),
                      fmaf(dt, fmaf(h2, j.z, a.z), v.z), 0.0f);
}

// Hermite corrector (time-symmetric form):
//   v1 = v + dt/2 (a + a1) + dt^2/12 (j - j1),  x1 = x + dt/2 (v + v1) + dt^2/12 (a - a1)
__global__ void hermite_correct_kernel(float4 *pos, float4 *vel, float4 *acc, float4 *jerk,
                                       const float4 *a1v, const float4 *j1v, float dt, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 x = pos[i], v = vel[i], a = acc[i], j = jerk[i], a1 = a1v[i], j1 = j1v[i];
  const float h = 0.5f * dt, q = dt * dt * (1.0f / 12.0f);
  float4 v1, x1;
  v1.x = fmaf(q, j.x - j1.x, fmaf(h, a.x + a1.x, v.x));
  v1.y = fmaf(q, j.y - j1.y, fmaf(h, a.y + a1.y, v.y));
  v1.z = fmaf(q, j.z - j1.z, fmaf(h, a.z + a1.z, v.z));
  v1.w = v.w;
  x1.x = fmaf(q, a.x - a1.x, fmaf(h, v.x + v1.x, x.x));
  x1.y = fmaf(q, a.y - a1.y, fmaf(h, v.y + v1.y, x.y));
  x1.z = fmaf(q, a.z - a1.z, fmaf(h, v.z + v1.z, x.z));
  x1.w = x.w;
  pos[i] = x1;
  vel[i] = v1;
  acc[i] = a1;
  jerk[i] = j1;
}

// Acceleration and jerk at (pos, vel) into (acc, jerk): GAJ kernel + finalize.
int gaj_eval(const float4 *pos, const float4 *vel, float4 *acc, float4 *jerk, int n,
             const nbody_params &p, const VjpScratch &sc, cudaStream_t s) {
  int *err = nullptr;
  NB_TRY(error_word(&err));
  if (sc.d->packed) {  // (x, m) and velocities of source pairs, interleaved
    const unsigned pblocks = unsigned(((n + 1) / 2 + 255) / 256);
    if (sc.d->sym)
      interleave_vjp_pairs_blocked_kernel<<<pblocks, 256, 0, s>>>(
          pos, vel, sc.jp, n, sc.d->tile_i,
          VjpAtomicPrep{sc.acc64, sc.vpart, sc.ticket, p.eps2, sc.fscale, sc.finv, 1, 16});
    else
      interleave_vjp_pairs_kernel<<<pblocks, 256, 0, s>>>(pos, vel, sc.jp, n);
    NB_CUDA(cudaGetLastError());
  }
  VjpArgs a{};
  a.pos = pos;
  a.lam = vel;
  a.jpair = sc.jp;
  a.part_hi = sc.part_hi;
  a.part_lo = sc.part_lo;
  a.stride = n;
  a.bstride = sc.bstride;
  a.err = err;
  a.n = n;
  a.slices = sc.slices;
  a.slice_len = sc.slice_len;
  a.eps2 = p.eps2;
  a.comp = (p.flags & NBODY_NO_COMPENSATION) ? 0 : 1;
  a.acc64 = sc.acc64;
  a.fscale = sc.acc64 ? sc.fscale : nullptr;
  const TimerMark tm = timer_begin(0, s);
  cudaError_t e = sc.d->launch(a, sc.grid, s);
  timer_end(tm, s);
  if (e != cudaSuccess)
    return set_error_msg(NBODY_ECUDA, "jerk kernel launch failed: %s", cudaGetErrorString(e));
  gaj_finalize_kernel<<<unsigned((n + 255) / 256), 256, 0, s>>>(
      sc.part_hi, sc.part_lo, n, sc.bstride, sc.slices, n, p.G, acc, jerk, sc.acc64,
      sc.acc64 ? sc.finv : nullptr);
  NB_CUDA(cudaGetLastError());
  return NBODY_OK;
}

int check_jerk_params(const nbody_params *params, uint32_t extra_flags) {
  if (!params) return set_error_msg(NBODY_EINVAL, "params is NULL");
  const nbody_params &p = *params;
  if (p.law != NBODY_LAW_GRAV)
    return set_error_msg(NBODY_EINVAL, "acceleration + jerk is defined for gravity only");
  if (p.flags & ~(uint32_t)(NBODY_NO_COMPENSATION | NBODY_FIXED_POINT | extra_flags))
    return set_error_msg(NBODY_EUNSUPPORTED, "unsupported flag bits 0x%x", p.flags);
  if (!(p.eps2 >= 0.0f) || !std::isfinite(p.G))
    return set_error_msg(NBODY_EINVAL, "bad G or eps2");
  if ((p.flags & NBODY_FIXED_POINT) && !(p.eps2 > 0.0f))
    return set_error_msg(NBODY_EINVAL, "fixed-point accumulation needs eps2 > 0");
  return NBODY_OK;
}

}  // namespace

extern "C" {

int nbody_adjoint(const void *pos_m, const void *prm, const void *lam, void *grad_x,
                  float *grad_m, double *grad_types, int32_t ntypes, float alpha, int64_t n,
                  const nbody_params *params, nbody_stream_t stream) {
  clear_error();
  const NvtxRange nvtx_range("nbody_adjoint");
  NB_TRY(check_common(params, pos_m, prm, n, ntypes, grad_types));
  NB_TRY(check_dev(pos_m, "pos_m", true));
  NB_TRY(check_dev(lam, "lam", true));
  NB_TRY(check_dev(grad_x, "grad_x", true));
  NB_TRY(check_dev(prm, "prm", false));
  if (grad_m && (reinterpret_cast<uintptr_t>(grad_m) & 3u))
    return set_error_msg(NBODY_EALIGN, "grad_m is not 4-byte aligned");
  if (!std::isfinite(alpha)) return set_error_msg(NBODY_EINVAL, "alpha must be finite");
  if (n == 0) return NBODY_OK;
  int dev = 0, sms = 0;
  NB_TRY(check_device(&dev, &sms));
  NB_TRY(check_dev_ptrs({pos_m, prm, lam, grad_x, grad_m, grad_types}));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const nbody_params p = *params;
  VjpScratch sc{};
  NB_TRY(vjp_prepare(p.law, int(n), p.tile, p.jsplit, sms, s, &sc, 0, vjp_atomic_mode(p)));
  const int acc = (p.flags & NBODY_ACCUMULATE) ? 1 : 0;
  bool launched = false;
  if (grad_types && !acc && p.law != NBODY_LAW_GRAV) {
    zero_doubles_kernel<<<1, 32, 0, s>>>(grad_types, 2 * ntypes);
    NB_CUDA(cudaGetLastError());
    launched = true;
  }
  return vjp_once(static_cast<const float4 *>(pos_m), static_cast<const float4 *>(prm),
                  static_cast<const float4 *>(lam), static_cast<float4 *>(grad_x), grad_m,
                  grad_types, ntypes, alpha, acc, int(n), p, sc, nullptr, 0.0f, s, launched);
}

int nbody_adjoint_leapfrog(const void *xs, const void *prm, int64_t n, int32_t k, float dt,
                           int32_t first, void *lam_x, void *lam_v, float *grad_m,
                           double *grad_types, int32_t ntypes, const nbody_params *params,
                           nbody_stream_t stream) {
  clear_error();
  const NvtxRange nvtx_range("nbody_adjoint_leapfrog");
  NB_TRY(check_common(params, xs, prm, n, ntypes, grad_types));
  if (k < 0) return set_error_msg(NBODY_EINVAL, "k must be >= 0");
  if (!std::isfinite(dt)) return set_error_msg(NBODY_EINVAL, "dt must be finite");
  NB_TRY(check_dev(xs, "xs", true));
  NB_TRY(check_dev(lam_x, "lam_x", true));
  NB_TRY(check_dev(lam_v, "lam_v", true));
  NB_TRY(check_dev(prm, "prm", false));
  if (n == 0 || k == 0) return NBODY_OK;
  int dev = 0, sms = 0;
  NB_TRY(check_device(&dev, &sms));
  NB_TRY(check_dev_ptrs({xs, prm, lam_x, lam_v, grad_m, grad_types}));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const nbody_params p = *params;
  VjpScratch sc{};
  NB_TRY(vjp_prepare(p.law, int(n), p.tile, p.jsplit, sms, s, &sc, 0, vjp_atomic_mode(p)));
  float4 *lx = static_cast<float4 *>(lam_x);
  float4 *lv = static_cast<float4 *>(lam_v);
  const float4 *X = static_cast<const float4 *>(xs);
  const float4 *q = static_cast<const float4 *>(prm);
  // First reverse drift of the chunk: lam_v += dt lam_x.
  axpy4_kernel<<<unsigned((n + 255) / 256), 256, 0, s>>>(dt, lx, lv, int(n));
  NB_CUDA(cudaGetLastError());
  for (int st = k - 1; st >= 0; --st) {
    const float w = (st == 0 && first) ? 0.5f * dt : dt;
    // lam_x += w J(x_st)^T lam_v, then (except after the last) lam_v += dt lam_x.
    NB_TRY(vjp_once(X + size_t(st) * size_t(n), q, lv, lx, grad_m, grad_types, ntypes, w, 1,
                    int(n), p, sc, st > 0 ? lv : nullptr, dt, s, true));
  }
  return NBODY_OK;
}

int nbody_forces_jerk(const void *pos_m, const void *vel, void *acc, void *jerk, int64_t n,
                      const nbody_params *params, nbody_stream_t stream) {
  clear_error();
  const NvtxRange nvtx_range("nbody_forces_jerk");
  NB_TRY(check_jerk_params(params, 0));
  if (n < 0 || n > 0x7fffffffLL) return set_error_msg(NBODY_EINVAL, "n out of range");
  if (n == 0) return NBODY_OK;
  NB_TRY(check_dev(pos_m, "pos_m", true));
  NB_TRY(check_dev(vel, "vel", true));
  NB_TRY(check_dev(acc, "acc", true));
  NB_TRY(check_dev(jerk, "jerk", true));
  int dev = 0, sms = 0;
  NB_TRY(check_device(&dev, &sms));
  NB_TRY(check_dev_ptrs({pos_m, vel, acc, jerk}));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  VjpScratch sc{};
  NB_TRY(vjp_prepare(kLawGAJ, int(n), params->tile, params->jsplit, sms, s, &sc, 0,
                     vjp_atomic_mode(*params)));
  return gaj_eval(static_cast<const float4 *>(pos_m), static_cast<const float4 *>(vel),
                  static_cast<float4 *>(acc), static_cast<float4 *>(jerk), int(n), *params, sc, s);
}

int nbody_hermite_step(void *pos_m, void *vel, void *acc, void *jerk, int64_t n, float dt,
                       int32_t nsteps, const nbody_params *params, nbody_stream_t stream) {
  clear_error();
  const NvtxRange nvtx_range("nbody_hermite_step");
  NB_TRY(check_jerk_params(params, NBODY_ACC_VALID));
  if (n < 0 || n > 0x7fffffffLL) return set_error_msg(NBODY_EINVAL, "n out of range");
  if (nsteps < 0) return set_error_msg(NBODY_EINVAL, "nsteps must be >= 0");
  if (!std::isfinite(dt)) return set_error_msg(NBODY_EINVAL, "dt must be finite");
  if (n == 0) return NBODY_OK;
  NB_TRY(check_dev(pos_m, "pos_m", true));
  NB_TRY(check_dev(vel, "vel", true));
  NB_TRY(check_dev(acc, "acc", true));
  NB_TRY(check_dev(jerk, "jerk", true));
  int dev = 0, sms = 0;
  NB_TRY(check_device(&dev, &sms));
  NB_TRY(check_dev_ptrs({pos_m, vel, acc, jerk}));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // scratch: GAJ partials, then predicted (x, v) and the new (a, j)
  VjpScratch sc{};
  const size_t q = round_up(size_t(n) * sizeof(float4), 256);
  NB_TRY(vjp_prepare(kLawGAJ, int(n), params->tile, params->jsplit, sms, s, &sc, 4 * q,
                     vjp_atomic_mode(*params)));
  float4 *xp = reinterpret_cast<float4 *>(sc.extra);
  float4 *vp = reinterpret_cast<float4 *>(sc.extra + q);
  float4 *a1 = reinterpret_cast<float4 *>(sc.extra + 2 * q);
  float4 *j1 = reinterpret_cast<float4 *>(sc.extra + 3 * q);
  float4 *X = static_cast<float4 *>(pos_m);
  float4 *V = static_cast<float4 *>(vel);
  float4 *A = static_cast<float4 *>(acc);
  float4 *J = static_cast<float4 *>(jerk);
  const int nn = int(n);
  if (!(params->flags & NBODY_ACC_VALID)) NB_TRY(gaj_eval(X, V, A, J, nn, *params, sc, s));
  const unsigned blocks = unsigned((n + 255) / 256);
  for (int st = 0; st < nsteps; ++st) {
    hermite_predict_kernel<<<blocks, 256, 0, s>>>(X, V, A, J, dt, nn, xp, vp);
    NB_CUDA(cudaGetLastError());
    NB_TRY(gaj_eval(xp, vp, a1, j1, nn, *params, sc, s));
    hermite_correct_kernel<<<blocks, 256, 0, s>>>(X, V, A, J, a1, j1, dt, nn);
    NB_CUDA(cudaGetLastError());
  }
  return NBODY_OK;
}

}  // extern "C"
