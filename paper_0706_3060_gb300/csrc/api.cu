// api.cu -- C-ABI entry points for single systems: pack, forces, leapfrog steps,
// tile queries and library housekeeping (declared in include/nbody.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "api_common.h"
#include "aux_kernels.cuh"

using namespace nbody;

namespace nbody {

int launch_finalize(const FinalizeArgs &f, cudaStream_t s, int *nblk_out, bool pdl) {
  const int nblk = std::max(1, (f.n + kFinThreads - 1) / kFinThreads);
  NB_CUDA(launch_kernel(finalize_kernel, nblk, kFinThreads, 0, s, pdl, f));
  if (nblk_out) *nblk_out = nblk;
  return NBODY_OK;
}

int launch_kick_drift(float4 *pos, float4 *vel, const float4 *acc, int n, float dt,
                      float4 *trace1, const int *sys_of, const void *sys, float4 *x_lo,
                      float4 *v_lo, cudaStream_t s) {
  if (n <= 0) return NBODY_OK;
  kick_drift_kernel<<<(n + 255) / 256, 256, 0, s>>>(pos, vel, acc, n, dt, trace1, sys_of,
                                                    static_cast<const SysInfo *>(sys), x_lo, v_lo);
  NB_CUDA(cudaGetLastError());
  return NBODY_OK;
}

}  // namespace nbody

namespace {

constexpr int kMaxN = 0x7fffffff;

// Tile table of a call: the law's own, or the fixed-point gravity table.
int table_of(const nbody_params &p) {
  return (p.flags & NBODY_FIXED_POINT) ? kTableGravFixed : p.law;
}

int check_params(const nbody_params *p, const void *prm) {
  if (!p) return set_error_msg(NBODY_EINVAL, "params is NULL");
  if (p->law != NBODY_LAW_GRAV && p->law != NBODY_LAW_LJC && p->law != NBODY_LAW_LJC_LINEAR)
    return set_error_msg(NBODY_EINVAL, "unknown law %d", p->law);
  const uint32_t known = NBODY_COMPUTE_POT | NBODY_PRECISE_RSQRT | NBODY_NO_COMPENSATION |
                         NBODY_ACC_VALID | NBODY_ACCUMULATE | NBODY_FIXED_POINT;
  if (p->flags & ~known) return set_error_msg(NBODY_EINVAL, "unknown flag bits 0x%x", p->flags);
  if (p->law != NBODY_LAW_GRAV && !prm)
    return set_error_msg(NBODY_EINVAL, "LJC law needs the prm array");
  if (p->law == NBODY_LAW_GRAV && !(p->eps2 >= 0.0f))
    return set_error_msg(NBODY_EINVAL, "eps2 must be >= 0");
  if (p->law == NBODY_LAW_GRAV && !std::isfinite(p->G))
    return set_error_msg(NBODY_EINVAL, "G must be finite");
  if (p->flags & NBODY_FIXED_POINT) {
    if (p->law != NBODY_LAW_GRAV)
      return set_error_msg(NBODY_EUNSUPPORTED, "fixed-point accumulation is for gravity only");
    if (!(p->eps2 > 0.0f))
      return set_error_msg(NBODY_EINVAL, "fixed-point accumulation needs eps > 0 (its bound)");
  }
  int count = 0;
  tiles_for(table_of(*p), &count);
  if (p->tile < -1 || p->tile >= count) return set_error_msg(NBODY_EINVAL, "bad tile %d", p->tile);
  if (p->jsplit < 0) return set_error_msg(NBODY_EINVAL, "bad jsplit %d", p->jsplit);
  return NBODY_OK;
}

int check_ptr(const void *p, const char *name, bool required = true) {
  if (!p) return required ? set_error_msg(NBODY_EINVAL, "%s is NULL", name) : NBODY_OK;
  if (!aligned16(p)) return set_error_msg(NBODY_EALIGN, "%s is not 16-byte aligned", name);
  return NBODY_OK;
}

// Whether a symmetric gravity plan of this call may add its per-block partials
// atomically in 64-bit fixed point: the scale needs eps > 0 (the bound on every
// sum), and NBODY_NO_COMPENSATION asks for plain FP32 sums instead.
bool atomic_ok(const nbody_params &p) {
  if (p.law != NBODY_LAW_GRAV || !(p.eps2 > 0.0f)) return false;
  return (p.flags & NBODY_FIXED_POINT) || !(p.flags & NBODY_NO_COMPENSATION);
}

// Scratch layout for one single-system evaluation.
struct Scratch {
  float *fscale;  // fixed-point scale (device word) and its inverse: arena header
  double *finv;
  unsigned *ticket;  // atomic plans: last-block ticket of the scale's mass sum (header)
  unsigned *diag_ticket;  // last-block ticket of the finalize's diagnostics sum (header)
  double *msum;      // atomic plans: per-block |m| sums of the interleave launch
  float4 *jbuf;
  float4 *part_hi;
  float4 *part_lo;
  long long *acc64;  // atomic plans: eight int64 accumulators per particle
  double *diag_part;
  double *diag_rows;
};

// Byte sizes of the Scratch regions: scale words, pair buffer, partials (or the
// atomic plan's accumulators), diagnostics. The symmetric tiles write no low
// parts and read their sources in whole blocks (nb x B particles, the last block
// padded).
struct ScratchSizes {
  size_t jb, part, lopart, dpart, drows, msum;
  size_t body() const { return jb + part + lopart + dpart + drows + msum; }  // past the header
  size_t total() const { return kArenaHeader + body(); }
};

ScratchSizes scratch_sizes(int law, int n, const Plan1 &plan, int diag_rows) {
  ScratchSizes z{};
  const bool lo = !plan.atomic && (!plan.tile->sym || plan.tile->fixed);  // FX: int64 (z, w)
  const int64_t jn = plan.tile->sym ? int64_t(plan.slices) * plan.slice_len : n;
  z.part = plan.atomic ? round_up(size_t(8) * size_t(n) * sizeof(long long), 256)
                       : round_up(size_t(plan.slices) * size_t(n) * sizeof(float4), 256);
  z.lopart = lo ? z.part : 0;
  const int nblk = std::max(1, (n + kFinThreads - 1) / kFinThreads);
  z.dpart = round_up(size_t(nblk) * kDiagFields * sizeof(double), 256);
  z.drows = round_up(size_t(std::max(diag_rows, 1)) * kDiagFields * sizeof(double), 256);
  z.jb = jbuf_bytes(law, jn);
  z.msum = plan.atomic ? round_up(size_t((n + 511) / 512) * sizeof(double), 256) : 0;
  return z;
}

size_t scratch_bytes(int law, int n, const Plan1 &plan, int diag_rows) {
  return scratch_sizes(law, n, plan, diag_rows).total();
}

int get_scratch(cudaStream_t s, int law, int n, const Plan1 &plan, int diag_rows, Scratch *out) {
  const ScratchSizes z = scratch_sizes(law, n, plan, diag_rows);
  void *base = nullptr;
  char *hdr = nullptr;
  NB_TRY(workspace(s, z.body(), &base, &hdr));
  out->finv = reinterpret_cast<double *>(hdr);
  out->fscale = reinterpret_cast<float *>(hdr + 8);
  out->ticket = reinterpret_cast<unsigned *>(hdr + 16);
  out->diag_ticket = reinterpret_cast<unsigned *>(hdr + 20);
  char *b = static_cast<char *>(base);
  out->msum = plan.atomic ? reinterpret_cast<double *>(b + z.body() - z.msum) : nullptr;
  out->jbuf = reinterpret_cast<float4 *>(b);
  b += z.jb;
  out->acc64 = plan.atomic ? reinterpret_cast<long long *>(b) : nullptr;
  out->part_hi = plan.atomic ? nullptr : reinterpret_cast<float4 *>(b);
  out->part_lo = z.lopart ? reinterpret_cast<float4 *>(b + z.part) : nullptr;
  out->diag_part = reinterpret_cast<double *>(b + z.part + z.lopart);
  out->diag_rows = reinterpret_cast<double *>(b + z.part + z.lopart + z.dpart);
  return NBODY_OK;
}

// One force evaluation into scratch partials, then one finalize launch.
// first_eval: the first evaluation of this call (atomic plans form the
// fixed-point scale there; the masses do not change between the steps of a call).
// sources_ready: the previous finalize of this call wrote the pair-interleaved
// sources (no interleave launch). prepare_next: this finalize drifts (kFinKickDrift)
// and writes them for the next evaluation; returns in *prepared whether it did.
// kd: a first half-kick and drift that the interleave launch applies (packed tiles).
// chained: a kernel of this call precedes in the stream, so the first launch here may
// be a programmatic dependent launch too (the later ones always are).
int eval_and_finalize(const float4 *pos, const float4 *prm, const nbody_params &p, int n,
                      const Plan1 &plan, const Scratch &sc, int *err, bool pot,
                      FinalizeArgs f, cudaStream_t s, int *nblk, bool first_eval,
                      bool sources_ready = false, bool prepare_next = false,
                      bool *prepared = nullptr, const KickDrift *kd = nullptr,
                      bool chained = false) {
  const bool fx = (p.flags & NBODY_FIXED_POINT) != 0 || plan.atomic;
  const AtomicPrep at{sc.acc64, sc.msum, sc.ticket, p.eps2, sc.fscale, sc.finv,
                      first_eval ? 1 : 0};
  NB_TRY(launch_forces(pos, prm, p.law, p.flags, p.eps2, n, plan, sc.part_hi, sc.part_lo,
                       sc.jbuf, err, pot, s, nullptr,
                       (fx && !plan.atomic) ? sc.fscale : nullptr,
                       plan.atomic ? &at : nullptr, true, sources_ready, kd, chained));
  f.fx_inv = fx ? sc.finv : nullptr;
  f.acc64 = sc.acc64;
  f.part_hi = sc.part_hi;
  f.part_lo = sc.part_lo;
  f.stride = n;
  f.slices = plan.atomic ? 1 : plan.slices;
  f.sym_block = (plan.tile->sym && !plan.atomic) ? plan.tile->tile_i : 0;
  f.sym_split = (plan.tile->sym && !plan.atomic) ? plan.sym_split : 1;
  f.sys_of = nullptr;
  f.sys = nullptr;
  f.n = n;
  f.law = p.law;
  f.G = p.G;
  f.diag_part = sc.diag_part;
  f.plain = (p.flags & NBODY_NO_COMPENSATION) ? 1 : 0;
  const bool prep = prepare_next && plan.tile->packed && (f.mode & kFinKickDrift);
  f.jnext = prep ? sc.jbuf : nullptr;
  f.jn_block = plan.tile->sym ? plan.tile->tile_i : 0;
  f.jn_words = p.law == NBODY_LAW_GRAV ? 2 : 3;
  f.rezero = (prep && plan.atomic) ? 1 : 0;
  f.diag_ticket = sc.diag_ticket;
  if (prepared) *prepared = prep;
  return launch_finalize(f, s, nblk, true);
}

int prepare_fixed(const float4 *pos, int n, const nbody_params &p, const Plan1 &plan,
                  const Scratch &sc, cudaStream_t s) {
  // atomic plans form their scale inside the interleave launch
  if (!(p.flags & NBODY_FIXED_POINT) || plan.atomic) return NBODY_OK;
  fixed_scale_kernel<<<1, 256, 0, s>>>(pos, n, p.eps2, sc.fscale, sc.finv);
  NB_CUDA(cudaGetLastError());
  return NBODY_OK;
}

int forces_device(const float4 *pos, const float4 *prm, float4 *acc, float4 *acc_lo, int n,
                  const nbody_params &p, int sms, cudaStream_t s) {
  Plan1 plan{};
  NB_TRY(plan_single(table_of(p), n, p.tile, p.jsplit, sms, &plan, true, atomic_ok(p)));
  Scratch sc{};
  NB_TRY(get_scratch(s, p.law, n, plan, 0, &sc));
  NB_TRY(prepare_fixed(pos, n, p, plan, sc, s));
  int *err = nullptr;
  NB_TRY(error_word(&err));
  FinalizeArgs f{};
  f.pos = const_cast<float4 *>(pos);
  f.acc = acc;
  f.acc_lo = acc_lo;
  f.mode = kFinWriteAcc;
  return eval_and_finalize(pos, prm, p, n, plan, sc, err, (p.flags & NBODY_COMPUTE_POT) != 0, f,
                           s, nullptr, true);
}

int step_device(float4 *pos, float4 *vel, float4 *acc, const float4 *prm, int n, float dt,
                int nsteps, int report_every, double *diag_dev, float4 *trace, float4 *state_lo,
                const nbody_params &p, int sms, cudaStream_t s) {
  Plan1 plan{};
  NB_TRY(plan_single(table_of(p), n, p.tile, p.jsplit, sms, &plan, true, atomic_ok(p)));
  const int rows = report_every > 0 ? nsteps / report_every + 1 : 0;
  Scratch sc{};
  NB_TRY(get_scratch(s, p.law, n, plan, rows, &sc));
  NB_TRY(prepare_fixed(pos, n, p, plan, sc, s));
  int *err = nullptr;
  NB_TRY(error_word(&err));
  auto report = [&](int step) { return report_every > 0 && step % report_every == 0; };
  const bool want_pot = (p.flags & NBODY_COMPUTE_POT) != 0;
  if (trace) NB_CUDA(cudaMemcpyAsync(trace, pos, size_t(n) * sizeof(float4),
                                     cudaMemcpyDeviceToDevice, s));
  int row = 0;
  bool first_eval = true;  // the fixed-point scale of atomic plans is formed once per call
  bool ready = false;      // the last finalize wrote the next evaluation's source pairs
  bool launched = false;   // a kernel of this call precedes (programmatic dependent launch)
  FinalizeArgs f{};
  f.pos = pos;
  f.vel = vel;
  f.acc = acc;
  f.acc_lo = nullptr;
  f.dt = dt;
  f.x_lo = state_lo;
  f.v_lo = state_lo ? state_lo + n : nullptr;
  // Launches: one force evaluation and one finalize per step. The finalize also
  // sums the diagnostics of a report step, and (all but the last step) drifts the
  // positions and writes them into the next evaluation's source copy; the first
  // half-kick from a caller's acceleration rides on the interleave launch.
  // Step 0: a(x_0) from the caller or from one evaluation; then kick + drift.
  KickDrift kd{pos, vel, acc, trace ? trace + size_t(n) : nullptr, f.x_lo, f.v_lo, dt};
  bool kd_pending = false;  // the first evaluation's interleave launch applies kd
  if (!(p.flags & NBODY_ACC_VALID) || report(0)) {
    f.mode = kFinWriteAcc | (report(0) ? kFinDiag : 0) | (nsteps > 0 ? kFinKickDrift : 0);
    f.trace_next = (trace && nsteps > 0) ? trace + size_t(n) : nullptr;
    f.diag_out = report(0) ? sc.diag_rows + kDiagFields * row++ : nullptr;
    NB_TRY(eval_and_finalize(pos, prm, p, n, plan, sc, err,
                             report(0) || (nsteps == 0 && want_pot), f, s, nullptr, first_eval,
                             false, nsteps > 0, &ready));
    first_eval = false;
    launched = true;
  } else if (nsteps > 0) {
    if (plan.tile->packed) {
      kd_pending = true;
    } else {
      NB_TRY(launch_kick_drift(pos, vel, acc, n, dt, kd.trace1, nullptr, nullptr, f.x_lo,
                               f.v_lo, s));
      launched = true;
    }
  }
  for (int st = 1; st <= nsteps; ++st) {
    const bool rep = report(st);
    const bool last = (st == nsteps);
    f.mode = kFinWriteAcc | kFinKickSync | (rep ? kFinDiag : 0) | (last ? 0 : kFinKickDrift);
    f.trace_next = (trace && !last) ? trace + size_t(st + 1) * size_t(n) : nullptr;
    f.diag_out = rep ? sc.diag_rows + kDiagFields * row++ : nullptr;
    NB_TRY(eval_and_finalize(pos, prm, p, n, plan, sc, err, rep || (last && want_pot), f, s,
                             nullptr, first_eval, ready, !last, &ready,
                             kd_pending ? &kd : nullptr, launched));
    first_eval = false;
    kd_pending = false;
    launched = true;
  }
  if (rows > 0)
    NB_CUDA(cudaMemcpyAsync(diag_dev, sc.diag_rows, size_t(rows) * kDiagFields * sizeof(double),
                            cudaMemcpyDefault, s));
  return NBODY_OK;
}

}  // namespace

extern "C" {

int nbody_version(void) { return 10000; }

const char *nbody_last_error(void) { return last_error_text(); }

int nbody_release(void) {
  clear_error();
  release_all();
  return NBODY_OK;
}

int nbody_check(nbody_stream_t stream) {
  clear_error();
  int dev = 0, sms = 0;
  NB_TRY(check_device(&dev, &sms));
  return sync_and_check(reinterpret_cast<cudaStream_t>(stream));
}

int nbody_pack_grav(const double *x, const double *y, const double *z, const double *m,
                    void *pos_m, int64_t n, nbody_stream_t stream) {
  clear_error();
  if (n < 0 || n > kMaxN) return set_error_msg(NBODY_EINVAL, "n out of range: %lld", (long long)n);
  if (n == 0) return NBODY_OK;
  if (!x || !y || !z || !m) return set_error_msg(NBODY_EINVAL, "x, y, z and m must be non-NULL");
  NB_TRY(check_ptr(pos_m, "pos_m"));
  NB_TRY(check_device(nullptr, nullptr));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  pack_grav_kernel<<<unsigned((n + 255) / 256), 256, 0, s>>>(x, y, z, m,
                                                             static_cast<float4 *>(pos_m), n);
  NB_CUDA(cudaGetLastError());
  return NBODY_OK;
}

int nbody_pack_ljc(const double *q, const double *sigma, const double *eps, const int32_t *type,
                   double kq, void *prm, int64_t n, nbody_stream_t stream) {
  clear_error();
  if (n < 0 || n > kMaxN) return set_error_msg(NBODY_EINVAL, "n out of range: %lld", (long long)n);
  if (n == 0) return NBODY_OK;
  if (!q || !sigma || !eps || !type)
    return set_error_msg(NBODY_EINVAL, "q, sigma, eps and type must be non-NULL");
  if (!(kq >= 0.0) || !std::isfinite(kq)) return set_error_msg(NBODY_EINVAL, "kq must be >= 0");
  NB_TRY(check_ptr(prm, "prm"));
  NB_TRY(check_device(nullptr, nullptr));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  pack_ljc_kernel<<<unsigned((n + 255) / 256), 256, 0, s>>>(q, sigma, eps, type, std::sqrt(kq),
                                                            static_cast<float4 *>(prm), n);
  NB_CUDA(cudaGetLastError());
  return NBODY_OK;
}

int nbody_forces(const void *pos_m, const void *prm, void *acc, void *acc_lo, int64_t n,
                 const nbody_params *params, nbody_stream_t stream) {
  clear_error();
  const NvtxRange nvtx_range("nbody_forces");
  if (n < 0 || n > kMaxN) return set_error_msg(NBODY_EINVAL, "n out of range: %lld", (long long)n);
  if (!params) return set_error_msg(NBODY_EINVAL, "params is NULL");
  if (n == 0) return NBODY_OK;
  NB_TRY(check_params(params, prm));
  NB_TRY(check_ptr(pos_m, "pos_m"));
  NB_TRY(check_ptr(acc, "acc"));
  NB_TRY(check_ptr(prm, "prm", false));
  NB_TRY(check_ptr(acc_lo, "acc_lo", false));
  int dev = 0, sms = 0;
  NB_TRY(check_device(&dev, &sms));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const nbody_params p = *params;
  const int host = is_host_pointer(pos_m);
  if (is_host_pointer(acc) != host || (prm && is_host_pointer(prm) != host) ||
      (acc_lo && is_host_pointer(acc_lo) != host))
    return set_error_msg(NBODY_EINVAL, "pointers must be all host or all device");
  const size_t bytes = size_t(n) * sizeof(float4);
  if (!host)
    return forces_device(static_cast<const float4 *>(pos_m), static_cast<const float4 *>(prm),
                         static_cast<float4 *>(acc), static_cast<float4 *>(acc_lo), int(n), p,
                         sms, s);
  void *st = nullptr;
  NB_TRY(staging(s, 4 * bytes, &st));
  float4 *d_pos = static_cast<float4 *>(st);
  float4 *d_prm = d_pos + n;
  float4 *d_acc = d_prm + n;
  float4 *d_lo = d_acc + n;
  NB_CUDA(cudaMemcpyAsync(d_pos, pos_m, bytes, cudaMemcpyHostToDevice, s));
  if (prm) NB_CUDA(cudaMemcpyAsync(d_prm, prm, bytes, cudaMemcpyHostToDevice, s));
  NB_TRY(forces_device(d_pos, prm ? d_prm : nullptr, d_acc, acc_lo ? d_lo : nullptr, int(n), p,
                       sms, s));
  NB_CUDA(cudaMemcpyAsync(acc, d_acc, bytes, cudaMemcpyDeviceToHost, s));
  if (acc_lo) NB_CUDA(cudaMemcpyAsync(acc_lo, d_lo, bytes, cudaMemcpyDeviceToHost, s));
  return sync_and_check(s);
}

int nbody_workspace_size(const nbody_params *params, int64_t n, int32_t report_rows,
                         size_t *bytes) {
  clear_error();
  if (!bytes) return set_error_msg(NBODY_EINVAL, "bytes is NULL");
  if (n < 0 || n > kMaxN) return set_error_msg(NBODY_EINVAL, "n out of range: %lld", (long long)n);
  if (report_rows < 0) return set_error_msg(NBODY_EINVAL, "report_rows must be >= 0");
  if (!params) return set_error_msg(NBODY_EINVAL, "params is NULL");
  // prm only matters for the LJC laws' presence check: any non-null marker will do
  NB_TRY(check_params(params, params->law == NBODY_LAW_GRAV ? nullptr : params));
  if (n == 0) {
    *bytes = 0;
    return NBODY_OK;
  }
  int dev = 0, sms = 0;
  NB_TRY(check_device(&dev, &sms));
  Plan1 plan{};
  NB_TRY(plan_single(table_of(*params), n, params->tile, params->jsplit, sms, &plan, true,
                     atomic_ok(*params)));
  *bytes = scratch_bytes(params->law, int(n), plan, report_rows);
  return NBODY_OK;
}

int nbody_step(void *pos_m, void *vel, void *acc, const void *prm, int64_t n, float dt,
               int32_t nsteps, int32_t report_every, double *diag, void *trace, void *state_lo,
               const nbody_params *params, nbody_stream_t stream) {
  clear_error();
  const NvtxRange nvtx_range("nbody_step");
  if (n < 0 || n > kMaxN) return set_error_msg(NBODY_EINVAL, "n out of range: %lld", (long long)n);
  if (nsteps < 0) return set_error_msg(NBODY_EINVAL, "nsteps must be >= 0");
  if (report_every < 0) return set_error_msg(NBODY_EINVAL, "report_every must be >= 0");
  if (!std::isfinite(dt)) return set_error_msg(NBODY_EINVAL, "dt must be finite");
  if (report_every > 0 && !diag) return set_error_msg(NBODY_EINVAL, "diag is NULL");
  if (!params) return set_error_msg(NBODY_EINVAL, "params is NULL");
  if (n == 0) return NBODY_OK;
  NB_TRY(check_params(params, prm));
  NB_TRY(check_ptr(pos_m, "pos_m"));
  NB_TRY(check_ptr(vel, "vel"));
  NB_TRY(check_ptr(acc, "acc"));
  NB_TRY(check_ptr(prm, "prm", false));
  NB_TRY(check_ptr(trace, "trace", false));
  NB_TRY(check_ptr(state_lo, "state_lo", false));
  int dev = 0, sms = 0;
  NB_TRY(check_device(&dev, &sms));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const nbody_params p = *params;
  const int host = is_host_pointer(pos_m);
  if (is_host_pointer(vel) != host || is_host_pointer(acc) != host ||
      (prm && is_host_pointer(prm) != host))
    return set_error_msg(NBODY_EINVAL, "pos_m, vel, acc and prm must be all host or all device");
  if (trace && is_host_pointer(trace))
    return set_error_msg(NBODY_EINVAL, "trace must be device memory");
  if (state_lo && is_host_pointer(state_lo) != host)
    return set_error_msg(NBODY_EINVAL, "state_lo must live where pos_m lives");
  const int rows = report_every > 0 ? nsteps / report_every + 1 : 0;
  const bool host_diag = rows > 0 && is_host_pointer(diag);
  const size_t bytes = size_t(n) * sizeof(float4);
  if (!host) {
    NB_TRY(step_device(static_cast<float4 *>(pos_m), static_cast<float4 *>(vel),
                       static_cast<float4 *>(acc), static_cast<const float4 *>(prm), int(n), dt,
                       nsteps, report_every, diag, static_cast<float4 *>(trace),
                       static_cast<float4 *>(state_lo), p, sms, s));
    return host_diag ? sync_and_check(s) : NBODY_OK;
  }
  void *st = nullptr;
  NB_TRY(staging(s, 6 * bytes, &st));
  float4 *d_pos = static_cast<float4 *>(st);
  float4 *d_vel = d_pos + n;
  float4 *d_acc = d_vel + n;
  float4 *d_prm = d_acc + n;
  float4 *d_lo = d_prm + n;
  if (state_lo) NB_CUDA(cudaMemcpyAsync(d_lo, state_lo, 2 * bytes, cudaMemcpyHostToDevice, s));
  NB_CUDA(cudaMemcpyAsync(d_pos, pos_m, bytes, cudaMemcpyHostToDevice, s));
  NB_CUDA(cudaMemcpyAsync(d_vel, vel, bytes, cudaMemcpyHostToDevice, s));
  if (p.flags & NBODY_ACC_VALID) NB_CUDA(cudaMemcpyAsync(d_acc, acc, bytes, cudaMemcpyHostToDevice, s));
  if (prm) NB_CUDA(cudaMemcpyAsync(d_prm, prm, bytes, cudaMemcpyHostToDevice, s));
  NB_TRY(step_device(d_pos, d_vel, d_acc, prm ? d_prm : nullptr, int(n), dt, nsteps,
                     report_every, diag, static_cast<float4 *>(trace), state_lo ? d_lo : nullptr,
                     p, sms, s));
  if (state_lo) NB_CUDA(cudaMemcpyAsync(state_lo, d_lo, 2 * bytes, cudaMemcpyDeviceToHost, s));
  NB_CUDA(cudaMemcpyAsync(pos_m, d_pos, bytes, cudaMemcpyDeviceToHost, s));
  NB_CUDA(cudaMemcpyAsync(vel, d_vel, bytes, cudaMemcpyDeviceToHost, s));
  NB_CUDA(cudaMemcpyAsync(acc, d_acc, bytes, cudaMemcpyDeviceToHost, s));
  return sync_and_check(s);
}

int nbody_timing_enable(int32_t on) {
  clear_error();
  return timing_enable(on);
}

int nbody_timing_read(int32_t which, int64_t *launches, double *total_ms) {
  clear_error();
  return timing_read(which, launches, total_ms);
}

int nbody_tile_count(int32_t law) {
  clear_error();
  if (law < 0 || law >= kTables) return set_error_msg(-NBODY_EINVAL, "bad law %d", law);
  int count = 0;
  tiles_for(law, &count);
  return count;
}

int nbody_tile_info(int32_t law, int32_t tile, int32_t *threads, int32_t *i_per_thread,
                    int32_t *j_lanes, int32_t *j_tile, int32_t *kind) {
  clear_error();
  if (law < 0 || law >= kTables) return set_error_msg(NBODY_EINVAL, "bad law %d", law);
  int count = 0;
  const TileDesc *t = tiles_for(law, &count);
  if (tile < 0 || tile >= count) return set_error_msg(NBODY_EINVAL, "bad tile %d", tile);
  if (threads) *threads = t[tile].nt;
  if (i_per_thread) *i_per_thread = t[tile].i;
  if (j_lanes) *j_lanes = t[tile].sw;
  if (j_tile) *j_tile = t[tile].jt;
  if (kind)
    *kind = (t[tile].packed ? NBODY_TILE_PACKED : 0) | (t[tile].sym ? NBODY_TILE_SYMMETRIC : 0);
  return NBODY_OK;
}

int nbody_set_tuned(int32_t law, int32_t log2n, int32_t tile, int32_t jsplit) {
  clear_error();
  return set_tuned(law, log2n, tile, jsplit);
}

int nbody_get_config(int32_t law, int64_t n, int32_t *tile, int32_t *jsplit) {
  clear_error();
  if (law < 0 || law >= kTables) return set_error_msg(NBODY_EINVAL, "bad law %d", law);
  if (!tile || !jsplit) return set_error_msg(NBODY_EINVAL, "NULL output");
  int t = 0, j = 0;
  get_config(law, n, &t, &j);
  *tile = t;
  *jsplit = j;
  return NBODY_OK;
}

}  // extern "C"
