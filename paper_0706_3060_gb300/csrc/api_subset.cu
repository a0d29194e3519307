// api_subset.cu -- nbody_forces_subset: forces on a list of target particles
// against all sources, the evaluation of block time-step schemes (Sec. 3.4: "forces
// are calculated on only a subset of the particles at any one time"), where the
// active set can be far smaller than N and the j-range split ("replication")
// supplies the parallelism.
#include <cuda_runtime.h>

#include <algorithm>
#include <initializer_list>

#include "api_common.h"
#include "aux_types.h"

using namespace nbody;

namespace {

// Gather the targets; an index outside [0, n) is reported through the error
// word and replaced by particle 0 so that no access leaves the arrays.
__global__ void gather_targets_kernel(const float4 *pos, const float4 *prm, const int *idx,
                                      int n_t, int n, float4 *tpos, float4 *tprm, int *tidx,
                                      int *err) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_t) return;
  int g = idx[k];
  if (g < 0 || g >= n) {
    set_error(err, kDevBadItem);
    g = 0;
  }
  tidx[k] = g;
  tpos[k] = pos[g];
  if (prm) tprm[k] = prm[g];
}

}  // namespace

extern "C" int nbody_forces_subset(const void *pos_m, const void *prm, const int32_t *idx,
                                   int64_t n_active, void *acc, int64_t n,
                                   const nbody_params *params, nbody_stream_t stream) {
  clear_error();
  const NvtxRange nvtx_range("nbody_forces_subset");
  if (!params) return set_error_msg(NBODY_EINVAL, "params is NULL");
  if (n < 0 || n > 0x7fffffffLL || n_active < 0 || n_active > 0x7fffffffLL)
    return set_error_msg(NBODY_EINVAL, "n or n_active out of range");
  if (n_active == 0) return NBODY_OK;
  if (n == 0) return set_error_msg(NBODY_EINVAL, "targets given but no sources (n = 0)");
  const nbody_params p = *params;
  if (p.law != NBODY_LAW_GRAV && p.law != NBODY_LAW_LJC && p.law != NBODY_LAW_LJC_LINEAR)
    return set_error_msg(NBODY_EINVAL, "unknown law %d", p.law);
  if (p.flags & ~(uint32_t)(NBODY_COMPUTE_POT | NBODY_PRECISE_RSQRT | NBODY_NO_COMPENSATION))
    return set_error_msg(NBODY_EINVAL, "unsupported flag bits 0x%x", p.flags);
  if (p.law != NBODY_LAW_GRAV && !prm) return set_error_msg(NBODY_EINVAL, "LJC needs prm");
  if (!(p.eps2 >= 0.0f)) return set_error_msg(NBODY_EINVAL, "eps2 must be >= 0");
  if (!pos_m || !acc || !idx) return set_error_msg(NBODY_EINVAL, "pos_m, idx and acc are required");
  for (const void *q : {pos_m, prm, static_cast<const void *>(acc)})
    if (q && !aligned16(q)) return set_error_msg(NBODY_EALIGN, "array not 16-byte aligned");
  if (reinterpret_cast<uintptr_t>(idx) & 3u)
    return set_error_msg(NBODY_EALIGN, "idx is not 4-byte aligned");
  int cnt = 0;
  tiles_for(p.law, &cnt);
  if (p.tile < -1 || p.tile >= cnt) return set_error_msg(NBODY_EINVAL, "bad tile %d", p.tile);
  if (p.jsplit < 0) return set_error_msg(NBODY_EINVAL, "bad jsplit %d", p.jsplit);
  int dev = 0, sms = 0;
  NB_TRY(check_device(&dev, &sms));
  for (const void *q : {pos_m, prm, static_cast<const void *>(idx), static_cast<const void *>(acc)})
    if (q && is_host_pointer(q)) return set_error_msg(NBODY_EINVAL, "device pointers only");

  const int nt = int(n_active), ns = int(n);
  Plan1 plan{};
  NB_TRY(plan_targets(p.law, nt, ns, p.tile, p.jsplit, sms, &plan));
  const size_t jb = jbuf_bytes(p.law, ns);
  const size_t tb = round_up(size_t(nt) * sizeof(float4), 256);
  const size_t ib = round_up(size_t(nt) * sizeof(int), 256);
  const size_t part = round_up(size_t(plan.slices) * size_t(nt) * sizeof(float4), 256);
  void *base = nullptr;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  NB_TRY(workspace(s, jb + 2 * tb + ib + 2 * part, &base));
  char *b = static_cast<char *>(base);
  float4 *jbuf = reinterpret_cast<float4 *>(b);
  float4 *tpos = reinterpret_cast<float4 *>(b + jb);
  float4 *tprm = reinterpret_cast<float4 *>(b + jb + tb);
  int *tidx = reinterpret_cast<int *>(b + jb + 2 * tb);
  float4 *part_hi = reinterpret_cast<float4 *>(b + jb + 2 * tb + ib);
  float4 *part_lo = reinterpret_cast<float4 *>(b + jb + 2 * tb + ib + part);
  int *err = nullptr;
  NB_TRY(error_word(&err));
  const float4 *P = static_cast<const float4 *>(pos_m);
  const float4 *Q = static_cast<const float4 *>(prm);
  gather_targets_kernel<<<(nt + 255) / 256, 256, 0, s>>>(P, Q, idx, nt, ns, tpos,
                                                         Q ? tprm : nullptr, tidx, err);
  NB_CUDA(cudaGetLastError());
  Targets tg{tpos, Q ? tprm : nullptr, tidx, nt};
  NB_TRY(launch_forces(P, Q, p.law, p.flags, p.eps2, ns, plan, part_hi, part_lo, jbuf, err,
                       (p.flags & NBODY_COMPUTE_POT) != 0, s, &tg));
  FinalizeArgs f{};
  f.part_hi = part_hi;
  f.part_lo = part_lo;
  f.stride = nt;
  f.slices = plan.slices;
  f.n = nt;
  f.law = p.law;
  f.G = p.G;
  f.pos = tpos;
  f.acc = static_cast<float4 *>(acc);
  f.mode = kFinWriteAcc;
  f.plain = (p.flags & NBODY_NO_COMPENSATION) ? 1 : 0;
  return launch_finalize(f, s, nullptr);
}
