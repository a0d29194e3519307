// api_static.cu -- nbody_forces_static: the force evaluation of nbody_forces for
// callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc (or anything that does): code that runs
// under a memory budget fixed at start-up, a host process whose allocator is
// owned by another framework, or a real-time loop where an allocation could
// block or fail in the middle of a run. nbody_forces grows a per-stream
// workspace on demand; this entry point instead uses one scratch array that is
// part of the library image itself.
//
// The scratch is a file-scope __device__ array of kStaticScratchBytes. Every
// GPU that loads this library holds it until the process exits. In host code
// the array's name is only a host-side stand-in, not a device address, so the
// first call on each device (with that device current) asks the runtime for
// the real address with cudaGetSymbolAddress and keeps it; make that first
// call before any stream capture. All calls share the array and it keeps the
// last call's contents: each call overwrites every scratch element it reads
// before reading it, so nothing stale leaks into a result, but two calls whose
// work overlaps on the GPU (for example on two streams) race on the same memory
// and must be serialized by the caller.
//
// A bounded wait that runs out in one of these kernels is recorded in the
// library's device error word (itself a __device__ variable, so reporting needs
// no allocation either) and reported by the next nbody_check.
#include <cuda_runtime.h>

#include <initializer_list>
#include <mutex>

#include "api_common.h"
#include "aux_types.h"
#include "static_plan.h"

namespace {

constexpr int kMaxDevices = 64;

// Partial sums and the pair-interleaved copy of the sources.
static __device__ __align__(256) unsigned char g_static_scratch[nbody::kStaticScratchBytes];

std::mutex g_static_mu;
unsigned char *g_static_addr[kMaxDevices];

int static_address(int dev, unsigned char **out) {
  if (dev < 0 || dev >= kMaxDevices)
    return nbody::set_error_msg(NBODY_EUNSUPPORTED, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_addr[dev]) {
    void *p = nullptr;
    const cudaError_t rc = cudaGetSymbolAddress(&p, g_static_scratch);
    if (rc != cudaSuccess) {
      cudaGetLastError();
      return nbody::set_error_msg(NBODY_ECUDA, "cudaGetSymbolAddress failed: %s",
                                  cudaGetErrorString(rc));
    }
    g_static_addr[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_static_addr[dev];
  return NBODY_OK;
}

}  // namespace

namespace nbody {

namespace {
// n too large for the scratch even with one j-slice (pair copy + 2 float4 per target)?
int static_size_check(int law, int64_t n) {
  const size_t jb = jbuf_bytes(law, n);
  const size_t per_slice = round_up(size_t(n) * sizeof(float4), 256);
  if (jb + 2 * per_slice > kStaticScratchBytes)
    return set_error_msg(NBODY_EINVAL,
                         "n = %lld needs %zu bytes of scratch; the static scratch of "
                         "nbody_forces_static holds %zu bytes (n <= %.0f)",
                         (long long)n, jb + 2 * per_slice, kStaticScratchBytes,
                         (kStaticScratchBytes - 1024) /
                             ((law == NBODY_LAW_GRAV ? 3.0 : 3.5) * sizeof(float4)));
  return NBODY_OK;
}

// Plan one call and lay it out in the scratch: the pair copy of the sources,
// then `slices` high and `slices` low partial sums of n float4 each.
int static_plan(int law, int64_t n, int tile, int jsplit, int sms, Plan1 *plan,
                StaticLayout *lay) {
  NB_TRY(static_size_check(law, n));
  const size_t jb = jbuf_bytes(law, n);
  const size_t per_slice = round_up(size_t(n) * sizeof(float4), 256);
  const size_t max_slices = (kStaticScratchBytes - jb) / (2 * per_slice);
  // Symmetric tiles are never taken here (their partials grow as n^2): a tuned
  // symmetric entry falls back to the law's default one-sided tile.
  NB_TRY(plan_single(law, n, tile, jsplit, sms, plan));
  if (size_t(plan->slices) > max_slices) {
    // Too many j-slices for the scratch: plan again with the tile the first plan
    // resolved to, asking for at most max_slices (plan_targets never rounds a
    // requested split up).
    int count = 0;
    const TileDesc *tiles = tiles_for(law, &count);
    const int resolved = int(plan->tile - tiles);
    NB_TRY(plan_single(law, n, resolved, int(max_slices), sms, plan));
  }
  if (size_t(plan->slices) > max_slices || plan->tile->sym)
    return set_error_msg(NBODY_EINVAL,
                         "no plan for n = %lld fits the static scratch (%d slices, at most %zu)",
                         (long long)n, plan->slices, max_slices);
  int count = 0;
  const TileDesc *tiles = tiles_for(law, &count);
  lay->tile = int(plan->tile - tiles);
  lay->slices = plan->slices;
  lay->jbuf = 0;
  lay->part_hi = jb;
  lay->part_lo = jb + size_t(plan->slices) * per_slice;
  lay->end = jb + 2 * size_t(plan->slices) * per_slice;
  return NBODY_OK;
}
}  // namespace

int static_layout(int law, int64_t n, int tile, int jsplit, int sms, StaticLayout *out) {
  if (law != NBODY_LAW_GRAV && law != NBODY_LAW_LJC && law != NBODY_LAW_LJC_LINEAR)
    return set_error_msg(NBODY_EINVAL, "unknown law %d", law);
  if (n < 1 || n > 0x7fffffffLL || sms < 1 || !out)
    return set_error_msg(NBODY_EINVAL, "bad arguments");
  Plan1 plan{};
  return static_plan(law, n, tile, jsplit, sms, &plan, out);
}

}  // namespace nbody

using namespace nbody;

extern "C" int nbody_forces_static(const void *pos_m, const void *prm, void *acc, int64_t n,
                                   const nbody_params *params, nbody_stream_t stream) {
  clear_error();
  if (!params) return set_error_msg(NBODY_EINVAL, "params is NULL");
  if (n < 0 || n > 0x7fffffffLL)
    return set_error_msg(NBODY_EINVAL, "n out of range: %lld", (long long)n);
  if (n == 0) return NBODY_OK;
  const nbody_params p = *params;
  if (p.law != NBODY_LAW_GRAV && p.law != NBODY_LAW_LJC && p.law != NBODY_LAW_LJC_LINEAR)
    return set_error_msg(NBODY_EINVAL, "unknown law %d", p.law);
  if (p.flags & ~(uint32_t)(NBODY_COMPUTE_POT | NBODY_PRECISE_RSQRT | NBODY_NO_COMPENSATION))
    return set_error_msg(NBODY_EINVAL, "unsupported flag bits 0x%x", p.flags);
  if (p.law != NBODY_LAW_GRAV && !prm) return set_error_msg(NBODY_EINVAL, "LJC needs prm");
  if (!(p.eps2 >= 0.0f)) return set_error_msg(NBODY_EINVAL, "eps2 must be >= 0");
  if (!pos_m || !acc) return set_error_msg(NBODY_EINVAL, "pos_m and acc are required");
  for (const void *q : {pos_m, prm, static_cast<const void *>(acc)})
    if (q && !aligned16(q)) return set_error_msg(NBODY_EALIGN, "array not 16-byte aligned");
  int cnt = 0;
  const TileDesc *tiles = tiles_for(p.law, &cnt);
  if (p.tile < -1 || p.tile >= cnt) return set_error_msg(NBODY_EINVAL, "bad tile %d", p.tile);
  if (p.tile >= 0 && tiles[p.tile].sym)
    return set_error_msg(NBODY_EINVAL,
                         "tile %d is Newton-symmetric; nbody_forces_static runs one-sided tiles "
                         "only",
                         p.tile);
  if (p.jsplit < 0) return set_error_msg(NBODY_EINVAL, "bad jsplit %d", p.jsplit);
  // Size check before touching the GPU: the pair copy of the sources plus two
  // float4 partial sums per target must fit, with at least one j-slice.
  NB_TRY(static_size_check(p.law, n));

  int dev = 0, sms = 0;
  NB_TRY(check_device(&dev, &sms));
  for (const void *q : {pos_m, prm, static_cast<const void *>(acc)})
    if (q && is_host_pointer(q))
      return set_error_msg(NBODY_EINVAL, "nbody_forces_static takes device pointers only");
  unsigned char *scratch = nullptr;
  NB_TRY(static_address(dev, &scratch));
  int *err = nullptr;
  NB_TRY(error_word(&err));

  Plan1 plan{};
  StaticLayout lay{};
  NB_TRY(static_plan(p.law, n, p.tile, p.jsplit, sms, &plan, &lay));
  float4 *jbuf = reinterpret_cast<float4 *>(scratch + lay.jbuf);
  float4 *part_hi = reinterpret_cast<float4 *>(scratch + lay.part_hi);
  float4 *part_lo = reinterpret_cast<float4 *>(scratch + lay.part_lo);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  NB_TRY(launch_forces(static_cast<const float4 *>(pos_m), static_cast<const float4 *>(prm),
                       p.law, p.flags, p.eps2, int(n), plan, part_hi, part_lo, jbuf, err,
                       (p.flags & NBODY_COMPUTE_POT) != 0, s, nullptr, nullptr, nullptr,
                       /*timed=*/false));
  FinalizeArgs f{};
  f.part_hi = part_hi;
  f.part_lo = part_lo;
  f.stride = n;  // the force kernel indexes slice * n + i
  f.slices = plan.slices;
  f.n = int(n);
  f.law = p.law;
  f.G = p.G;
  f.pos = const_cast<float4 *>(static_cast<const float4 *>(pos_m));
  f.acc = static_cast<float4 *>(acc);
  f.mode = kFinWriteAcc;
  f.plain = (p.flags & NBODY_NO_COMPENSATION) ? 1 : 0;
  return launch_finalize(f, s, nullptr);
}
