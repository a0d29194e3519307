// api_tune.cu -- nbody_tune: the library's own autotuner. For one tile table
// and problem size it times every compiled tile x j-split through the public
// entry points (CUDA events on the caller's stream), installs the fastest as
// the tuned entry of that size bucket and returns it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "api_common.h"

using namespace nbody;

namespace {

constexpr int kSplits[] = {0, 1, 2, 4, 8, 16, 32};

// One call of the entry point that table `table` configures.
int run_once(int table, const void *pos, const void *prm, int64_t n, float eps2, int tile,
             int jsplit, float4 *out0, float4 *out1, float *outm, cudaStream_t s) {
  nbody_params p{};
  p.G = 1.0f;
  p.eps2 = eps2;
  p.tile = tile;
  p.jsplit = jsplit;
  nbody_stream_t st = reinterpret_cast<nbody_stream_t>(s);
  switch (table) {
    case NBODY_LAW_GRAV:
    case NBODY_LAW_LJC:
    case NBODY_LAW_LJC_LINEAR:
      p.law = table;
      return nbody_forces(pos, prm, out0, nullptr, n, &p, st);
    case kTableGravFixed:
      p.law = NBODY_LAW_GRAV;
      p.flags = NBODY_FIXED_POINT;
      return nbody_forces(pos, prm, out0, nullptr, n, &p, st);
    case kTableVjpGrav:
    case kTableVjpLJC:
    case kTableVjpLJCLin:
      // lambda = the positions: any finite values time the same
      p.law = table == kTableVjpLJC      ? NBODY_LAW_LJC
              : table == kTableVjpLJCLin ? NBODY_LAW_LJC_LINEAR
                                         : NBODY_LAW_GRAV;
      return nbody_adjoint(pos, table == kTableVjpGrav ? nullptr : prm, pos, out0, outm,
                           nullptr, 0, 1.0f, n, &p, st);
    case kTableJerk:
      p.law = NBODY_LAW_GRAV;
      return nbody_forces_jerk(pos, pos, out0, out1, n, &p, st);
    default:
      return set_error_msg(NBODY_EUNSUPPORTED, "table %d is not tuned by nbody_tune", table);
  }
}

}  // namespace

extern "C" {

int nbody_tune(int32_t table, const void *pos_m, const void *prm, int64_t n, float eps2,
               int32_t reps, int32_t *best_tile, int32_t *best_jsplit, float *best_ms,
               nbody_stream_t stream) {
  clear_error();
  const NvtxRange nvtx_range("nbody_tune");
  if (table < 0 || table >= kTables || table == kTableBatched)
    return set_error_msg(NBODY_EUNSUPPORTED, "table %d is not tuned by nbody_tune", table);
  if (n < 1 || n > 0x7fffffffLL) return set_error_msg(NBODY_EINVAL, "n out of range");
  if (reps < 1 || reps > 1000) return set_error_msg(NBODY_EINVAL, "reps must be in 1..1000");
  if (!pos_m) return set_error_msg(NBODY_EINVAL, "pos_m is NULL");
  const bool needs_prm = table == NBODY_LAW_LJC || table == NBODY_LAW_LJC_LINEAR ||
                         table == kTableVjpLJC || table == kTableVjpLJCLin;
  if (needs_prm && !prm) return set_error_msg(NBODY_EINVAL, "this table needs prm");
  if (table == kTableGravFixed && !(eps2 > 0.0f))
    return set_error_msg(NBODY_EINVAL, "fixed-point tuning needs eps2 > 0");
  if (!(eps2 >= 0.0f)) return set_error_msg(NBODY_EINVAL, "eps2 must be >= 0");
  int dev = 0, sms = 0;
  NB_TRY(check_device(&dev, &sms));
  if (is_host_pointer(pos_m) || (prm && is_host_pointer(prm)))
    return set_error_msg(NBODY_EINVAL, "nbody_tune takes device inputs");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

  // outputs: two float4 arrays and one float array from the staging arena (the
  // device paths called below use only the workspace arena)
  const size_t q = round_up(size_t(n) * sizeof(float4), 256);
  void *base = nullptr;
  NB_TRY(staging(s, 2 * q + round_up(size_t(n) * sizeof(float), 256), &base));
  char *b = static_cast<char *>(base);
  float4 *o0 = reinterpret_cast<float4 *>(b);
  float4 *o1 = reinterpret_cast<float4 *>(b + q);
  float *om = reinterpret_cast<float *>(b + 2 * q);

  int count = 0;
  const TileDesc *tiles = tiles_for(table, &count);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  NB_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return set_error_msg(NBODY_ECUDA, "cudaEventCreate failed");
  }
  int st = NBODY_OK;
  bool ev_fail = false;
  float best = -1.0f;
  int bt = -1, bj = 0;
  std::vector<float> ts(static_cast<size_t>(reps));
  for (int t = 0; t < count && st == NBODY_OK; ++t) {
    for (int js : kSplits) {
      if (js > 0 && int64_t(js) * tiles[t].jt > n) continue;  // slices shorter than a j-tile
      if (tiles[t].sym) {  // j-split = source parts per block; skip what the plan refuses
        // softened gravity (forces and the VJP) accumulates in fixed point where
        // the slots would not fit (no partial-sum cap)
        const bool atomic =
            (sym_atomic_law(table) || table == kTableVjpGrav || table == kTableJerk) &&
            eps2 > 0.0f;
        if (!atomic && !sym_fits(n, tiles[t].tile_i)) continue;
        if (js > 0 && table == kTableVjpGrav) {  // the VJP plan takes powers of two
          if ((js & (js - 1)) != 0 || js > std::min(8, tiles[t].tile_i / 64)) continue;
        } else if (js > 0) {  // only splits the plan takes as given (not rounded or refused)
          Plan1 probe{};
          if (table >= kTableVjpGrav || table == kTableBatched ||
              plan_single(table, n, t, js, sms, &probe, true, atomic) != NBODY_OK ||
              probe.sym_split != js) {
            clear_error();
            continue;
          }
        }
      }
      if (js == 0 && tiles[t].tile_i > 4 * n) continue;       // far more targets than particles
      st = run_once(table, pos_m, prm, n, eps2, t, js, o0, o1, om, s);  // warm-up
      for (int r = 0; r < reps && st == NBODY_OK; ++r) {
        ev_fail = cudaEventRecord(e0, s) != cudaSuccess;
        if (!ev_fail) st = run_once(table, pos_m, prm, n, eps2, t, js, o0, o1, om, s);
        if (!ev_fail && st == NBODY_OK)
          ev_fail = cudaEventRecord(e1, s) != cudaSuccess ||
                    cudaEventSynchronize(e1) != cudaSuccess ||
                    cudaEventElapsedTime(&ts[size_t(r)], e0, e1) != cudaSuccess;
        if (ev_fail) st = NBODY_ECUDA;
      }
      if (st != NBODY_OK) break;
      std::vector<float> sorted(ts);
      std::nth_element(sorted.begin(), sorted.begin() + reps / 2, sorted.end());
      const float med = sorted[size_t(reps / 2)];
      if (best < 0.0f || med < best) {
        best = med;
        bt = t;
        bj = js;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (ev_fail) return set_error_msg(NBODY_ECUDA, "timing events failed");
  if (st != NBODY_OK) return st;
  NB_TRY(sync_and_check(s));
  if (bt < 0) return set_error_msg(NBODY_EINVAL, "no tile fits n = %lld", (long long)n);
  int lg = 0;
  while ((int64_t(1) << (lg + 1)) <= n && lg < 62) ++lg;
  NB_TRY(set_tuned(table, lg, bt, bj));
  if (best_tile) *best_tile = bt;
  if (best_jsplit) *best_jsplit = bj;
  if (best_ms) *best_ms = best;
  return NBODY_OK;
}

}  // extern "C"
