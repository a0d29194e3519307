// api_common.h -- host-side helpers shared by the C-ABI translation units:
// error reporting, argument checks, per-(device, stream) workspaces, device
// capability checks and tuned tile selection.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <mutex>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "nbody.h"
#include "tiles.h"

namespace nbody {

// NVTX range over one C-ABI call, for timeline profilers and ncu's --nvtx
// filters (a no-op unless a tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

int set_error_msg(int code, const char *fmt, ...);
void clear_error();

#define NB_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return ::nbody::set_error_msg(e_ == cudaErrorMemoryAllocation ? NBODY_ENOMEM      \
                                                                    : NBODY_ECUDA,      \
                                    "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),    \
                                    __FILE__, __LINE__);                                \
  } while (0)

#define NB_TRY(expr)             \
  do {                           \
    int s_ = (expr);             \
    if (s_ != NBODY_OK) return s_; \
  } while (0)

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Device readiness: current device is sm_103 (the only compiled target).
// Also returns the SM count.
int check_device(int *device, int *sms);

// 1 if p is host memory (pageable or pinned), 0 if device/managed memory.
int is_host_pointer(const void *p);

// Scratch owned by the library, one arena per (device, stream). The pointer
// stays valid until the next call on the same (device, stream) asks for more.
// Each workspace arena starts with a header of kArenaHeader bytes for per-call
// device words (zeroed when the arena is allocated; no layout overlaps it):
// *out points past it, *header (if asked) at it.
constexpr size_t kArenaHeader = 256;
int workspace(cudaStream_t s, size_t bytes, void **out, char **header = nullptr);
int staging(cudaStream_t s, size_t bytes, void **out);
// Device error word of the current device (a __device__ int of the library, zero
// when the module loads; no allocation).
int error_word(int **out);
// Synchronize `s`, then read and clear the error word.
int sync_and_check(cudaStream_t s);

// Tile tables: 0 gravity, 1 LJC, 2 LJC linear, 3 the batched mixed-law kernel,
// 4 gravity with fixed-point accumulation, 5 the gravity VJP, 6 the LJC VJP,
// 7 acceleration + jerk, 8 the LJC(linear) VJP. Tables 5-8 describe kernels of
// vjp_kernel.cuh (their
// TileDesc has no force launcher; vjp_tiles() gives the launchers).
constexpr int kTableBatched = 3;
constexpr int kTableGravFixed = 4;
constexpr int kTableVjpGrav = 5;
constexpr int kTableVjpLJC = 6;
constexpr int kTableJerk = 7;
constexpr int kTableVjpLJCLin = 8;
constexpr int kTables = 9;
const TileDesc *tiles_for(int law, int *count);
// Decide (tile, slices, slice_len) for a single-system evaluation.
struct Plan1 {
  const TileDesc *tile;
  int slices;      // partial slots per particle
  int slice_len;   // sources per slice (symmetric tiles: per part of a block)
  int n_itiles;
  int grid;
  int sym_split;   // symmetric tiles: source parts per block (1 otherwise)
  bool atomic;     // symmetric gravity: per-block partials added with integer atomics
                   // into fixed-point accumulators per particle (scratch 64 bytes
                   // per particle) instead of one slot per block
};
// allow_sym: the Newton-symmetric tiles may be used (targets are the sources
// and the partials have room for one slot per block); otherwise a tuned
// symmetric tile falls back to the default tile and an explicit one is refused.
// The untuned tile of a table at size n (never a symmetric one).
int default_tile(int law, int64_t n);
// Whether a Newton-symmetric tile with blocks of `block` particles may run at n:
// nb (nb + 1) / 2 block pairs within the grid limit and nb x n float4 partials
// (nb = ceil(n / block)) within an eighth of the device's memory, at most 16 GiB.
bool sym_fits(int64_t n, int block);
// atomic_ok: a symmetric gravity tile may accumulate atomically in fixed point
// (the caller has eps > 0 and does not ask for plain FP32 sums); such a plan has
// no partial-sum cap, only the grid limit on block pairs.
int plan_single(int law, int64_t n, int tile, int jsplit, int sms, Plan1 *out,
                bool allow_sym = false, bool atomic_ok = false);
// Same for n_t targets against n sources (i-tiles over targets, j-slices over sources).
int plan_targets(int law, int64_t n_t, int64_t n, int tile, int jsplit, int sms, Plan1 *out,
                 bool allow_sym = false, bool atomic_ok = false);
// Whether the symmetric tiles of tile table `law` can accumulate atomically
// (gravity and fixed-point gravity).
bool sym_atomic_law(int law);

// Optional separate targets for launch_forces (subset evaluations).
struct Targets {
  const float4 *tpos;  // gathered target positions (n_t)
  const float4 *tprm;  // gathered target LJC parameters or null
  const int *tidx;     // global index of each target (self mask)
  int n_t;
};

// Launch: all-pairs partial sums into part_hi/lo (slices x n).
// Bytes of the pair-interleaved source copy that packed tiles read.
size_t jbuf_bytes(int law, int64_t n);

// Atomic plans (symmetric gravity in fixed point): the accumulators, which the
// interleave launch before the force kernel zeroes, and the words from which that
// launch forms the fixed-point scale (see interleave_pairs_blocked_kernel).
struct AtomicPrep {
  long long *acc64;  // 8 x n int64 accumulators (integer parts and fractions of x, y, z, w)
  double *msum;      // one FP64 |m| sum per interleave block: ceil(n / 512) doubles
  unsigned *ticket;  // zero before the launch (the arena header); zero again after it
  float eps2;
  float *scale;      // out: 2^S, read by the force kernel
  double *inv;       // out: 2^-S, read by the finalize kernel
  int form_scale;    // 1: form the scale in this launch; 0: an earlier launch of the
                     // same call did (same masses and eps), *scale and *inv hold it
};

// First half-kick and drift that the interleave launch applies before it copies
// the sources (a leapfrog step from a known acceleration, NBODY_ACC_VALID): pos
// (the evaluation's positions, drifted in place), vel, acc, the two-float low
// parts (or null) and the trace row of the drifted positions (or null).
struct KickDrift {
  float4 *pos;
  float4 *vel;
  const float4 *acc;
  float4 *trace1;
  float4 *x_lo;
  float4 *v_lo;
  float dt;
};

// jbuf: scratch of jbuf_bytes(law, n) for the pair-interleaved sources of packed tiles.
// fscale: device word with the fixed-point scale, required exactly for fixed tiles
// (atomic plans take theirs from `at`). at: required exactly for atomic plans.
// timed: bracket the force kernel with the kernel timers when they are enabled (they
// create CUDA events on first use; the allocation-free entry point passes false).
// sources_ready: jbuf already holds the pair-interleaved sources at `pos` (and an
// atomic plan's accumulators are zero), written by the previous step's finalize:
// no interleave launch. kd: the interleave launch first applies this kick-drift to
// the positions at `pos` (kd->pos == pos; packed tiles, all targets, not with
// sources_ready). chained: the previous operation in `s` is a kernel of this
// library issued by the same call, so the first launch may be a programmatic
// dependent launch (the later ones always are).
int launch_forces(const float4 *pos, const float4 *prm, int law, uint32_t flags, float eps2,
                  int n, const Plan1 &p, float4 *part_hi, float4 *part_lo, float4 *jbuf,
                  int *err, bool pot, cudaStream_t s, const Targets *tg = nullptr,
                  const float *fscale = nullptr, const AtomicPrep *at = nullptr,
                  bool timed = true, bool sources_ready = false,
                  const KickDrift *kd = nullptr, bool chained = false);

size_t round_up(size_t x, size_t a);

int set_tuned(int law, int log2n, int tile, int jsplit);
int get_config(int law, int64_t n, int *tile, int *jsplit);
const char *last_error_text();
void release_all();

// Kernel timers (nbody_timing_*): bracket a launch with events when enabled.
struct TimerMark {
  cudaEvent_t start = nullptr;
  int which = -1;
};
TimerMark timer_begin(int which, cudaStream_t s);
void timer_end(const TimerMark &m, cudaStream_t s);
int timing_enable(int on);
int timing_read(int which, int64_t *launches, double *total_ms);

// O(N) kernel launches (aux_kernels.cuh), used by several entry points.
struct FinalizeArgs;
// pdl: a programmatic dependent launch after the force kernel of the same call.
int launch_finalize(const FinalizeArgs &f, cudaStream_t s, int *nblk_out, bool pdl = false);
int launch_kick_drift(float4 *pos, float4 *vel, const float4 *acc, int n, float dt,
                      float4 *trace1, const int *sys_of, const void *sys, float4 *x_lo,
                      float4 *v_lo, cudaStream_t s);

}  // namespace nbody
