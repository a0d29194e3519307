// aux_types.h -- data shared by the O(N) kernels and their host-side callers.
#pragma once

#include <cuda_runtime.h>

namespace nbody {

// Per-system data of a batched run (one entry per system).
struct SysInfo {
  int law;      // kLawGrav / kLawLJC
  int slices;   // partial slots written for this system
  float G;
  float dt;
};

enum : int {
  kFinWriteAcc = 1,   // store acc (and acc_lo)
  kFinKickSync = 2,   // v += dt/2 a       (completes the previous step)
  kFinDiag = 4,       // FP64 diagnostics with the synchronized velocity
  kFinKickDrift = 8,  // v += dt/2 a; x += dt v   (starts the next step)
};

struct FinalizeArgs {
  const float4 *part_hi;
  const float4 *part_lo;
  long long stride;
  int slices;
  const int *sys_of;     // batched: system of each particle (-1: gap), or null
  const SysInfo *sys;    // batched: per-system info, or null
  int n;
  int law;
  float G;
  float dt;
  float4 *pos;
  float4 *vel;
  float4 *acc;
  float4 *acc_lo;        // may be null
  float4 *trace_next;    // positions after the drift, or null
  const double *fx_inv;  // fixed-point partials (int64): value = sum * (*fx_inv); else null
  // fixed-point accumulators of atomic plans (eight int64 arrays of stride
  // `stride`, one element per particle: the integer parts of x, y, z, w, then
  // their fractions in units of 2^-32; with fx_inv), else null
  long long *acc64;
  float4 *x_lo;          // compensated state: low parts of x and v, or null
  float4 *v_lo;
  int mode;
  double *diag_part;     // [gridDim.x][8]
  // Newton-symmetric tiles with the source split (sym_kernel.cuh): block size
  // and parts per block; slot k of particle i counts only if k / split >=
  // i / block or k % split is i's part. sym_split <= 1: every slot counts.
  int sym_block;
  int sym_split;
  // 1: add the slots in plain FP32 (NBODY_NO_COMPENSATION); 0: compensated
  // (TwoSum into a high and a low part).
  int plain;
  // Steps of nbody_step: with kFinKickDrift, also write the drifted positions
  // into the pair-interleaved source copy that the next force evaluation reads
  // (null: none), so that it needs no interleave launch. jn_block: block size of
  // the blocked layout of the symmetric tiles (0: one source pair after another);
  // jn_words: float4 words per source pair (2 gravity, 3 LJC); only each pair's
  // (x x y y) word and the (z z) half of its second word change.
  float4 *jnext;
  int jn_block;
  int jn_words;
  int rezero;  // atomic plans: zero the accumulators after reading them
  // With kFinDiag: also add the block rows of diag_part into diag_out (8 doubles)
  // in the last block to finish, which diag_ticket (zero before the launch, zero
  // again after it) elects; null: only the block rows are written.
  double *diag_out;
  unsigned *diag_ticket;
};

constexpr int kFinThreads = 64;  // many CTAs: the finalize is latency-bound at small n
constexpr int kDiagFields = 8;  // K, U, Px, Py, Pz, Lx, Ly, Lz

}  // namespace nbody
