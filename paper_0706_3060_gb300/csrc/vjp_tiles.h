// vjp_tiles.h -- host-side tables of the compiled VJP and jerk kernel
// configurations (tile tables 5, 6 and 7).
#pragma once

#include <cuda_runtime.h>

#include "tiles.h"
#include "sym_vjp_kernel.cuh"
#include "vjp_kernel.cuh"

namespace nbody {

struct VjpDesc {
  int tile_i;   // targets per CTA
  int jt;       // j-tile length
  int threads;  // consumer threads + one producer warp
  size_t smem;
  bool packed;  // gravity sources and lambdas in the pair-interleaved layout
  cudaError_t (*launch)(const VjpArgs &, int grid, cudaStream_t);
  int (*occupancy)();  // resident CTAs per SM, cached per device
  bool sym = false;    // Newton-symmetric block pairs (sym_vjp_kernel.cuh): tile_i and
                       // jt are the block size; one partial slot per block, no low parts
};

// Launchers of tile table `table` (kTableVjpGrav, kTableVjpLJC, kTableJerk or
// kTableVjpLJCLin);
// nullptr for any other table.
const VjpDesc *vjp_tiles(int table, int *count);
// The same tables as TileDesc rows (for tile_count / tile_info / tuning).
const TileDesc *vjp_tile_descs(int table, int *count);

}  // namespace nbody
