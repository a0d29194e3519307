// force_grav_fixed.cu -- gravity kernels with 64-bit fixed-point accumulation
// (NBODY_FIXED_POINT; Sec. 3.2, the GRAPE-6 scheme), results independent of the
// j-split.
#include "tiles.h"

namespace nbody {

const TileDesc *grav_fixed_tiles(int *count) {
  static const TileDesc tiles[] = {
      TileImpl<kLawGrav, 128, 2, 1, 512, true, 4, 1, true>::desc(),  // 0: packed, 256 targets
      TileImpl<kLawGrav, 256, 4, 1, 256, false, 2, 1, true>::desc(), // 1: scalar, 1024
      TileImpl<kLawGrav, 128, 2, 4, 256, false, 2, 1, true>::desc(), // 2: 64 targets, 4 j-lanes
      TileImpl<kLawGrav, 64, 2, 8, 128, false, 2, 1, true>::desc(),  // 3: 16 targets, 8 j-lanes
      // Newton-symmetric block pairs (sym_kernel.cuh), fixed-point partials per block
      SymImpl<128, 8, 3, true>::desc(),  // 4: blocks of 1024, 3 CTAs/SM
      SymImpl<128, 4, 1, true>::desc(),  // 5: blocks of 512
  };
  *count = int(sizeof(tiles) / sizeof(tiles[0]));
  return tiles;
}

}  // namespace nbody
