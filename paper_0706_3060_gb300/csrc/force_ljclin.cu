// force_ljclin.cu -- instantiations of the all-pairs kernel for Lennard-Jones plus
// Coulomb with a dielectric growing linearly with distance (Table 1 "LJC(linear)").
#include "tiles.h"

namespace nbody {

const TileDesc *ljclin_tiles(int *count) {
  static const TileDesc tiles[] = {
      TileImpl<kLawLJCLin, 256, 2, 1, 256>::desc(),        // 0: 512 targets per item
      TileImpl<kLawLJCLin, 128, 2, 4, 256>::desc(),        // 1: 64 targets, 4 j-lanes
      TileImpl<kLawLJCLin, 64, 2, 8, 128>::desc(),         // 2: 16 targets, 8 j-lanes
      TileImpl<kLawLJCLin, 128, 2, 1, 256, true>::desc(),  // 3: packed, 256 targets
      TileImpl<kLawLJCLin, 256, 2, 1, 512, true>::desc(),  // 4: packed, 512 targets
      // Newton-symmetric block pairs (sym_ljc_kernel.cuh)
      SymLjcImpl<kLawLJCLin, 128, 4>::desc(),  // 5: blocks of 512
      SymLjcImpl<kLawLJCLin, 128, 2>::desc(),  // 6: blocks of 256
      SymLjcImpl<kLawLJCLin, 64, 4>::desc(),   // 7: blocks of 256, 2-warp CTAs
      // small N: more CTAs per SM (as LJC tiles 18-20)
      SymLjcImpl<kLawLJCLin, 128, 8, 2>::desc(),  // 8: blocks of 1024
      SymLjcImpl<kLawLJCLin, 64, 8, 4>::desc(),   // 9: blocks of 512, 2-warp CTAs
      SymLjcImpl<kLawLJCLin, 64, 4, 8>::desc(),   // 10: blocks of 256, 8 CTAs per SM
  };
  *count = int(sizeof(tiles) / sizeof(tiles[0]));
  return tiles;
}

}  // namespace nbody
