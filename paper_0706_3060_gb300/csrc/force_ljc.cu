// force_ljc.cu -- instantiations of the all-pairs kernel for Lennard-Jones plus
// Coulomb with a constant dielectric (Table 1 "LJC(constant)").
#include "tiles.h"

namespace nbody {

const TileDesc *ljc_tiles(int *count) {
  static const TileDesc tiles[] = {
      TileImpl<kLawLJC, 256, 2, 1, 256>::desc(),  // 0: 512 targets per item
      TileImpl<kLawLJC, 128, 4, 1, 256>::desc(),  // 1: 512
      TileImpl<kLawLJC, 256, 4, 1, 256>::desc(),  // 2: 1024
      TileImpl<kLawLJC, 128, 2, 4, 256>::desc(),  // 3: 64 targets, 4 j-lanes
      TileImpl<kLawLJC, 64, 2, 8, 128>::desc(),   // 4: 16 targets, 8 j-lanes
      // packed f32x2 math over source pairs
      TileImpl<kLawLJC, 256, 2, 1, 256, true>::desc(),   // 5: 512 targets
      TileImpl<kLawLJC, 128, 2, 1, 256, true>::desc(),   // 6: 256
      TileImpl<kLawLJC, 64, 2, 1, 256, true>::desc(),    // 7: 128
      TileImpl<kLawLJC, 256, 2, 1, 512, true>::desc(),   // 8: 512, longer j-tiles
      TileImpl<kLawLJC, 128, 2, 4, 256, true>::desc(),   // 9: packed, 64 targets, 4 j-lanes
      TileImpl<kLawLJC, 128, 2, 2, 256, true>::desc(),   // 10: packed, 128 targets, 2 j-lanes
      TileImpl<kLawLJC, 64, 2, 8, 256, true>::desc(),    // 11: packed, 16 targets, 8 j-lanes
      // as 10 and 9 with registers capped for 3 CTAs per SM (more warps at small N)
      TileImpl<kLawLJC, 128, 2, 2, 256, true, 2, 3>::desc(),  // 12: 128 targets, 2 j-lanes
      TileImpl<kLawLJC, 128, 2, 4, 256, true, 2, 3>::desc(),  // 13: 64 targets, 4 j-lanes
      // Newton-symmetric block pairs (sym_ljc_kernel.cuh): each unordered pair once
      SymLjcImpl<kLawLJC, 128, 4>::desc(),     // 14: blocks of 512
      SymLjcImpl<kLawLJC, 128, 2>::desc(),     // 15: blocks of 256
      SymLjcImpl<kLawLJC, 64, 4>::desc(),      // 16: blocks of 256, 2-warp CTAs
      SymLjcImpl<kLawLJC, 128, 8, 2>::desc(),  // 17: blocks of 1024
      // small N: eight targets per thread in narrower CTAs, more CTAs per SM
      SymLjcImpl<kLawLJC, 64, 8, 4>::desc(),   // 18: blocks of 512, 2-warp CTAs
      SymLjcImpl<kLawLJC, 32, 8, 8>::desc(),   // 19: blocks of 256, 1-warp CTAs
      SymLjcImpl<kLawLJC, 64, 4, 8>::desc(),   // 20: blocks of 256, 2-warp CTAs, 8 per SM
  };
  *count = int(sizeof(tiles) / sizeof(tiles[0]));
  return tiles;
}

}  // namespace nbody
