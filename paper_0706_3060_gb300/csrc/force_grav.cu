// force_grav.cu -- instantiations of the all-pairs kernel for softened gravity
// (Eq. 1, Table 1 "Gravity (accel)").
#include "tiles.h"

namespace nbody {

const TileDesc *grav_tiles(int *count) {
  // (threads, targets/thread, j-lanes/warp, j-tile)
  static const TileDesc tiles[] = {
      TileImpl<kLawGrav, 256, 4, 1, 256>::desc(),  // 0: 1024 targets per item
      TileImpl<kLawGrav, 128, 8, 1, 256>::desc(),  // 1: 1024
      TileImpl<kLawGrav, 256, 2, 1, 256>::desc(),  // 2: 512
      TileImpl<kLawGrav, 128, 4, 1, 256>::desc(),  // 3: 512
      TileImpl<kLawGrav, 128, 2, 4, 256>::desc(),  // 4: 64 targets, 4 j-lanes (small N)
      TileImpl<kLawGrav, 64, 2, 8, 128>::desc(),   // 5: 16 targets, 8 j-lanes (tiny N)
      // packed f32x2 math over source pairs
      TileImpl<kLawGrav, 256, 2, 1, 256, true>::desc(),  // 6: 512 targets
      TileImpl<kLawGrav, 256, 4, 1, 256, true>::desc(),  // 7: 1024
      TileImpl<kLawGrav, 128, 4, 1, 256, true>::desc(),  // 8: 512
      TileImpl<kLawGrav, 128, 2, 1, 256, true>::desc(),  // 9: 256
      TileImpl<kLawGrav, 256, 2, 1, 512, true>::desc(),  // 10: 512, longer j-tiles
      TileImpl<kLawGrav, 256, 3, 1, 256, true>::desc(),  // 11: 768
      TileImpl<kLawGrav, 256, 2, 1, 512, true, 4>::desc(),  // 12: as 10, pair loop unrolled x4
      TileImpl<kLawGrav, 128, 2, 1, 512, true, 4>::desc(),  // 13: 256, unrolled x4
      TileImpl<kLawGrav, 256, 2, 1, 512, true, 2, 3>::desc(),  // 14: as 10, 3 CTAs/SM bound
      TileImpl<kLawGrav, 128, 2, 1, 512, true, 2, 6>::desc(),  // 15: 256, 6 CTAs/SM bound
      // packed with j-lanes (small N)
      TileImpl<kLawGrav, 128, 2, 4, 256, true>::desc(),  // 16: 64 targets, 4 j-lanes
      TileImpl<kLawGrav, 128, 2, 2, 256, true>::desc(),  // 17: 128 targets, 2 j-lanes
      TileImpl<kLawGrav, 64, 2, 8, 256, true>::desc(),   // 18: 16 targets, 8 j-lanes
      // finer items for mid N (more CTAs, fuller last wave), pair loop unrolled x4
      TileImpl<kLawGrav, 64, 2, 1, 512, true, 4>::desc(),    // 19: 128 targets, 1 warp
      TileImpl<kLawGrav, 64, 4, 1, 512, true, 4>::desc(),    // 20: 256 targets, 1 warp
      TileImpl<kLawGrav, 128, 2, 2, 512, true, 4>::desc(),   // 21: 128 targets, 2 j-lanes
      TileImpl<kLawGrav, 256, 1, 1, 512, true, 4>::desc(),   // 22: 256 targets, 1 each
      // Newton-symmetric block pairs (sym_kernel.cuh): each unordered pair once
      SymImpl<128, 8>::desc(),  // 23: blocks of 1024
      SymImpl<128, 4>::desc(),  // 24: blocks of 512
      SymImpl<128, 8, 3>::desc(),  // 25: blocks of 1024, registers capped for 3 CTAs/SM
      SymImpl<128, 6>::desc(),     // 26: blocks of 768 (3 CTAs/SM)
  };
  *count = int(sizeof(tiles) / sizeof(tiles[0]));
  return tiles;
}

}  // namespace nbody
