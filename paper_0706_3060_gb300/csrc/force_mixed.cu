// force_mixed.cu -- persistent work-list instantiations for batched ensembles
// that mix gravity and LJC systems in one launch (Sec. 3.4, small systems).
#include "tiles.h"

namespace nbody {

const TileDesc *mixed_tiles(int *count) {
  static const TileDesc tiles[] = {
      TileImpl<kLawMixed, 128, 2, 4, 256>::desc(),  // 0: 64 targets, 4 j-lanes
      TileImpl<kLawMixed, 128, 2, 1, 256>::desc(),  // 1: 256 targets
      TileImpl<kLawMixed, 128, 2, 2, 256>::desc(),  // 2: 128 targets, 2 j-lanes
      TileImpl<kLawMixed, 64, 2, 8, 128>::desc(),   // 3: 16 targets, 8 j-lanes
      // packed f32x2 over source pairs of each system (pair buffers per law)
      TileImpl<kLawMixed, 128, 2, 4, 256, true>::desc(),  // 4: 64 targets, 4 j-lanes
      TileImpl<kLawMixed, 128, 2, 2, 256, true>::desc(),  // 5: 128 targets, 2 j-lanes
      TileImpl<kLawMixed, 128, 2, 1, 256, true>::desc(),  // 6: 256 targets
      TileImpl<kLawMixed, 64, 2, 8, 256, true>::desc(),   // 7: 16 targets, 8 j-lanes
      // as 6 and 5 with registers capped for 3 CTAs per SM
      TileImpl<kLawMixed, 128, 2, 1, 256, true, 2, 3>::desc(),  // 8: 256 targets
      TileImpl<kLawMixed, 128, 2, 2, 256, true, 2, 3>::desc(),  // 9: 128 targets, 2 j-lanes
      // Newton-symmetric block-pair items (sym_batch_kernel.cuh)
      SymBatchImpl<128, 2>::desc(),     // 10: blocks of 256
      SymBatchImpl<64, 4>::desc(),      // 11: blocks of 256, 2-warp CTAs
      SymBatchImpl<128, 4>::desc(),     // 12: blocks of 512
      SymBatchImpl<64, 2>::desc(),      // 13: blocks of 128, 2-warp CTAs
  };
  *count = int(sizeof(tiles) / sizeof(tiles[0]));
  return tiles;
}

}  // namespace nbody
