// Host-only check of nbody_forces_static's plan: for every law, a sweep of sizes,
// every one-sided tile, j-splits and SM counts, and with symmetric tiles installed
// as the tuned choice (as the stored tuning does from a few thousand particles
// up), every accepted plan must keep the pair copy and both partial-sum arrays
// inside the static scratch, never pick a symmetric tile, and every refused size
// must be one whose single-slice layout does not fit. Needs no GPU: the planner
// reads only the tile and tuning tables. Prints one line per failure; exit 0 when
// all pass.
#include <cstdio>
#include <cstdint>

#include "nbody.h"
#include "static_plan.h"

static int g_fail = 0;

#define CHECK(cond, ...)                 \
  do {                                   \
    if (!(cond)) {                       \
      if (g_fail < 50) {                 \
        std::printf("FAIL %s: ", #cond); \
        std::printf(__VA_ARGS__);        \
        std::printf("\n");               \
      }                                  \
      ++g_fail;                          \
    }                                    \
  } while (0)

static size_t jbuf_of(int law, int64_t n) {  // pair copy: 2 (gravity) or 3 float4 per pair
  const size_t b = size_t((n + 1) / 2) * (law == NBODY_LAW_GRAV ? 2 : 3) * 16;
  return (b + 255) / 256 * 256;
}

int main() {
  const int laws[] = {NBODY_LAW_GRAV, NBODY_LAW_LJC, NBODY_LAW_LJC_LINEAR};
  // the tuned choice a GPU session installs: symmetric tiles from 2^12 on, with
  // and without a source split
  for (int law : laws) {
    const int cnt = nbody_tile_count(law);
    int sym = -1;
    for (int t = 0; t < cnt; ++t) {
      int kind = 0;
      nbody_tile_info(law, t, nullptr, nullptr, nullptr, nullptr, &kind);
      if (kind & NBODY_TILE_SYMMETRIC) sym = t;
    }
    CHECK(sym >= 0, "law %d has a symmetric tile", law);
    for (int b = 12; b <= 24; ++b) nbody_set_tuned(law, b, sym, (b & 1) ? 2 : 0);
  }
  const int64_t sizes[] = {1,      2,      3,      31,     1000,   4097,   70001,  131071,
                           131072, 200000, 262144, 300001, 524288, 600000, 699000, 699050,
                           699051, 700000, 1048576, 4000000};
  const int splits[] = {0, 1, 3, 8, 64, 1000};
  const int sms_list[] = {1, 8, 152, 304, 2048};
  long long accepted = 0, refused = 0;
  for (int law : laws) {
    const int cnt = nbody_tile_count(law);
    for (int64_t n : sizes) {
      const size_t per_slice = (size_t(n) * 16 + 255) / 256 * 256;
      const bool fits = jbuf_of(law, n) + 2 * per_slice <= nbody::kStaticScratchBytes;
      for (int tile = -1; tile < cnt; ++tile) {
        int kind = 0;
        if (tile >= 0) nbody_tile_info(law, tile, nullptr, nullptr, nullptr, nullptr, &kind);
        if (kind & NBODY_TILE_SYMMETRIC) continue;  // refused by the entry point itself
        for (int js : splits)
          for (int sms : sms_list) {
            nbody::StaticLayout L{};
            const int rc = nbody::static_layout(law, n, tile, js, sms, &L);
            if (rc != NBODY_OK) {
              ++refused;
              CHECK(!fits, "law %d n %lld tile %d js %d sms %d refused (%s)", law, (long long)n,
                    tile, js, sms, nbody_last_error());
              continue;
            }
            ++accepted;
            CHECK(fits, "law %d n %lld accepted but does not fit", law, (long long)n);
            int k2 = 0;
            nbody_tile_info(law, L.tile, nullptr, nullptr, nullptr, nullptr, &k2);
            CHECK(!(k2 & NBODY_TILE_SYMMETRIC), "law %d n %lld tile %d js %d: symmetric tile %d",
                  law, (long long)n, tile, js, L.tile);
            CHECK(tile < 0 || L.tile == tile, "explicit tile %d replaced by %d", tile, L.tile);
            CHECK(L.slices >= 1, "slices %d", L.slices);
            const size_t part = size_t(L.slices) * size_t(n) * 16;  // slice * n + i, float4
            CHECK(L.jbuf == 0 && L.part_hi >= jbuf_of(law, n), "jbuf overlaps part_hi");
            CHECK(L.part_lo >= L.part_hi + part, "part_hi overlaps part_lo (n %lld slices %d)",
                  (long long)n, L.slices);
            CHECK(L.end >= L.part_lo + part, "part_lo overruns end");
            CHECK(L.end <= nbody::kStaticScratchBytes,
                  "law %d n %lld tile %d js %d sms %d: end %zu > scratch (slices %d)", law,
                  (long long)n, tile, js, sms, L.end, L.slices);
            CHECK(L.part_hi % 16 == 0 && L.part_lo % 16 == 0, "partials not 16-byte aligned");
          }
      }
    }
  }
  std::printf("accepted %lld refused %lld failures %d\n", accepted, refused, g_fail);
  return g_fail == 0 ? 0 : 1;
}
