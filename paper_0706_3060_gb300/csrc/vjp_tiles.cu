// vjp_tiles.cu -- the compiled VJP (gravity, LJC) and acceleration + jerk tile
// configurations: threads, targets per thread, j-lanes per warp, j-tile length,
// packed f32x2 sources, unroll of the pair loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "api_common.h"
#include "vjp_tiles.h"

namespace nbody {
namespace {

template <int LAW, int NT, int I, int SW, int JT, bool PK = false, int PU = 2>
struct VjpImpl {
  using T = VjpTile<LAW, NT, I, SW, JT, PK>;
  static cudaError_t launch(const VjpArgs &a, int grid, cudaStream_t s) {
    auto k = vjp_kernel<LAW, NT, I, SW, JT, PK, PU>;
    if (T::kSmemBytes > 32 * 1024) {  // per-device attribute: set once per device
      static std::atomic<bool> opted[kMaxDevicesTile];
      int dev = 0;
      const bool known = cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < kMaxDevicesTile;
      if (!known || !opted[dev].load(std::memory_order_acquire)) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)T::kSmemBytes);
        if (e != cudaSuccess) return e;
        if (known) opted[dev].store(true, std::memory_order_release);
      }
    }
    return launch_kernel(k, grid, T::kThreads, T::kSmemBytes, s, a.pdl != 0, a);
  }
  static int occupancy() {  // cached per device, as for the force tiles
    static std::atomic<int> cached[kMaxDevicesTile];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevicesTile) {
      cudaGetLastError();
      dev = -1;
    }
    if (dev >= 0) {
      const int c = cached[dev].load(std::memory_order_relaxed);
      if (c > 0) return c;
    }
    int nb = 0;
    auto k = vjp_kernel<LAW, NT, I, SW, JT, PK, PU>;
    if (T::kSmemBytes > 32 * 1024)
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::kSmemBytes);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, T::kThreads, T::kSmemBytes) !=
        cudaSuccess) {
      cudaGetLastError();
      return 1;
    }
    nb = std::max(nb, 1);
    if (dev >= 0) cached[dev].store(nb, std::memory_order_relaxed);
    return nb;
  }
  static VjpDesc desc() {
    return VjpDesc{T::kTileI, JT, T::kThreads, T::kSmemBytes, PK, &launch, &occupancy};
  }
  static TileDesc tile() {
    return TileDesc{LAW, NT, I, SW, JT, T::kTileI, T::kThreads, T::kSmemBytes, PK, false,
                    nullptr, &occupancy};
  }
};

// Newton-symmetric gravity VJP (GAJ false) and acceleration + jerk (GAJ true)
// tiles: blocks of NT * I particles, one CTA per block pair; `tile_i` and `jt`
// report the block size.
template <int LAW, int NT, int I, int MINB>
struct SymVjpImplT {
  using T = std::conditional_t<
      LAW == kLawGAJ, SymGajTile<NT, I>,
      std::conditional_t<is_ljc(LAW), SymLjcVjpTile<NT, I>, SymVjpTile<NT, I>>>;
  static constexpr auto kernel() {
    if constexpr (LAW == kLawGAJ)
      return sym_gaj_kernel<NT, I, MINB>;
    else if constexpr (is_ljc(LAW))
      return sym_ljc_vjp_kernel<NT, I, LAW == kLawLJCLin, MINB>;
    else
      return sym_gvjp_kernel<NT, I, MINB>;
  }
  static cudaError_t launch(const VjpArgs &a, int grid, cudaStream_t s) {
    auto k = kernel();
    {  // opt in always: the static mbarrier counts against the 48 KB default too
      static std::atomic<bool> opted[kMaxDevicesTile];
      int dev = 0;
      const bool known = cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < kMaxDevicesTile;
      if (!known || !opted[dev].load(std::memory_order_acquire)) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)T::kSmemBytes);
        if (e != cudaSuccess) return e;
        if (known) opted[dev].store(true, std::memory_order_release);
      }
    }
    return launch_kernel(k, grid, NT, T::kSmemBytes, s, a.pdl != 0, a);
  }
  static int occupancy() {
    static std::atomic<int> cached[kMaxDevicesTile];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevicesTile) {
      cudaGetLastError();
      dev = -1;
    }
    if (dev >= 0) {
      const int c = cached[dev].load(std::memory_order_relaxed);
      if (c > 0) return c;
    }
    int nb = 0;
    auto k = kernel();
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::kSmemBytes);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, NT, T::kSmemBytes) !=
        cudaSuccess) {
      cudaGetLastError();
      return 1;
    }
    nb = std::max(nb, 1);
    if (dev >= 0) cached[dev].store(nb, std::memory_order_relaxed);
    return nb;
  }
  static VjpDesc desc() {
    VjpDesc d{T::kB, T::kB, NT, T::kSmemBytes, true, &launch, &occupancy};
    d.sym = true;
    return d;
  }
  static TileDesc tile() {
    TileDesc d{LAW, NT, I, 1, T::kB, T::kB, NT, T::kSmemBytes, true, false, nullptr,
               &occupancy};
    d.sym = true;
    return d;
  }
};

template <int NT, int I, int MINB = 1>
using SymVjpImpl = SymVjpImplT<kLawGrav, NT, I, MINB>;
template <int NT, int I, int MINB = 1>
using SymGajImpl = SymVjpImplT<kLawGAJ, NT, I, MINB>;
template <int LAW, int NT, int I, int MINB = 1>
using SymLjcVjpImpl = SymVjpImplT<LAW, NT, I, MINB>;

// Rows: (law, consumer threads, targets per thread, j-lanes, j-tile, packed,
// unroll). Row 0 is the default for large N, row 1 for small N (below 8192).
// Tables: gravity VJP, LJC VJP, LJC(linear) VJP, acceleration + jerk.
#define NB_VJP_GRAV_ROWS(X)                                         \
  X(kLawGrav, 256, 2, 1, 256, true, 2)                              \
  X(kLawGrav, 128, 2, 4, 256, false, 2)                             \
  X(kLawGrav, 128, 2, 1, 512, true, 4)                              \
  X(kLawGrav, 256, 2, 1, 512, true, 2)                              \
  X(kLawGrav, 128, 2, 1, 256, true, 2)                              \
  X(kLawGrav, 256, 1, 1, 256, true, 4)                              \
  X(kLawGrav, 128, 4, 1, 256, true, 1)                              \
  X(kLawGrav, 128, 1, 8, 256, false, 2)                             \
  X(kLawGrav, 256, 1, 1, 512, true, 4)                              \
  X(kLawGrav, 128, 1, 1, 256, true, 4)                              \
  X(kLawGrav, 512, 1, 1, 256, true, 4)                              \
  X(kLawGrav, 128, 2, 1, 256, true, 4)
#define NB_VJP_LJC_ROWS(X)                                          \
  X(kLawLJC, 256, 2, 1, 256, false, 2)                              \
  X(kLawLJC, 128, 1, 4, 256, false, 2)                              \
  X(kLawLJC, 128, 2, 1, 256, false, 2)                              \
  X(kLawLJC, 256, 1, 1, 256, false, 2)                              \
  X(kLawLJC, 128, 2, 2, 256, false, 2)                              \
  X(kLawLJC, 256, 2, 1, 256, true, 2)                               \
  X(kLawLJC, 128, 2, 1, 256, true, 2)                               \
  X(kLawLJC, 256, 1, 1, 256, true, 2)                               \
  X(kLawLJC, 128, 1, 1, 512, true, 4)
#define NB_VJP_LJCLIN_ROWS(X)                                       \
  X(kLawLJCLin, 128, 2, 1, 256, true, 2)                            \
  X(kLawLJCLin, 128, 1, 4, 256, false, 2)                           \
  X(kLawLJCLin, 256, 1, 1, 256, true, 2)                            \
  X(kLawLJCLin, 256, 2, 1, 256, false, 2)
#define NB_VJP_GAJ_ROWS(X)                                          \
  X(kLawGAJ, 256, 2, 1, 256, false, 2)                              \
  X(kLawGAJ, 128, 2, 4, 256, false, 2)                              \
  X(kLawGAJ, 128, 2, 1, 256, false, 2)                              \
  X(kLawGAJ, 256, 1, 1, 256, false, 2)                              \
  X(kLawGAJ, 128, 2, 1, 512, false, 4)                              \
  X(kLawGAJ, 256, 2, 1, 256, true, 2)                               \
  X(kLawGAJ, 128, 2, 1, 512, true, 4)                               \
  X(kLawGAJ, 256, 1, 1, 256, true, 4)                               \
  X(kLawGAJ, 128, 2, 1, 256, true, 2)

#define NB_VJP_DESC(L, NT, I, SW, JT, PK, PU) VjpImpl<L, NT, I, SW, JT, PK, PU>::desc(),
#define NB_VJP_TILE(L, NT, I, SW, JT, PK, PU) VjpImpl<L, NT, I, SW, JT, PK, PU>::tile(),

// the gravity VJP table ends with the Newton-symmetric tiles: blocks of 512, 256,
// 512 with registers capped for 3 CTAs/SM, 256 in 2-warp CTAs (6 per SM), 384
#define NB_VJP_GRAV_SYM(F)                                                         \
  SymVjpImpl<128, 4>::F(), SymVjpImpl<128, 2>::F(), SymVjpImpl<128, 4, 3>::F(),    \
      SymVjpImpl<64, 4, 6>::F(), SymVjpImpl<128, 3, 4>::F(),

const VjpDesc kGravDesc[] = {NB_VJP_GRAV_ROWS(NB_VJP_DESC) NB_VJP_GRAV_SYM(desc)};
// the LJC VJP tables end with their Newton-symmetric tiles: blocks of 256 (4 warps
// x 2 targets), 256 in 2-warp CTAs (x 4 targets), 128 in 2-warp CTAs
#define NB_LJC_VJP_SYM(L, F)                                             \
  SymLjcVjpImpl<L, 128, 2>::F(), SymLjcVjpImpl<L, 64, 4>::F(), SymLjcVjpImpl<L, 64, 2>::F(),

const VjpDesc kLjcDesc[] = {NB_VJP_LJC_ROWS(NB_VJP_DESC) NB_LJC_VJP_SYM(kLawLJC, desc)};
// the jerk table ends with its Newton-symmetric tiles: blocks of 512 (3 CTAs/SM),
// 256 in 2-warp CTAs, 256
#define NB_GAJ_SYM(F) \
  SymGajImpl<128, 4, 3>::F(), SymGajImpl<64, 4, 6>::F(), SymGajImpl<128, 2>::F(),

const VjpDesc kGajDesc[] = {NB_VJP_GAJ_ROWS(NB_VJP_DESC) NB_GAJ_SYM(desc)};
const VjpDesc kLjcLinDesc[] = {NB_VJP_LJCLIN_ROWS(NB_VJP_DESC)
                                   NB_LJC_VJP_SYM(kLawLJCLin, desc)};
const TileDesc kGravTile[] = {NB_VJP_GRAV_ROWS(NB_VJP_TILE) NB_VJP_GRAV_SYM(tile)};
const TileDesc kLjcTile[] = {NB_VJP_LJC_ROWS(NB_VJP_TILE) NB_LJC_VJP_SYM(kLawLJC, tile)};
const TileDesc kGajTile[] = {NB_VJP_GAJ_ROWS(NB_VJP_TILE) NB_GAJ_SYM(tile)};
const TileDesc kLjcLinTile[] = {NB_VJP_LJCLIN_ROWS(NB_VJP_TILE)
                                    NB_LJC_VJP_SYM(kLawLJCLin, tile)};

#undef NB_VJP_DESC
#undef NB_VJP_TILE
#undef NB_VJP_GRAV_ROWS
#undef NB_VJP_GRAV_SYM
#undef NB_GAJ_SYM
#undef NB_LJC_VJP_SYM
#undef NB_VJP_LJC_ROWS
#undef NB_VJP_GAJ_ROWS
#undef NB_VJP_LJCLIN_ROWS

template <class T, size_t N>
constexpr int count_of(const T (&)[N]) {
  return int(N);
}

}  // namespace

const VjpDesc *vjp_tiles(int table, int *count) {
  switch (table) {
    case kTableVjpGrav: *count = count_of(kGravDesc); return kGravDesc;
    case kTableVjpLJC: *count = count_of(kLjcDesc); return kLjcDesc;
    case kTableJerk: *count = count_of(kGajDesc); return kGajDesc;
    case kTableVjpLJCLin: *count = count_of(kLjcLinDesc); return kLjcLinDesc;
    default: *count = 0; return nullptr;
  }
}

const TileDesc *vjp_tile_descs(int table, int *count) {
  switch (table) {
    case kTableVjpGrav: *count = count_of(kGravTile); return kGravTile;
    case kTableVjpLJC: *count = count_of(kLjcTile); return kLjcTile;
    case kTableJerk: *count = count_of(kGajTile); return kGajTile;
    case kTableVjpLJCLin: *count = count_of(kLjcLinTile); return kLjcLinTile;
    default: *count = 0; return nullptr;
  }
}

}  // namespace nbody
