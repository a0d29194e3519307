// tiles.h -- host-side table of compiled force-kernel tile configurations.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <utility>

#include "force_kernel.cuh"
#include "sym_kernel.cuh"
#include "sym_ljc_kernel.cuh"
#include "sym_batch_kernel.cuh"

namespace nbody {

constexpr int kMaxDevicesTile = 64;

using ForceLauncher = cudaError_t (*)(const ForceArgs &, int grid, bool pot, bool precise,
                                      cudaStream_t);
using ForceOccupancy = int (*)();  // resident CTAs per SM of the (pot=0, precise=0) kernel

struct TileDesc {
  int law;
  int nt;     // consumer threads
  int i;      // targets per thread
  int sw;     // j-lanes per warp
  int jt;     // j-tile length
  int tile_i; // targets per item
  int threads;
  size_t smem;
  bool packed;  // gravity sources in the pair-interleaved layout (f32x2 math)
  bool fixed;   // 64-bit fixed-point partial sums (NBODY_FIXED_POINT)
  ForceLauncher launch;
  ForceOccupancy occupancy;
  bool sym = false;  // Newton-symmetric block-pair kernel (sym_kernel.cuh): one
                     // partial slot per block, j-split not used, no low parts
};

// Defined in force_grav.cu / force_ljc.cu / force_ljclin.cu / force_mixed.cu.
const TileDesc *grav_tiles(int *count);
const TileDesc *ljc_tiles(int *count);
const TileDesc *ljclin_tiles(int *count);
const TileDesc *grav_fixed_tiles(int *count);
const TileDesc *mixed_tiles(int *count);

// Launch `k` on `s`; with `pdl` as a programmatic dependent launch, which lets
// its CTAs be scheduled while the previous kernel in the stream finishes (the
// kernel waits for that kernel in griddep_start before touching memory).
template <typename... P, typename... A>
inline cudaError_t launch_kernel(void (*k)(P...), int grid, int block, size_t smem,
                                 cudaStream_t s, bool pdl, A &&...args) {
  if (!pdl) {
    k<<<grid, block, smem, s>>>(std::forward<A>(args)...);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(unsigned(block));
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
}

template <int LAW, int NT, int I, int SW, int JT, bool PK = false, int PU = 2, int MINB = 1,
          bool FX = false>
struct TileImpl {
  using T = ForceTile<LAW, NT, I, SW, JT>;
  template <bool POT, bool PRE>
  static cudaError_t go(const ForceArgs &a, int grid, cudaStream_t s) {
    auto k = force_kernel<LAW, NT, I, SW, JT, POT, PRE, PK, PU, MINB, FX>;
    if (T::kSmemBytes > 32 * 1024) {
      // the opt-in is a per-device function attribute: set it once per device
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
  static cudaError_t launch(const ForceArgs &a, int grid, bool pot, bool precise,
                            cudaStream_t s) {
    if (pot) return precise ? go<true, true>(a, grid, s) : go<true, false>(a, grid, s);
    return precise ? go<false, true>(a, grid, s) : go<false, false>(a, grid, s);
  }
  // Resident CTAs per SM, queried once per device and kept (the query costs a few
  // microseconds, which small-N calls would otherwise pay every time).
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
    auto k = force_kernel<LAW, NT, I, SW, JT, false, false, PK, PU, MINB, FX>;
    if (T::kSmemBytes > 32 * 1024)
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::kSmemBytes);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, T::kThreads, T::kSmemBytes) !=
        cudaSuccess) {
      cudaGetLastError();
      return 1;
    }
    nb = nb > 0 ? nb : 1;
    if (dev >= 0) cached[dev].store(nb, std::memory_order_relaxed);
    return nb;
  }
  static TileDesc desc() {
    return TileDesc{LAW, NT, I, SW, JT, T::kTileI, T::kThreads, T::kSmemBytes, PK, FX, &launch,
                    &occupancy};
  }
};

// Newton-symmetric gravity tiles: blocks of NT * I particles, one CTA per block
// pair; `jt` and `tile_i` report the block size. FX: 64-bit fixed-point partials.
template <int NT, int I, int MINB = 1, bool FX = false>
struct SymImpl {
  using T = SymTile<NT, I>;
  template <bool POT, bool PRE>
  static cudaError_t go(const ForceArgs &a, int grid, cudaStream_t s) {
    auto k = sym_grav_kernel<NT, I, POT, PRE, MINB, FX>;
    const size_t smem = T::smem_bytes(POT);
    {  // opt in always: the static mbarrier counts against the 48 KB default too
      static std::atomic<bool> opted[kMaxDevicesTile];
      int dev = 0;
      const bool known = cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < kMaxDevicesTile;
      if (!known || !opted[dev].load(std::memory_order_acquire)) {
        cudaError_t e =
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (known) opted[dev].store(true, std::memory_order_release);
      }
    }
    return launch_kernel(k, grid, NT, smem, s, a.pdl != 0, a);
  }
  static cudaError_t launch(const ForceArgs &a, int grid, bool pot, bool precise,
                            cudaStream_t s) {
    if (pot) return precise ? go<true, true>(a, grid, s) : go<true, false>(a, grid, s);
    return precise ? go<false, true>(a, grid, s) : go<false, false>(a, grid, s);
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
    auto k = sym_grav_kernel<NT, I, false, false, MINB, FX>;
    const size_t smem = T::smem_bytes(false);
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, NT, smem) != cudaSuccess) {
      cudaGetLastError();
      return 1;
    }
    nb = std::max(nb, 1);
    if (dev >= 0) cached[dev].store(nb, std::memory_order_relaxed);
    return nb;
  }
  static TileDesc desc() {
    TileDesc d{kLawGrav, NT, I, 1, T::kB, T::kB, NT, T::smem_bytes(false), true, FX,
               &launch, &occupancy};
    d.sym = true;
    return d;
  }
};

// Newton-symmetric LJC tiles (constant or linear dielectric), as SymImpl.
template <int LAW, int NT, int I, int MINB = 1>
struct SymLjcImpl {
  using T = SymLjcTile<NT, I>;
  template <bool POT, bool PRE>
  static cudaError_t go(const ForceArgs &a, int grid, cudaStream_t s) {
    auto k = sym_ljc_kernel<LAW, NT, I, POT, PRE, MINB>;
    const size_t smem = T::smem_bytes(POT);
    {  // opt in always: the static mbarrier counts against the 48 KB default too
      static std::atomic<bool> opted[kMaxDevicesTile];
      int dev = 0;
      const bool known = cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < kMaxDevicesTile;
      if (!known || !opted[dev].load(std::memory_order_acquire)) {
        cudaError_t e =
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (known) opted[dev].store(true, std::memory_order_release);
      }
    }
    return launch_kernel(k, grid, NT, smem, s, a.pdl != 0, a);
  }
  static cudaError_t launch(const ForceArgs &a, int grid, bool pot, bool precise,
                            cudaStream_t s) {
    if (pot) return precise ? go<true, true>(a, grid, s) : go<true, false>(a, grid, s);
    return precise ? go<false, true>(a, grid, s) : go<false, false>(a, grid, s);
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
    auto k = sym_ljc_kernel<LAW, NT, I, false, false, MINB>;
    const size_t smem = T::smem_bytes(false);
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, NT, smem) != cudaSuccess) {
      cudaGetLastError();
      return 1;
    }
    nb = std::max(nb, 1);
    if (dev >= 0) cached[dev].store(nb, std::memory_order_relaxed);
    return nb;
  }
  static TileDesc desc() {
    TileDesc d{LAW, NT, I, 1, T::kB, T::kB, NT, T::smem_bytes(false), true, false,
               &launch, &occupancy};
    d.sym = true;
    return d;
  }
};

// Newton-symmetric batched tiles (persistent work list of block-pair items over
// systems of mixed law; no potential).
template <int NT, int I, int MINB = 1>
struct SymBatchImpl {
  using T = SymMixedTile<NT, I>;
  template <bool PRE>
  static cudaError_t go(const ForceArgs &a, int grid, cudaStream_t s) {
    auto k = sym_batch_kernel<NT, I, PRE, MINB>;
    {  // opt in always: the static shared words count against the 48 KB default too
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
  static cudaError_t launch(const ForceArgs &a, int grid, bool pot, bool precise,
                            cudaStream_t s) {
    if (pot) return cudaErrorInvalidValue;  // batched runs compute no potential
    return precise ? go<true>(a, grid, s) : go<false>(a, grid, s);
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
    auto k = sym_batch_kernel<NT, I, false, MINB>;
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
  static TileDesc desc() {
    TileDesc d{kLawMixed, NT, I, 1, T::kB, T::kB, NT, T::kSmemBytes, true, false, &launch,
               &occupancy};
    d.sym = true;
    return d;
  }
};

}  // namespace nbody
