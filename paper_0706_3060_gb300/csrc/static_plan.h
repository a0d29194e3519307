// static_plan.h -- the plan and scratch layout of nbody_forces_static, as a host
// function with plain types (no CUDA headers), so that it can be checked on a
// machine without a GPU.
#pragma once

#include <cstddef>
#include <cstdint>

namespace nbody {

// Bytes of the static scratch array of nbody_forces_static.
constexpr size_t kStaticScratchBytes = size_t(32) << 20;  // 32 MiB

// Where one call puts its data inside the static scratch (byte offsets).
struct StaticLayout {
  int tile;        // row of the law's force table that runs (never a symmetric one)
  int slices;      // j-slices, i.e. partial sums per target
  size_t jbuf;     // pair-interleaved copy of the sources (packed tiles)
  size_t part_hi;  // slices x n float4 high parts, slice-major
  size_t part_lo;  // slices x n float4 low parts, slice-major
  size_t end;      // first byte past the last one used; never above kStaticScratchBytes
};

// Plan a call of nbody_forces_static for `n` particles of force law `law` with
// the caller's tile (-1: tuned/default) and jsplit (0: automatic) on a GPU with
// `sms` multiprocessors. Host only: it reads the tuned table and tile tables but
// touches no device. Returns NBODY_OK and fills `out`, or NBODY_EINVAL when n is
// larger than the scratch holds (or, defensively, when no j-split fits).
int static_layout(int law, int64_t n, int tile, int jsplit, int sms, StaticLayout *out);

}  // namespace nbody
