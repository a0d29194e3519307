// api_common.cu -- host helpers behind the C ABI (see api_common.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <utility>
#include <vector>

#include "api_common.h"
#include "leapfrog.cuh"
#include "vjp_tiles.h"

namespace nbody {

// The device error word: one int per device in the library image itself (zero
// when the module loads), so reporting a kernel's error never allocates. Kernels
// record the first error with atomicCAS; sync_and_check reads and clears it.
__device__ int g_dev_err_word;

namespace {
thread_local std::string t_err;

struct Arena {
  void *ptr = nullptr;
  size_t cap = 0;
};

std::mutex g_mu;
std::map<std::pair<int, cudaStream_t>, Arena> g_ws;
std::map<std::pair<int, cudaStream_t>, Arena> g_stage;
std::map<int, int *> g_err_word;  // device -> address of g_dev_err_word there
std::map<int, int> g_checked;  // device -> sms

struct Tuned {
  int tile = -1;
  int jsplit = 0;
};
Tuned g_tuned[kTables][64];

int grow(std::map<std::pair<int, cudaStream_t>, Arena> &tab, cudaStream_t s, size_t bytes,
         void **out) {
  int dev = 0;
  NB_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_mu);
  Arena &a = tab[{dev, s}];
  if (a.cap < bytes) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    NB_CUDA(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone)
      return set_error_msg(NBODY_EINVAL,
                           "workspace of %zu bytes needed during stream capture; run the "
                           "same call once before capturing",
                           bytes);
    // The old buffer may still be in use by work queued on this stream: free it
    // in stream order, then allocate the larger one.
    if (a.ptr) NB_CUDA(cudaFreeAsync(a.ptr, s));
    a.ptr = nullptr;
    a.cap = 0;
    size_t want = bytes + bytes / 4 + 4096;
    cudaError_t e = cudaMallocAsync(&a.ptr, want, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      a.ptr = nullptr;
      return set_error_msg(NBODY_ENOMEM, "workspace allocation of %zu bytes failed: %s", want,
                           cudaGetErrorString(e));
    }
    a.cap = want;
    // a workspace arena's header holds per-call words (the fixed-point scale and
    // the ticket of its last-block sum), which must start at zero
    NB_CUDA(cudaMemsetAsync(a.ptr, 0, kArenaHeader, s));
  }
  *out = a.ptr;
  return NBODY_OK;
}
}  // namespace

int set_error_msg(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_err = buf;
  return code;
}

void clear_error() { t_err.clear(); }

const char *last_error_text() { return t_err.c_str(); }

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int check_device(int *device, int *sms) {
  int dev = 0, count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || count == 0) {
    cudaGetLastError();
    return set_error_msg(NBODY_EUNSUPPORTED, "no CUDA device available (%s)",
                         cudaGetErrorString(e));
  }
  NB_CUDA(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_checked.find(dev);
    if (it != g_checked.end()) {
      if (device) *device = dev;
      if (sms) *sms = it->second;
      return NBODY_OK;
    }
  }
  int major = 0, minor = 0, nsm = 0;
  NB_CUDA(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
  NB_CUDA(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev));
  NB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  if (major != 10 || minor != 3)
    return set_error_msg(NBODY_EUNSUPPORTED,
                         "this library is compiled for sm_103a only; device %d is sm_%d%d", dev,
                         major, minor);
  std::lock_guard<std::mutex> lk(g_mu);
  g_checked[dev] = nsm;
  if (device) *device = dev;
  if (sms) *sms = nsm;
  return NBODY_OK;
}

int is_host_pointer(const void *p) {
  cudaPointerAttributes at{};
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) ? 0 : 1;
}

int workspace(cudaStream_t s, size_t bytes, void **out, char **header) {
  void *p = nullptr;
  NB_TRY(grow(g_ws, s, bytes + kArenaHeader, &p));
  *out = static_cast<char *>(p) + kArenaHeader;
  if (header) *header = static_cast<char *>(p);
  return NBODY_OK;
}
int staging(cudaStream_t s, size_t bytes, void **out) { return grow(g_stage, s, bytes, out); }

int error_word(int **out) {
  int dev = 0;
  NB_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_err_word.find(dev);
  if (it == g_err_word.end()) {
    void *p = nullptr;
    NB_CUDA(cudaGetSymbolAddress(&p, g_dev_err_word));
    it = g_err_word.emplace(dev, static_cast<int *>(p)).first;
  }
  *out = it->second;
  return NBODY_OK;
}

int sync_and_check(cudaStream_t s) {
  NB_CUDA(cudaStreamSynchronize(s));
  int *w = nullptr;
  NB_TRY(error_word(&w));
  int h = 0;
  NB_CUDA(cudaMemcpy(&h, w, sizeof(int), cudaMemcpyDeviceToHost));
  if (h != 0) {
    NB_CUDA(cudaMemset(w, 0, sizeof(int)));
    if (h == kDevTimeout)
      return set_error_msg(NBODY_ETIMEOUT, "a bounded device wait ran out (pipeline stalled)");
    return set_error_msg(NBODY_EINVAL, "device reported error code %d (bad work item)", h);
  }
  return NBODY_OK;
}

void release_all() {
  std::lock_guard<std::mutex> lk(g_mu);
  cudaDeviceSynchronize();
  for (auto *tab : {&g_ws, &g_stage}) {
    for (auto &kv : *tab)
      if (kv.second.ptr) cudaFree(kv.second.ptr);
    tab->clear();
  }
}

namespace {
struct TimerState {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending[2];
};
TimerState g_timer;

cudaEvent_t take_event() {
  if (!g_timer.pool.empty()) {
    cudaEvent_t e = g_timer.pool.back();
    g_timer.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}
}  // namespace

TimerMark timer_begin(int which, cudaStream_t s) {
  TimerMark m;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_timer.on) return m;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return m;
  }
  m.start = take_event();
  if (m.start && cudaEventRecord(m.start, s) == cudaSuccess) m.which = which;
  return m;
}

void timer_end(const TimerMark &m, cudaStream_t s) {
  if (m.which < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t stop = take_event();
  if (!stop || cudaEventRecord(stop, s) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  g_timer.pending[m.which].push_back({m.start, stop});
}

int timing_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_timer.on = on != 0;
  return NBODY_OK;
}

int timing_read(int which, int64_t *launches, double *total_ms) {
  if (which < 0 || which > 1) return set_error_msg(NBODY_EINVAL, "bad timer %d", which);
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> evs;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    evs.swap(g_timer.pending[which]);
  }
  double tot = 0.0;
  int st = NBODY_OK;
  for (auto &pr : evs) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(pr.second);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, pr.first, pr.second);
    if (e != cudaSuccess && st == NBODY_OK)
      st = set_error_msg(NBODY_ECUDA, "timer event: %s", cudaGetErrorString(e));
    tot += ms;
  }
  {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &pr : evs) {
      g_timer.pool.push_back(pr.first);
      g_timer.pool.push_back(pr.second);
    }
  }
  if (launches) *launches = int64_t(evs.size());
  if (total_ms) *total_ms = tot;
  return st;
}

const TileDesc *tiles_for(int law, int *count) {
  if (law >= kTableVjpGrav) return vjp_tile_descs(law, count);
  if (law == NBODY_LAW_GRAV) return grav_tiles(count);
  if (law == NBODY_LAW_LJC) return ljc_tiles(count);
  if (law == NBODY_LAW_LJC_LINEAR) return ljclin_tiles(count);
  if (law == kTableGravFixed) return grav_fixed_tiles(count);
  return mixed_tiles(count);
}

int set_tuned(int law, int log2n, int tile, int jsplit) {
  if (law < 0 || law >= kTables || log2n < 0 || log2n >= 64)
    return set_error_msg(NBODY_EINVAL, "bad law %d or log2n %d", law, log2n);
  int count = 0;
  tiles_for(law, &count);
  if (tile < -1 || tile >= count) return set_error_msg(NBODY_EINVAL, "bad tile %d", tile);
  if (jsplit < 0) return set_error_msg(NBODY_EINVAL, "bad jsplit %d", jsplit);
  std::lock_guard<std::mutex> lk(g_mu);
  g_tuned[law][log2n].tile = tile;
  g_tuned[law][log2n].jsplit = jsplit;
  return NBODY_OK;
}

static int log2_floor(int64_t n) {
  int b = 0;
  while ((int64_t(1) << (b + 1)) <= n && b < 62) ++b;
  return b;
}

// Default tile when nothing is tuned: big register blocks for large N, j-lanes
// inside the warp for small N (where there are too few targets to fill the GPU).
int default_tile(int law, int64_t n) {
  if (law == kTableBatched) return 0;
  if (law >= kTableVjpGrav) return n >= 8192 ? 0 : 1;
  if (law == kTableGravFixed) return n >= 4096 ? 0 : (n >= 1024 ? 2 : 3);
  if (law == NBODY_LAW_LJC_LINEAR) return n >= 16384 ? 3 : (n >= 1024 ? 1 : 2);
  if (law == NBODY_LAW_GRAV) {
    if (n >= 65536) return 0;
    if (n >= 8192) return 3;
    if (n >= 1024) return 4;
    return 5;
  }
  if (n >= 65536) return 0;
  if (n >= 16384) return 1;
  if (n >= 1024) return 3;
  return 4;
}

int get_config(int law, int64_t n, int *tile, int *jsplit) {
  int t = -1, j = 0;
  if (n >= 0) {
    std::lock_guard<std::mutex> lk(g_mu);
    const Tuned &tu = g_tuned[law][log2_floor(n > 0 ? n : 1)];
    t = tu.tile;
    j = tu.jsplit;
  }
  if (t < 0) t = default_tile(law, n);
  *tile = t;
  *jsplit = j;
  return NBODY_OK;
}

// Largest partial-sum buffer a symmetric tile may ask for (one float4 per
// particle and block): an eighth of the device's memory, at most 16 GiB (4 GiB
// when the device cannot be queried). Cached per device.
double sym_part_cap() {
  constexpr double kGiB = 1024.0 * 1024.0 * 1024.0;
  static std::atomic<double> cached[kMaxDevicesTile];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevicesTile) {
    cudaGetLastError();
    return 4.0 * kGiB;
  }
  double c = cached[dev].load(std::memory_order_relaxed);
  if (c > 0.0) return c;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return 4.0 * kGiB;
  }
  c = std::min(16.0 * kGiB, double(total_b) / 8.0);
  cached[dev].store(c, std::memory_order_relaxed);
  return c;
}

bool sym_fits(int64_t n, int block) {
  const long long nb = (n + block - 1) / block;
  return nb * (nb + 1) / 2 <= 0x7fffffffLL && double(nb) * double(n) * 16.0 <= sym_part_cap();
}

bool sym_atomic_law(int law) { return law == NBODY_LAW_GRAV || law == kTableGravFixed; }

int plan_single(int law, int64_t n, int tile, int jsplit, int sms, Plan1 *out, bool allow_sym,
                bool atomic_ok) {
  return plan_targets(law, n, n, tile, jsplit, sms, out, allow_sym, atomic_ok);
}

int plan_targets(int law, int64_t n_t, int64_t n, int tile, int jsplit, int sms, Plan1 *out,
                 bool allow_sym, bool atomic_ok) {
  out->atomic = false;
  if (law < 0 || law >= kTableVjpGrav)
    return set_error_msg(NBODY_EINVAL, "tile table %d is not a force table", law);
  int count = 0;
  const TileDesc *tiles = tiles_for(law, &count);
  int tj = 0;
  const bool tuned = tile < 0;
  if (tuned) get_config(law, n_t, &tile, &tj);
  if (jsplit <= 0) jsplit = tj;
  if (tile < 0 || tile >= count) return set_error_msg(NBODY_EINVAL, "bad tile %d", tile);
  if (tiles[tile].sym && (!allow_sym || n_t != n)) {
    if (!tuned)
      return set_error_msg(NBODY_EINVAL, "tile %d (symmetric) is not available for this call",
                           tile);
    tile = default_tile(law, n_t);
    jsplit = 0;
  }
  const TileDesc &d = tiles[tile];
  if (d.sym) {  // one CTA per block pair and source part, one partial slot per block and part
    const long long nb = (n + d.tile_i - 1) / d.tile_i;
    // atomic accumulation needs no partial slots: only the grid limit applies
    const bool atomic = atomic_ok && sym_atomic_law(law);
    const bool fits = atomic ? nb * (nb + 1) / 2 <= 0x7fffffffLL : sym_fits(n, d.tile_i);
    if (!fits) {
      if (!tuned)
        return set_error_msg(NBODY_EINVAL, "n = %lld too large for symmetric tile %d",
                             (long long)n, tile);
      return plan_targets(law, n_t, n, default_tile(law, n_t), 0, sms, out, false);
    }
    // Source parts per block: the j-split rounded down to a power of two of at
    // most 8 with each part at least 32 source pairs (as the one-sided tiles clamp
    // theirs); none when it is 0. More parts fill the GPU at small N but add slots
    // to the finalize, so the tuner, which times whole calls, chooses.
    const long long pairs = nb * (nb + 1) / 2;
    const int max_split = (law <= NBODY_LAW_LJC_LINEAR || law == kTableGravFixed)
                              ? std::min(8, std::max(1, d.tile_i / 64))
                              : 1;
    int S = 1;
    while (jsplit > 0 && S * 2 <= std::min(jsplit, max_split)) S *= 2;
    if (pairs * S > 0x7fffffffLL ||
        (!atomic && double(nb) * S * double(n) * 16.0 > sym_part_cap()))
      return set_error_msg(NBODY_EINVAL, "n = %lld too large for symmetric tile %d split %d",
                           (long long)n, tile, S);
    out->atomic = atomic;
    out->tile = &d;
    out->slices = int(nb * S);
    out->slice_len = d.tile_i / S;
    out->n_itiles = int(nb);
    out->grid = int(pairs * S);
    out->sym_split = S;
    return NBODY_OK;
  }
  const int n_it = int((n_t + d.tile_i - 1) / d.tile_i);
  const int max_slices = int((n + d.jt - 1) / d.jt);
  int S = jsplit;
  if (S <= 0) {
    // Pick the j-split whose item count fills whole waves of resident CTAs
    // best; prefer fewer slices among equals (less partial-sum traffic).
    const int cap = sms * d.occupancy();
    double best = -1.0;
    S = 1;
    for (int s = 1; s <= 64 && s <= max_slices; ++s) {
      const int len = int(round_up(size_t((n + s - 1) / s), size_t(d.jt)));
      const int ss = int((n + len - 1) / len);
      const double items = double(n_it) * ss;
      const double waves = items / cap;
      const double eff = waves / std::ceil(waves);
      const double score = eff - 0.002 * ss;
      if (score > best + 1e-12) {
        best = score;
        S = ss;
      }
    }
  }
  S = std::max(1, std::min(S, max_slices));
  int len = int(round_up(size_t((n + S - 1) / S), size_t(d.jt)));
  S = int((n + len - 1) / len);
  out->tile = &d;
  out->slices = S;
  out->slice_len = len;
  out->n_itiles = n_it;
  out->grid = n_it * S;
  out->sym_split = 1;
  return NBODY_OK;
}

// Position of particle i for the interleave kernels: read, or (kd.vel set) first
// kicked and drifted in place.
__device__ __forceinline__ float4 source_at(const float4 *pos, const KickDrift &kd, int i) {
  return kd.vel ? kick_drift_at(kd.pos, kd.vel, kd.acc, kd.dt, kd.trace1, kd.x_lo, kd.v_lo, i)
                : pos[i];
}

// Sources in pairs: jp[2p] = (x0, x1, y0, y1), jp[2p+1] = (z0, z1, m0, m1) for
// particles 2p, 2p+1; an odd count is padded with a massless particle far away
// (its pair terms are exactly zero).
__global__ void interleave_pairs_kernel(const float4 *pos, float4 *jp, int n, KickDrift kd) {
  griddep_start();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (2 * p >= n) return;
  const float4 a = source_at(pos, kd, 2 * p);
  const float4 b =
      (2 * p + 1 < n) ? source_at(pos, kd, 2 * p + 1) : make_float4(1e18f, 1e18f, 1e18f, 0.0f);
  jp[2 * p] = make_float4(a.x, b.x, a.y, b.y);
  jp[2 * p + 1] = make_float4(a.z, b.z, a.w, b.w);
}

// Sources of the symmetric tiles, block by block (B particles): the B/2 pairs
// (x0, x1, y0, y1) of block b, then their (z0, z1, m0, m1), so that lanes reading
// consecutive pairs read consecutive 16-byte words. Pairs past n are not written
// (the kernel copies only the block's own pairs).
// With at.acc64 (atomic plans) the kernel also zeroes the accumulators of its
// particles and forms the fixed-point scale without a launch of its own: every
// block sums |m| of its particles in FP64 in a fixed order, and the block that
// finishes last (atomicInc ticket, which wraps back to zero) adds the block sums
// in index order and writes the scale -- the same bits whichever block is last.
__global__ void __launch_bounds__(256) interleave_pairs_blocked_kernel(const float4 *pos,
                                                                       float4 *jp, int n, int B,
                                                                       AtomicPrep at,
                                                                       KickDrift kd) {
  griddep_start();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  double am = 0.0;
  if (2 * p < n) {
    const float4 a = source_at(pos, kd, 2 * p);
    const float4 b = (2 * p + 1 < n) ? source_at(pos, kd, 2 * p + 1)
                                     : make_float4(1e18f, 1e18f, 1e18f, 0.0f);
    const int blk = (2 * p) / B, pp = p - blk * (B / 2);
    const long long base = (long long)blk * B;
    jp[base + pp] = make_float4(a.x, b.x, a.y, b.y);
    jp[base + B / 2 + pp] = make_float4(a.z, b.z, a.w, b.w);
    if (at.acc64) {
      if (at.form_scale) am = fabs(double(a.w)) + fabs(double(b.w));
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        at.acc64[(long long)c * n + 2 * p] = 0;
        if (2 * p + 1 < n) at.acc64[(long long)c * n + 2 * p + 1] = 0;
      }
    }
  }
  if (!at.acc64 || !at.form_scale) return;  // the same for every thread of the launch
  __shared__ double red[8];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) am += __shfl_down_sync(0xffffffffu, am, off);
  if (lane == 0) red[warp] = am;
  __syncthreads();
  if (threadIdx.x == 0) {
    double bs = 0.0;
    for (int w = 0; w < 8; ++w) bs += red[w];
    at.msum[blockIdx.x] = bs;
    __threadfence();  // the block sum is visible before the ticket is taken
    last = atomicInc(at.ticket, gridDim.x - 1) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double v = 0.0;
  for (int k = threadIdx.x; k < int(gridDim.x); k += 256)
    v += reinterpret_cast<volatile double *>(at.msum)[k];
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double M = 0.0;
    for (int w = 0; w < 8; ++w) M += red[w];
    fixed_scale_of(M, at.eps2, at.scale, at.inv);
  }
}

// LJC sources of the symmetric tiles, block by block (B particles, 3B/2 float4
// per block): the B/2 pairs' (x0 x1 y0 y1), then (z0 z1 q0 q1), then
// (s0 s1 e0 e1). Pairs past n are not written.
__global__ void interleave_ljc_pairs_blocked_kernel(const float4 *pos, const float4 *prm,
                                                    float4 *jp, int n, int B, KickDrift kd) {
  griddep_start();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (2 * p >= n) return;
  const float4 a = source_at(pos, kd, 2 * p), qa = prm[2 * p];
  const bool two = 2 * p + 1 < n;
  const float4 b = two ? source_at(pos, kd, 2 * p + 1) : make_float4(1e18f, 1e18f, 1e18f, 0.0f);
  const float4 qb = two ? prm[2 * p + 1] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  const int blk = (2 * p) / B, P = B / 2, pp = p - blk * P;
  const long long q = (long long)blk * 3 * P + pp;
  jp[q] = make_float4(a.x, b.x, a.y, b.y);
  jp[q + P] = make_float4(a.z, b.z, qa.x, qb.x);
  jp[q + 2 * P] = make_float4(qa.y, qb.y, qa.z, qb.z);
}

// LJC sources in pairs: (x0, x1, y0, y1), (z0, z1, q0, q1), (s0, s1, e0, e1); the
// pad of an odd count is far away with no charge and no LJ well.
__global__ void interleave_ljc_pairs_kernel(const float4 *pos, const float4 *prm, float4 *jp,
                                            int n, KickDrift kd) {
  griddep_start();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (2 * p >= n) return;
  const float4 a = source_at(pos, kd, 2 * p), qa = prm[2 * p];
  const bool two = 2 * p + 1 < n;
  const float4 b = two ? source_at(pos, kd, 2 * p + 1) : make_float4(1e18f, 1e18f, 1e18f, 0.0f);
  const float4 qb = two ? prm[2 * p + 1] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  const long long q = 3LL * p;  // 64-bit: 3p passes 2^31 for n above ~1.4e9
  jp[q] = make_float4(a.x, b.x, a.y, b.y);
  jp[q + 1] = make_float4(a.z, b.z, qa.x, qb.x);
  jp[q + 2] = make_float4(qa.y, qb.y, qa.z, qb.z);
}

size_t jbuf_bytes(int law, int64_t n) {
  const size_t pairs = size_t((n + 1) / 2);
  return round_up(pairs * (law == NBODY_LAW_GRAV ? 2 : 3) * sizeof(float4), 256);
}

int launch_forces(const float4 *pos, const float4 *prm, int law, uint32_t flags, float eps2,
                  int n, const Plan1 &p, float4 *part_hi, float4 *part_lo, float4 *jbuf,
                  int *err, bool pot, cudaStream_t s, const Targets *tg,
                  const float *fscale, const AtomicPrep *at, bool timed,
                  bool sources_ready, const KickDrift *kd, bool chained) {
  const bool atomic = at && at->acc64;
  if (p.atomic != atomic || (atomic && (law != NBODY_LAW_GRAV || tg || !at->msum ||
                                        !at->ticket || !at->scale || !at->inv)))
    return set_error_msg(NBODY_EINVAL, "atomic plan and accumulators must come together");
  if (atomic) fscale = at->scale;
  if ((p.tile->fixed || p.atomic) != (fscale != nullptr))
    return set_error_msg(NBODY_EINVAL, "fixed-point tile and scale must come together");
  if (sources_ready && (!p.tile->packed || tg || (atomic && at->form_scale)))
    return set_error_msg(NBODY_EINVAL, "prepared sources need a packed tile, all targets "
                                       "and a formed scale");
  if (kd && (!p.tile->packed || tg || sources_ready || kd->pos != pos || !kd->vel || !kd->acc))
    return set_error_msg(NBODY_EINVAL, "a fused kick-drift needs a packed tile, all targets "
                                       "and the evaluation's own positions");
  if (p.tile->packed && !sources_ready) {
    if (!jbuf) return set_error_msg(NBODY_EINVAL, "packed tile without pair buffer");
    const int np = (n + 1) / 2;
    const KickDrift k = kd ? *kd : KickDrift{};
    const int g = (np + 255) / 256;
    const AtomicPrep ap = atomic ? *at : AtomicPrep{};
    if ((law == NBODY_LAW_LJC || law == NBODY_LAW_LJC_LINEAR) && p.tile->sym)
      NB_CUDA(launch_kernel(interleave_ljc_pairs_blocked_kernel, g, 256, 0, s, chained, pos, prm,
                            jbuf, n, p.tile->tile_i, k));
    else if (law == NBODY_LAW_LJC || law == NBODY_LAW_LJC_LINEAR)
      NB_CUDA(launch_kernel(interleave_ljc_pairs_kernel, g, 256, 0, s, chained, pos, prm, jbuf,
                            n, k));
    else if (p.tile->sym)
      NB_CUDA(launch_kernel(interleave_pairs_blocked_kernel, g, 256, 0, s, chained, pos, jbuf, n,
                            p.tile->tile_i, ap, k));
    else
      NB_CUDA(launch_kernel(interleave_pairs_kernel, g, 256, 0, s, chained, pos, jbuf, n, k));
    chained = true;
  }
  ForceArgs a{};
  a.jpair = jbuf;
  a.pos = pos;
  a.prm = prm;
  a.tpos = tg ? tg->tpos : pos;
  a.tprm = tg ? tg->tprm : prm;
  a.tidx = tg ? tg->tidx : nullptr;
  a.n_t = tg ? tg->n_t : n;
  a.part_hi = part_hi;
  a.part_lo = part_lo;
  a.stride = a.n_t;
  a.err = err;
  a.n = n;
  a.slices = p.slices;
  a.slice_len = p.slice_len;
  a.eps2 = eps2;
  a.items = nullptr;
  a.n_items = 0;
  a.counter = nullptr;
  a.comp = (flags & NBODY_NO_COMPENSATION) ? 0 : 1;
  a.fscale = fscale;
  a.acc64 = atomic ? at->acc64 : nullptr;
  a.pdl = chained ? 1 : 0;
  const TimerMark tm = timed ? timer_begin(0, s) : TimerMark{};
  cudaError_t e = p.tile->launch(a, p.grid, pot, (flags & NBODY_PRECISE_RSQRT) != 0, s);
  timer_end(tm, s);
  if (e != cudaSuccess)
    return set_error_msg(e == cudaErrorNoKernelImageForDevice ? NBODY_EUNSUPPORTED : NBODY_ECUDA,
                         "force kernel launch failed: %s", cudaGetErrorString(e));
  return NBODY_OK;
}

}  // namespace nbody
