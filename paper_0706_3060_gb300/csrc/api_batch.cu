// api_batch.cu -- batched ensembles: many independent systems of uneven size in
// one persistent launch per force evaluation (Sec. 3.4 on small systems: more
// parallel work by splitting the i- and j-ranges), with the
// whole leapfrog loop captured once into a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <initializer_list>
#include <cmath>
#include <vector>

#include "api_common.h"
#include "aux_types.h"

using namespace nbody;

struct nbody_batch_plan {
  int device = 0;
  int sms = 0;
  std::vector<nbody_system> sys;
  int64_t total = 0;
  const TileDesc *td = nullptr;
  uint32_t flags = 0;
  int n_items = 0;
  int max_slices = 1;
  int grid = 0;
  WorkItem *d_items = nullptr;
  SysInfo *d_sys = nullptr;
  int *d_sys_of = nullptr;
  int *d_counter = nullptr;  // one counter per force evaluation of a run
  int counters = 0;
  float4 *d_part = nullptr;  // [2][max_slices][total]
  // packed tiles: per-law pair buffers and, per system, (offset, pair base, n, law)
  float4 *d_jgrav = nullptr;
  float4 *d_jljc = nullptr;
  int4 *d_sysp = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  const void *gkey[4] = {nullptr, nullptr, nullptr, nullptr};
  int gsteps = -1;
  uint32_t gflags = 0;
};

namespace {

void free_plan(nbody_batch_plan *p) {
  if (!p) return;
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  cudaFree(p->d_items);
  cudaFree(p->d_sys);
  cudaFree(p->d_sys_of);
  cudaFree(p->d_counter);
  cudaFree(p->d_part);
  cudaFree(p->d_jgrav);
  cudaFree(p->d_jljc);
  cudaFree(p->d_sysp);
  delete p;
}

int ensure_counters(nbody_batch_plan *p, int need) {
  if (p->counters >= need) return NBODY_OK;
  if (p->d_counter) NB_CUDA(cudaFree(p->d_counter));
  p->d_counter = nullptr;
  NB_CUDA(cudaMalloc(&p->d_counter, sizeof(int) * size_t(need)));
  p->counters = need;
  return NBODY_OK;
}

// Packed tiles: every particle writes its half of its system's source pair in the
// layout of its law; the last particle of an odd system also writes the pad half
// (far away, no mass, charge or well), whose pair terms are exactly zero.
__global__ void interleave_systems_kernel(const float4 *pos, const float4 *prm,
                                          const int *sys_of, const int4 *sysp, int total,
                                          float4 *jgrav, float4 *jljc) {
  griddep_start();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int k = sys_of[i];
  if (k < 0) return;
  const int4 sp = sysp[k];  // offset, pair base, n, law
  const int local = i - sp.x;
  const int pair = sp.y + (local >> 1);
  const int half = local & 1;
  const bool pad = (local == sp.z - 1) && (sp.z & 1);
  const float4 x = pos[i];
  if (sp.w == NBODY_LAW_GRAV) {
    float *jp = reinterpret_cast<float *>(jgrav + 2 * pair);
    jp[0 + half] = x.x;
    jp[2 + half] = x.y;
    jp[4 + half] = x.z;
    jp[6 + half] = x.w;
    if (pad) {
      jp[1] = 1e18f;
      jp[3] = 1e18f;
      jp[5] = 1e18f;
      jp[7] = 0.0f;
    }
  } else {
    const float4 q = prm[i];
    float *jp = reinterpret_cast<float *>(jljc + 3 * pair);
    jp[0 + half] = x.x;
    jp[2 + half] = x.y;
    jp[4 + half] = x.z;
    jp[6 + half] = q.x;
    jp[8 + half] = q.y;
    jp[10 + half] = q.z;
    if (pad) {
      jp[1] = 1e18f;
      jp[3] = 1e18f;
      jp[5] = 1e18f;
      jp[7] = 0.0f;
      jp[9] = 0.0f;
      jp[11] = 0.0f;
    }
  }
}

// Newton-symmetric tiles: sources block by block (B particles) per system, in
// the law's layout: gravity (x x y y) then (z z m m) words of the block's pairs,
// LJC (x x y y), (z z q q), (s s e e); sysp = (offset, first float4 of the
// system's blocks, n, law). The last particle of an odd system also writes the
// pad half of its pair.
__global__ void interleave_systems_blocked_kernel(const float4 *pos, const float4 *prm,
                                                  const int *sys_of, const int4 *sysp,
                                                  int total, float4 *jgrav, float4 *jljc,
                                                  int B) {
  griddep_start();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int k = sys_of[i];
  if (k < 0) return;
  const int4 sp = sysp[k];
  const int local = i - sp.x;
  const int blk = local / B, P = B / 2;
  const int pp = (local - blk * B) >> 1;
  const int half = local & 1;
  const bool pad = (local == sp.z - 1) && (sp.z & 1);
  const float4 x = pos[i];
  if (sp.w == NBODY_LAW_GRAV) {
    const long long base = (long long)sp.y + (long long)blk * B + pp;
    float *a0 = reinterpret_cast<float *>(jgrav + base);
    float *a1 = reinterpret_cast<float *>(jgrav + base + P);
    a0[half] = x.x;
    a0[2 + half] = x.y;
    a1[half] = x.z;
    a1[2 + half] = x.w;
    if (pad) {
      a0[1] = 1e18f;
      a0[3] = 1e18f;
      a1[1] = 1e18f;
      a1[3] = 0.0f;
    }
  } else {
    const float4 q = prm[i];
    const long long base = (long long)sp.y + (long long)blk * 3 * P + pp;
    float *a0 = reinterpret_cast<float *>(jljc + base);
    float *a1 = reinterpret_cast<float *>(jljc + base + P);
    float *a2 = reinterpret_cast<float *>(jljc + base + 2 * P);
    a0[half] = x.x;
    a0[2 + half] = x.y;
    a1[half] = x.z;
    a1[2 + half] = q.x;
    a2[half] = q.y;
    a2[2 + half] = q.z;
    if (pad) {
      a0[1] = 1e18f;
      a0[3] = 1e18f;
      a1[1] = 1e18f;
      a1[3] = 0.0f;
      a2[1] = 0.0f;
      a2[3] = 0.0f;
    }
  }
}

// Enqueue nsteps leapfrog steps (or one force evaluation when nsteps == 0).
int enqueue_run(nbody_batch_plan *p, float4 *pos, float4 *vel, float4 *acc, const float4 *prm,
                int nsteps, uint32_t flags, int *err, cudaStream_t s) {
  const int total = int(p->total);
  const long long stride = p->total;
  float4 *part_hi = p->d_part;
  // the symmetric tiles write one partial per particle and block, without low parts
  float4 *part_lo = p->td->sym ? nullptr : p->d_part + size_t(p->max_slices) * size_t(stride);
  const int evals = nsteps + ((flags & NBODY_ACC_VALID) && nsteps > 0 ? 0 : 1);
  // Every evaluation has its own work counter so that the graph needs no
  // reset between launches of different steps; all are zeroed up front.
  NB_CUDA(cudaMemsetAsync(p->d_counter, 0, sizeof(int) * size_t(evals), s));
  int counter_idx = 0;
  // Every launch after the first kernel of the run is a programmatic dependent
  // launch (the memset before it is not a kernel).
  bool chained = false;
  auto eval = [&](int mode) -> int {
    const int g = (total + 255) / 256;
    if (p->td->sym) {
      NB_CUDA(launch_kernel(interleave_systems_blocked_kernel, g, 256, 0, s, chained, pos, prm,
                            p->d_sys_of, p->d_sysp, total, p->d_jgrav, p->d_jljc,
                            p->td->tile_i));
      chained = true;
    } else if (p->td->packed) {
      NB_CUDA(launch_kernel(interleave_systems_kernel, g, 256, 0, s, chained, pos, prm,
                            p->d_sys_of, p->d_sysp, total, p->d_jgrav, p->d_jljc));
      chained = true;
    }
    ForceArgs a{};
    a.jpair = p->d_jgrav;
    a.jpair2 = p->d_jljc;
    a.pos = pos;
    a.prm = prm;
    a.tpos = pos;
    a.tprm = prm;
    a.tidx = nullptr;
    a.n_t = total;
    a.part_hi = part_hi;
    a.part_lo = part_lo;
    a.stride = stride;
    a.err = err;
    a.items = p->d_items;
    a.n_items = p->n_items;
    a.counter = p->d_counter + counter_idx++;
    a.comp = (p->flags & NBODY_NO_COMPENSATION) ? 0 : 1;
    a.pdl = chained ? 1 : 0;
    const TimerMark tm = timer_begin(0, s);
    cudaError_t e = p->td->launch(a, p->grid, false, (p->flags & NBODY_PRECISE_RSQRT) != 0, s);
    timer_end(tm, s);
    if (e != cudaSuccess)
      return set_error_msg(NBODY_ECUDA, "batched force launch failed: %s", cudaGetErrorString(e));
    FinalizeArgs f{};
    f.part_hi = part_hi;
    f.part_lo = part_lo;
    f.stride = stride;
    f.slices = 1;
    f.sys_of = p->d_sys_of;
    f.sys = p->d_sys;
    f.n = total;
    f.pos = pos;
    f.vel = vel;
    f.acc = acc;
    f.mode = mode;
    f.plain = (p->flags & NBODY_NO_COMPENSATION) ? 1 : 0;
    chained = true;
    return launch_finalize(f, s, nullptr, true);
  };
  if (!(flags & NBODY_ACC_VALID) || nsteps == 0) {
    NB_TRY(eval(kFinWriteAcc | (nsteps > 0 ? kFinKickDrift : 0)));
  } else {
    NB_TRY(launch_kick_drift(pos, vel, acc, total, 0.0f, nullptr, p->d_sys_of, p->d_sys,
                             nullptr, nullptr, s));
    chained = true;
  }
  for (int st = 1; st <= nsteps; ++st)
    NB_TRY(eval(kFinWriteAcc | kFinKickSync | (st == nsteps ? 0 : kFinKickDrift)));
  return NBODY_OK;
}

}  // namespace

extern "C" {

int nbody_batch_plan_create(const nbody_system *systems, int32_t nsys, uint32_t flags,
                            int32_t tile, nbody_batch_plan **plan) {
  clear_error();
  if (!plan) return set_error_msg(NBODY_EINVAL, "plan is NULL");
  *plan = nullptr;
  if (!systems || nsys <= 0) return set_error_msg(NBODY_EINVAL, "need at least one system");
  if (flags & ~(uint32_t)(NBODY_PRECISE_RSQRT | NBODY_NO_COMPENSATION))
    return set_error_msg(NBODY_EINVAL, "unsupported plan flags 0x%x", flags);
  int count = 0;
  const TileDesc *tiles = tiles_for(kTableBatched, &count);
  if (tile < -1 || tile >= count) return set_error_msg(NBODY_EINVAL, "bad tile %d", tile);
  int dev = 0, sms = 0;
  NB_TRY(check_device(&dev, &sms));
  if (tile < 0) {
    int tj = 0;
    get_config(kTableBatched, 0, &tile, &tj);
    if (tile < 0 || tile >= count) tile = 0;
  }
  const TileDesc *td = &tiles[tile];

  // Validate the table: non-overlapping ranges inside [0, 2^31).
  std::vector<int> order(nsys);
  int64_t total = 0;
  for (int k = 0; k < nsys; ++k) {
    const nbody_system &s = systems[k];
    if (s.n < 1 || s.offset < 0 || s.offset + s.n > 0x7fffffffLL)
      return set_error_msg(NBODY_EINVAL, "system %d: bad offset/n", k);
    if (s.law != NBODY_LAW_GRAV && s.law != NBODY_LAW_LJC && s.law != NBODY_LAW_LJC_LINEAR)
      return set_error_msg(NBODY_EINVAL, "system %d: unknown law %d", k, s.law);
    if (!(s.eps2 >= 0.0f) || !std::isfinite(s.G) || !std::isfinite(s.dt))
      return set_error_msg(NBODY_EINVAL, "system %d: bad G / eps2 / dt", k);
    total = std::max<int64_t>(total, s.offset + s.n);
    order[k] = k;
  }
  std::sort(order.begin(), order.end(),
            [&](int a, int b) { return systems[a].offset < systems[b].offset; });
  for (int k = 1; k < nsys; ++k) {
    const nbody_system &a = systems[order[k - 1]], &b = systems[order[k]];
    if (a.offset + a.n > b.offset)
      return set_error_msg(NBODY_EINVAL, "systems %d and %d overlap", order[k - 1], order[k]);
  }

  // Work list: one item per (system, i-tile, j-slice). Items are cut to about
  // 1/16 of the average work per persistent CTA, so that the last items leave
  // little imbalance (measured on the 512-system ensemble: kernel 595 us with
  // 1/4, 577 us with 1/8, 561 us with 1/16; the finalize grows with the slices).
  const int occ = td->occupancy();
  const int grid = sms * occ;
  double work = 0.0;
  for (int k = 0; k < nsys; ++k) work += double(systems[k].n) * double(systems[k].n);
  const double target = std::max(work / (double(grid) * 16.0), double(td->tile_i) * td->jt);
  std::vector<WorkItem> items;
  std::vector<SysInfo> info(nsys);
  std::vector<int4> sysp(nsys);
  int max_slices = 1;
  long long pairs_law[2] = {0, 0};  // pair-buffer sizes per law (packed tiles)
  long long f4_law[2] = {0, 0};     // float4 sizes of the blocked buffers (symmetric tiles)
  for (int k = 0; k < nsys && td->sym; ++k) {
    // Newton-symmetric tiles: one item per block pair (bi <= bj) of each system,
    // one partial slot per block
    const nbody_system &s = systems[k];
    const int B = td->tile_i;
    const int nb = (s.n + B - 1) / B;
    if (nb > 0xffff)
      return set_error_msg(NBODY_EINVAL, "system %d: n = %d too large for symmetric tile %d",
                           k, s.n, tile);
    const int pl = (s.law == NBODY_LAW_GRAV) ? 0 : 1;
    const long long per_block = pl ? 3LL * (B / 2) : (long long)B;  // float4 per block
    const long long jb = f4_law[pl];
    f4_law[pl] += per_block * nb;
    if (f4_law[pl] > 0x7fffffffLL)
      return set_error_msg(NBODY_EINVAL, "ensemble too large for symmetric tile %d", tile);
    sysp[k] = make_int4(int(s.offset), int(jb), s.n, s.law);
    max_slices = std::max(max_slices, nb);
    info[k] = SysInfo{s.law, nb, s.G, s.dt};
    for (int bi = 0; bi < nb; ++bi)
      for (int bj = bi; bj < nb; ++bj) {
        WorkItem w{};
        w.i0 = int(s.offset) + bi * B;
        w.ni = std::min(B, s.n - bi * B);
        w.j0 = int(s.offset) + bj * B;
        w.nj = std::min(B, s.n - bj * B);
        w.law = (s.law == NBODY_LAW_LJC_LINEAR) ? kLawLJCLin : s.law;
        w.slice = bj | (bi << 16);
        w.eps2 = s.eps2;
        w.pj0 = int(jb + per_block * bj);
        items.push_back(w);
      }
  }
  for (int k = 0; k < nsys && !td->sym; ++k) {
    const nbody_system &s = systems[k];
    const int pl = (s.law == NBODY_LAW_GRAV) ? 0 : 1;  // both LJC laws share one layout
    const int pbase = int(pairs_law[pl]);
    pairs_law[pl] += (s.n + 1) / 2;
    sysp[k] = make_int4(int(s.offset), pbase, s.n, s.law);
    const int max_s = (s.n + td->jt - 1) / td->jt;
    int S = int(std::ceil(double(std::min(s.n, td->tile_i)) * s.n / target));
    S = std::max(1, std::min(S, max_s));
    const int len = int(round_up(size_t((s.n + S - 1) / S), size_t(td->jt)));
    S = (s.n + len - 1) / len;
    max_slices = std::max(max_slices, S);
    info[k] = SysInfo{s.law, S, s.G, s.dt};
    for (int i0 = 0; i0 < s.n; i0 += td->tile_i) {
      for (int sl = 0; sl < S; ++sl) {
        WorkItem w{};
        w.i0 = int(s.offset) + i0;
        w.ni = std::min(td->tile_i, s.n - i0);
        w.j0 = int(s.offset) + sl * len;
        w.nj = std::min(len, s.n - sl * len);
        w.law = (s.law == NBODY_LAW_LJC_LINEAR) ? kLawLJCLin : s.law;
        w.slice = sl;
        w.eps2 = s.eps2;
        w.pj0 = pbase + (sl * len) / 2;  // slices start at even local indices
        items.push_back(w);
      }
    }
  }
  // Longest-processing-time first: big items start early, small ones fill in.
  std::stable_sort(items.begin(), items.end(), [](const WorkItem &a, const WorkItem &b) {
    return (long long)a.ni * a.nj > (long long)b.ni * b.nj;
  });
  std::vector<int> sys_of(size_t(total), -1);
  for (int k = 0; k < nsys; ++k)
    for (int i = 0; i < systems[k].n; ++i) sys_of[size_t(systems[k].offset + i)] = k;

  nbody_batch_plan *p = new nbody_batch_plan();
  p->device = dev;
  p->sms = sms;
  p->sys.assign(systems, systems + nsys);
  p->total = total;
  p->td = td;
  p->flags = flags;
  p->n_items = int(items.size());
  p->max_slices = max_slices;
  p->grid = std::min(grid, p->n_items);
  auto fail = [&](int code) {
    free_plan(p);
    return code;
  };
  cudaError_t e = cudaSuccess;
  if ((e = cudaMalloc(&p->d_items, sizeof(WorkItem) * items.size())) != cudaSuccess ||
      (e = cudaMalloc(&p->d_sys, sizeof(SysInfo) * info.size())) != cudaSuccess ||
      (e = cudaMalloc(&p->d_sys_of, sizeof(int) * sys_of.size())) != cudaSuccess ||
      (e = cudaMalloc(&p->d_part, sizeof(float4) * (td->sym ? 1 : 2) * size_t(max_slices) *
                                      size_t(total))) != cudaSuccess ||
      (e = cudaMemcpy(p->d_items, items.data(), sizeof(WorkItem) * items.size(),
                      cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(p->d_sys, info.data(), sizeof(SysInfo) * info.size(),
                      cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(p->d_sys_of, sys_of.data(), sizeof(int) * sys_of.size(),
                      cudaMemcpyHostToDevice)) != cudaSuccess ||
      (td->packed &&
       ((e = cudaMalloc(&p->d_jgrav, sizeof(float4) * (td->sym ? size_t(f4_law[0] + 1)
                                                                 : 2 * size_t(pairs_law[0] + 1)))) !=
            cudaSuccess ||
        (e = cudaMalloc(&p->d_jljc, sizeof(float4) * (td->sym ? size_t(f4_law[1] + 1)
                                                                : 3 * size_t(pairs_law[1] + 1)))) !=
            cudaSuccess ||
        (e = cudaMalloc(&p->d_sysp, sizeof(int4) * sysp.size())) != cudaSuccess ||
        (e = cudaMemcpy(p->d_sysp, sysp.data(), sizeof(int4) * sysp.size(),
                        cudaMemcpyHostToDevice)) != cudaSuccess))) {
    cudaGetLastError();
    return fail(set_error_msg(NBODY_ENOMEM, "batch plan allocation failed: %s",
                              cudaGetErrorString(e)));
  }
  int st = ensure_counters(p, 8);
  if (st != NBODY_OK) return fail(st);
  *plan = p;
  return NBODY_OK;
}

int nbody_batch_plan_destroy(nbody_batch_plan *plan) {
  clear_error();
  if (plan) cudaDeviceSynchronize();
  free_plan(plan);
  return NBODY_OK;
}

int64_t nbody_batch_plan_particles(const nbody_batch_plan *plan) {
  return plan ? plan->total : 0;
}

int nbody_batch_run(nbody_batch_plan *plan, void *pos_m, void *vel, void *acc, const void *prm,
                    int32_t nsteps, uint32_t flags, int32_t use_graph, nbody_stream_t stream) {
  clear_error();
  const NvtxRange nvtx_range("nbody_batch_run");
  if (!plan) return set_error_msg(NBODY_EINVAL, "plan is NULL");
  if (nsteps < 0) return set_error_msg(NBODY_EINVAL, "nsteps must be >= 0");
  if (flags & ~(uint32_t)NBODY_ACC_VALID)
    return set_error_msg(NBODY_EINVAL, "unsupported run flags 0x%x", flags);
  for (const void *q : std::initializer_list<const void *>{pos_m, acc})
    if (!q) return set_error_msg(NBODY_EINVAL, "pos_m and acc are required");
  if (nsteps > 0 && !vel) return set_error_msg(NBODY_EINVAL, "vel is required for steps");
  for (const void *q : std::initializer_list<const void *>{pos_m, vel, acc, prm})
    if (q && !aligned16(q)) return set_error_msg(NBODY_EALIGN, "array not 16-byte aligned");
  bool any_ljc = false;
  for (const auto &s : plan->sys) any_ljc |= (s.law != NBODY_LAW_GRAV);
  if (any_ljc && !prm) return set_error_msg(NBODY_EINVAL, "LJC systems need prm");
  for (const void *q : std::initializer_list<const void *>{pos_m, vel, acc, prm})
    if (q && is_host_pointer(q)) return set_error_msg(NBODY_EINVAL, "device pointers only");
  int dev = 0;
  NB_TRY(check_device(&dev, nullptr));
  if (dev != plan->device) return set_error_msg(NBODY_EINVAL, "plan belongs to another device");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int *err = nullptr;
  NB_TRY(error_word(&err));
  NB_TRY(ensure_counters(plan, nsteps + 1));
  float4 *pos = static_cast<float4 *>(pos_m);
  float4 *v = static_cast<float4 *>(vel);
  float4 *a = static_cast<float4 *>(acc);
  const float4 *q = static_cast<const float4 *>(prm);
  if (!use_graph) return enqueue_run(plan, pos, v, a, q, nsteps, flags, err, s);

  const bool hit = plan->gexec && plan->gsteps == nsteps && plan->gflags == flags &&
                   plan->gkey[0] == pos_m && plan->gkey[1] == vel && plan->gkey[2] == acc &&
                   plan->gkey[3] == prm;
  if (!hit) {
    if (plan->gexec) {
      NB_CUDA(cudaGraphExecDestroy(plan->gexec));
      plan->gexec = nullptr;
    }
    if (!plan->cap_stream) NB_CUDA(cudaStreamCreateWithFlags(&plan->cap_stream, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    NB_CUDA(cudaStreamBeginCapture(plan->cap_stream, cudaStreamCaptureModeThreadLocal));
    int st = enqueue_run(plan, pos, v, a, q, nsteps, flags, err, plan->cap_stream);
    cudaError_t ce = cudaStreamEndCapture(plan->cap_stream, &g);
    if (st != NBODY_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (ce != cudaSuccess)
      return set_error_msg(NBODY_ECUDA, "graph capture failed: %s", cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&plan->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess)
      return set_error_msg(NBODY_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ce));
    plan->gsteps = nsteps;
    plan->gflags = flags;
    plan->gkey[0] = pos_m;
    plan->gkey[1] = vel;
    plan->gkey[2] = acc;
    plan->gkey[3] = prm;
  }
  NB_CUDA(cudaGraphLaunch(plan->gexec, s));
  return NBODY_OK;
}

int nbody_forces_batched(const nbody_system *systems, int32_t nsys, void *pos_m, void *vel,
                         void *acc, const void *prm, int32_t nsteps, uint32_t flags,
                         nbody_stream_t stream) {
  clear_error();
  const NvtxRange nvtx_range("nbody_forces_batched");
  nbody_batch_plan *p = nullptr;
  NB_TRY(nbody_batch_plan_create(systems, nsys,
                                 flags & (NBODY_PRECISE_RSQRT | NBODY_NO_COMPENSATION), -1, &p));
  int st = nbody_batch_run(p, pos_m, vel, acc, prm, nsteps, flags & NBODY_ACC_VALID, 0, stream);
  if (st == NBODY_OK) st = sync_and_check(reinterpret_cast<cudaStream_t>(stream));
  std::string keep = st != NBODY_OK ? std::string(last_error_text()) : std::string();
  nbody_batch_plan_destroy(p);
  if (st != NBODY_OK) set_error_msg(st, "%s", keep.c_str());
  return st;
}

}  // extern "C"
