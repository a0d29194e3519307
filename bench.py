"""Benchmark: all-pairs softened gravity + KDK leapfrog on one GB300.

Workload: Plummer sphere, N = 262144, eps = 0.04 N^(-1/3), dt = 1e-4 (the
large gravity workload at the size the headline metric is quoted on). One
"step" is one leapfrog step through the public C ABI (nbody_step with
NBODY_ACC_VALID): first half-kick + drift, the all-pairs force kernel, and the
finalize kernel (compensated partial sums, second half-kick).

Prints one JSON line: interactions/s (N^2 ordered pairs per step, the paper's
count), the force kernel's roofline fraction against the FP32 pipe, the FP64
oracle timed on the host cores, an end-to-end number through host buffers and
the sampled SM clocks. ``--impl reference`` times the FP64 oracle instead.
Under torchrun (N > 1 GPUs) every rank runs an independent replica.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_BENCH = 262144
DT = 1e-4
OPS_PER_PAIR = 12          # FP32 lane ops per pair of the plain gravity kernel (no potential)
# FP32 lane ops per unordered pair of the Newton-symmetric kernel: 3 sub, 3 FMA for s^2,
# 2 MUL for y^3, 2 MUL for the two mass weights, 3 + 3 FMA for the two accumulations
SYM_OPS_PER_UNORDERED_PAIR = 16
# the same for the Newton-symmetric gravity VJP: 6 for d and s^2, 2 for y^2, y^3, 6 for
# w, 6 for lam_j.d and lam_k.d, 2 for d.w, 2 for c, 3 for c d + w, 4 + 4 for the two sides
SYM_VJP_OPS_PER_UNORDERED_PAIR = 35
# and for the Newton-symmetric LJC kernel: the one-sided pair (23, 24 with the linear
# dielectric) plus 3 FMA for the source side
SYM_LJC_OPS_PER_UNORDERED_PAIR = 26
SYM_LJCLIN_OPS_PER_UNORDERED_PAIR = 27
# and for the Newton-symmetric acceleration + jerk: 6 for d and u, 3 for s^2, 2 for y^2,
# y^3, 3 for d.u, 2 for c, 3 for u + c d, then per side 1 weight + 3 + 3 FMA
SYM_GAJ_OPS_PER_UNORDERED_PAIR = 33
# and for the Newton-symmetric LJC VJP: the one-sided pair (48, 49 with the linear
# dielectric) plus 6 for the source's g, 3 for its F, 4 more for the D and E terms
SYM_LJC_VJP_OPS_PER_UNORDERED_PAIR = 61
SYM_LJCLIN_VJP_OPS_PER_UNORDERED_PAIR = 62
PAPER_FLOPS_PER_PAIR = 19  # the paper's flop count per gravity interaction (Table 1, Appendix)
FP32_LANES_PER_SM = 128    # FFMA/FADD/FMUL lanes per SM per clock (4 SMSPs x 32)
SM_MAX_MHZ = 2070.0
CPU_SAMPLE_TARGETS = 131072  # oracle sample: targets x all N sources (~10 s on 16 cores)
CPU_SAMPLE_TARGETS_1T = 2048  # the same on one thread (~3 s)


def _env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def metric_name():
    return "G pair-interactions/s (Plummer N=262144, leapfrog step)"


def config(n_gpus):
    return {"workload": f"plummer-{N_BENCH}-kdk-leapfrog", "n": N_BENCH,
            "eps": 4.0 / N_BENCH ** (1.0 / 3.0) * 0.01, "dt": DT,
            "pairs_per_step": N_BENCH * N_BENCH, "law": "gravity (Eq. 1)",
            "precision": ("FP32 pairs; plain FP32 sums within each block pair, per-block "
                          "partials added as 64-bit fixed point (integer atomics)"),
            "l2": "flushed between timed steps (256 MiB write)",
            "parallelism": f"replicas x{n_gpus}" if n_gpus > 1 else "single GPU"}


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = [r.split(",") for r in self.tmp.read().strip().splitlines() if r.strip()]
        os.unlink(self.tmp.name)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            r = [c.strip() for c in r]
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# oracle (CPU baseline / reference arm)
# ---------------------------------------------------------------------------
def oracle_rate(n_targets: int, seed: int = 1, threads: int | None = None):
    """Time the FP64 oracle on n_targets sampled targets against all N sources,
    on `threads` OpenMP threads (None: all host cores). Returns (pairs/s, s, threads)."""
    import oracle
    import workloads
    prev = oracle.set_threads(None)
    used = oracle.set_threads(threads if threads else os.cpu_count())
    g = workloads.plummer(N_BENCH, seed=seed, eps=workloads.plummer_softening(N_BENCH))
    x, _, m = g.f32_as_f64()
    idx = np.sort(np.random.default_rng(7).choice(N_BENCH, n_targets, replace=False))
    eps = float(np.float32(g.eps))
    oracle.grav_accel(x, m, eps=eps, idx=idx[:64])  # load + warm
    t0 = time.perf_counter()
    oracle.grav_accel(x, m, eps=eps, idx=idx)
    dt = time.perf_counter() - t0
    oracle.set_threads(prev)
    return n_targets * N_BENCH / dt, dt, used


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    import oracle
    oracle.build()
    cores = os.cpu_count()
    n_t = max(256, CPU_SAMPLE_TARGETS // 8)
    for _ in range(args.warmup):
        oracle_rate(n_t // 4)
    tot_pairs, tot_t = 0.0, 0.0
    for _ in range(args.steps):
        r, dt, cores = oracle_rate(n_t)
        tot_pairs += r * dt
        tot_t += dt
    val = tot_pairs / tot_t / 1e9
    out = {"impl": "reference", "metric": metric_name(), "value": val,
           "unit": "G pair-interactions/s", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded Plummer sphere)", "config": config(args.gpus),
           "cpu_baseline": {"value": val, "unit": "G pair-interactions/s", "cores": cores,
                            "kind": "oracle",
                            "sample": f"{n_t} seeded targets x all {N_BENCH} sources per step"},
           "e2e": {"value": val, "unit": "G pair-interactions/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="run only warmup + this many steps (for ncu launch lists)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 0)
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist

    import paper_0706_3060_gb300 as nb
    import workloads

    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    nb._lib.load()  # fails loudly if the CUDA library is not built

    g = workloads.plummer(N_BENCH, seed=1, eps=workloads.plummer_softening(N_BENCH))
    eps = float(np.float32(g.eps))
    x, v, m = g.f32()
    host_pos = np.concatenate([x, m[:, None]], 1).astype(np.float32)
    host_vel = np.concatenate([v, np.zeros((N_BENCH, 1), np.float32)], 1)
    pos = torch.from_numpy(host_pos).to(dev).contiguous()
    vel = torch.from_numpy(host_vel).to(dev).contiguous()
    acc = torch.empty_like(pos)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2
    stream = torch.cuda.current_stream(dev)

    # a(x_0) once, then steps reuse the acceleration of the previous step
    nb.step(pos, vel, acc, dt=DT, nsteps=0, eps=eps)
    for _ in range(args.warmup):
        flush.zero_()
        nb.step(pos, vel, acc, dt=DT, nsteps=1, eps=eps, acc_valid=True)
    torch.cuda.synchronize()
    if args.profile_steps:
        for _ in range(args.profile_steps):
            nb.step(pos, vel, acc, dt=DT, nsteps=1, eps=eps, acc_valid=True)
        torch.cuda.synchronize()
        return

    K = args.steps
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    nb.timing_read(0)
    nb.timing_enable(True)
    t_wall = time.perf_counter()
    for k in range(K):
        flush.zero_()
        starts[k].record(stream)
        nb.step(pos, vel, acc, dt=DT, nsteps=1, eps=eps, acc_valid=True)
        stops[k].record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    nb.timing_enable(False)
    n_force, force_ms = nb.timing_read(0)
    clk = clocks.stop()
    nb.sync_check()
    step_ms = float(sum(s.elapsed_time(e) for s, e in zip(starts, stops)))
    pairs = float(N_BENCH) * N_BENCH
    t_max, value = aggregate(step_ms / 1e3, pairs, K, world, dev)

    # roofline of the dominant kernel (the all-pairs force kernel)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    peak = sms * FP32_LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12          # T lane-op/s
    avg_force_s = force_ms / max(n_force, 1) / 1e3
    tile, _ = nb.get_config(nb.LAW_GRAV, N_BENCH)
    tinfo = nb.tile_info(nb.LAW_GRAV, tile)
    if tinfo["symmetric"]:
        # each unordered pair once, applied to both particles
        ops = SYM_OPS_PER_UNORDERED_PAIR * float(N_BENCH) * (N_BENCH - 1) / 2
        kname, opdesc = "sym_grav_kernel", {"ops_per_unordered_pair": SYM_OPS_PER_UNORDERED_PAIR,
                                            "unordered_pairs": N_BENCH * (N_BENCH - 1) // 2}
    else:
        ops = OPS_PER_PAIR * pairs
        kname, opdesc = "force_kernel<grav>", {"ops_per_pair": OPS_PER_PAIR}
    achieved = ops / avg_force_s / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None,
            "kernel": kname, "tile": tile, "launches_timed": n_force,
            "avg_launch_ms": avg_force_s * 1e3, **opdesc,
            "peak_basis": (f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x {SM_MAX_MHZ:.0f} MHz; "
                           "one FFMA/FADD/FMUL lane op = 1")}
    if clk.get("sm_mhz"):
        roof["frac_at_sampled_clock"] = achieved / (sms * FP32_LANES_PER_SM * clk["sm_mhz"] * 1e6
                                                    / 1e12)
    # DRAM bytes per launch from the committed ncu summary, only if it was taken
    # on the kernel that runs now (same sources and tuning table).
    summary = os.path.join(ROOT, "profiles", ("sym_grav_kernel_plummer262144.md"
                                              if tinfo["symmetric"] else
                                              "force_kernel_grav_plummer262144.md"))
    if os.path.exists(summary):
        import re
        txt = open(summary).read()
        mh = re.search(r"^kernel_hash: (\S+)", txt, re.M)
        mb = re.search(r"^dram_bytes_per_launch: (\d+)", txt, re.M)
        if mh and mb and mh.group(1) == kernel_hash():
            roof["traffic"] = int(mb.group(1))

    # kernels per timed step: kick-drift (fused into the pair interleave of packed
    # tiles), force, finalize(+kick)
    per_step = 3
    out = {"metric": metric_name(), "value": value, "unit": "G pair-interactions/s",
           "n_gpus": world, "steps": K, "warmup": args.warmup, "ms_per_step": step_ms / K,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic (seeded Plummer sphere)", "config": config(world),
           "roofline": roof, "clocks": clk, "gpu_launches": per_step * K,
           "interactions_counted": ("N^2 ordered pair interactions per step"
                                    + ("; the Newton-symmetric kernel evaluates each unordered "
                                       "pair once and applies it to both particles"
                                       if tinfo["symmetric"] else "")),
           "paper_convention_gflops": paper_gflops(value),
           "wall_s_timed_region": t_wall}

    # end to end through the C ABI with pinned host buffers (copies inside)
    hp = torch.from_numpy(host_pos.copy()).pin_memory()
    hv = torch.from_numpy(host_vel.copy()).pin_memory()
    ha = torch.empty_like(hp).pin_memory()
    nb.step(hp, hv, ha, dt=DT, nsteps=0, eps=eps)
    Ke = max(3, min(K, 10))
    te = float("inf")
    for _ in range(3):  # best of three wall-clock runs: host-side noise only adds time
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(Ke):
            nb.step(hp, hv, ha, dt=DT, nsteps=1, eps=eps, acc_valid=True)
        te = min(te, time.perf_counter() - t0)
    out["e2e"] = {"value": pairs * Ke / te / 1e9, "unit": "G pair-interactions/s",
                  "h2d_bytes_per_step": 3 * N_BENCH * 16, "d2h_bytes_per_step": 3 * N_BENCH * 16,
                  "path": ("nbody_step on pinned host buffers (staged H2D, step, D2H, sync); "
                           f"best of 3 wall-clock runs of {Ke} steps")}

    if rank == 0 and world == 1:
        r, dt_cpu, used = oracle_rate(CPU_SAMPLE_TARGETS)
        r1, dt1, _ = oracle_rate(CPU_SAMPLE_TARGETS_1T, threads=1)
        out["cpu_baseline"] = {"value": r / 1e9, "unit": "G pair-interactions/s",
                               "cores": used, "kind": "oracle",
                               "sample": (f"{CPU_SAMPLE_TARGETS} seeded targets x all {N_BENCH} "
                                          f"sources, FP64, {dt_cpu:.1f} s"),
                               "single_thread_value": r1 / 1e9,
                               "single_thread_sample": (f"{CPU_SAMPLE_TARGETS_1T} targets, "
                                                        f"{dt1:.1f} s")}
    if not args.no_extras and rank == 0:
        try:
            out["extras"] = extras(nb, torch, dev, g, eps)
        except Exception as exc:  # the headline line still prints; the failure is reported
            out["extras"] = {"error": repr(exc)}
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def paper_gflops(gpairs_per_s: float) -> float:
    """Interactions per second in the paper's convention (19 flops per gravity
    interaction, rsqrt counted as one), for comparison with Table 1."""
    return PAPER_FLOPS_PER_PAIR * gpairs_per_s


def aggregate(t_local: float, pairs_per_step: float, steps: int, world: int, device):
    """Whole-job throughput: every rank ran `steps` steps of `pairs_per_step` pairs;
    the job time is the slowest rank's (MAX all-reduce). Returns (t_max, G pairs/s)."""
    import torch
    t_max = t_local
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([t_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    return t_max, world * pairs_per_step * steps / t_max / 1e9


def kernel_hash() -> str:
    """Identity of the timed force kernel: its sources with comments and spacing
    removed (a comment edit does not change the kernel) and the tuned gravity
    entry for the bench size (other tuning-table entries do not change it)."""
    import hashlib
    import re
    h = hashlib.sha1()
    pkg = os.path.join(ROOT, "paper_0706_3060_gb300")
    for f in ("csrc/force_kernel.cuh", "csrc/sym_kernel.cuh", "csrc/device_common.cuh",
              "csrc/fixed_point.cuh", "csrc/force_grav.cu"):
        with open(os.path.join(pkg, f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    bucket = str(int(math.floor(math.log2(N_BENCH))))
    with open(os.path.join(pkg, "tuned.json")) as fh:
        data = json.load(fh)
    ent = sorted((k, json.dumps({x: v.get("0", {}).get(bucket, {}).get(x)
                                 for x in ("tile", "jsplit")}, sort_keys=True))
                 for k, v in data.items())
    h.update(json.dumps(ent).encode())
    return h.hexdigest()[:16]


def extras(nb, torch, dev, g, eps):
    """Accuracy and the secondary forms, measured on the same GPU (not timed above)."""
    import oracle
    ex = {}
    x, v, m = g.f32()
    pos = torch.from_numpy(np.concatenate([x, m[:, None]], 1)).to(dev).contiguous()
    acc = nb.forces(pos, eps=eps).cpu().numpy()
    idx = np.sort(np.random.default_rng(0).choice(N_BENCH, 1024, replace=False))
    ref = oracle.grav_accel(x.astype(np.float64), m.astype(np.float64), eps=eps, idx=idx)
    e = np.linalg.norm(acc[idx, :3] - ref, axis=1) / np.linalg.norm(ref, axis=1)
    ex["force_err_rms"] = float(np.sqrt(np.mean(e * e)))
    ex["force_err_max"] = float(e.max())
    ex["force_err_sample"] = "1024 seeded targets vs FP64 oracle"
    ex["default_mode"] = ("hardware rsqrt; Newton-symmetric tile: plain sums per block pair, "
                          "per-block partials added as 64-bit fixed point with integer atomics "
                          "(with NBODY_NO_COMPENSATION: stored per block and added plainly)")
    # the other precision modes on the same targets: Newton-refined rsqrt, plain
    # FP32 sums, 64-bit fixed-point sums (error and device time per evaluation)
    out_acc = torch.empty_like(pos)
    for name, kw in (("precise_rsqrt", {"precise": True}),
                     ("uncompensated", {"compensated": False}),
                     ("fixed_point", {"fixed": True})):
        am = nb.forces(pos, eps=eps, **kw).cpu().numpy()
        em = np.linalg.norm(am[idx, :3] - ref, axis=1) / np.linalg.norm(ref, axis=1)
        ms = _device_ms(torch, lambda: nb.forces(pos, eps=eps, out=out_acc, **kw), reps=3)
        ex[f"{name}_err_rms"] = float(np.sqrt(np.mean(em * em)))
        ex[f"{name}_err_max"] = float(em.max())
        ex[f"{name}_262144_gpairs_per_s"] = float(N_BENCH) ** 2 / ms / 1e6
    # energy drift over 100 steps at dt = 1e-4 (FP64 diagnostics on the GPU)
    vel = torch.from_numpy(np.concatenate([v, np.zeros((N_BENCH, 1), np.float32)], 1)).to(dev)
    a2 = torch.empty_like(pos)
    d = nb.step(pos, vel, a2, dt=DT, nsteps=100, eps=eps, report_every=100).cpu().numpy()
    E0, E1 = d[0, 0] + d[0, 1], d[1, 0] + d[1, 1]
    ex["energy_drift_100_steps"] = float((E1 - E0) / abs(E0))
    ex.update(size_sweep_extras(nb, torch, dev))
    ex.update(batched_extras(nb, torch, dev))
    ex.update(adjoint_extras(nb, torch, dev))
    ex.update(secondary_kernel_extras(nb, torch, dev, pos, eps))
    ex["roofline_by_form"] = roofline_by_form(nb, torch, dev)
    ex["oracle_gpairs_per_s"] = oracle_family_rates()
    return ex


def roofline_by_form(nb, torch, dev):
    """Each all-pairs kernel against the FP32 lane peak: its FP32 lane ops per
    pair (counted from the source; MUFU apart) times the pairs of one launch,
    over the launch's device time from the library's kernel timers (CUDA events
    on the launching stream), median of 3 timed launches after one warm-up."""
    import workloads
    props = torch.cuda.get_device_properties(dev)
    peak = props.multi_processor_count * FP32_LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12
    K = 332.0637

    def kernel_ms(fn, which):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(3):
            nb.timing_read(which)
            nb.timing_enable(True)
            fn()
            torch.cuda.synchronize()
            nb.timing_enable(False)
            k, ms = nb.timing_read(which)
            ts.append(ms / max(k, 1))
        return float(np.median(ts))

    def grav(n, seed=1):
        g = workloads.plummer(n, seed=seed, eps=workloads.plummer_softening(n))
        x, v, m = g.f32()
        p = torch.from_numpy(np.concatenate([x, m[:, None]], 1)).to(dev).contiguous()
        vv = torch.from_numpy(np.concatenate([v, np.zeros((n, 1), np.float32)], 1)).to(dev)
        return p, vv.contiguous(), float(np.float32(g.eps))

    def ljc(n, kq):
        s = workloads.ljc_sphere(n, seed=2)
        x, _, m, q, st, et = s.f32()
        p = torch.from_numpy(np.concatenate([x, m[:, None]], 1)).to(dev).contiguous()
        prm = nb.pack_ljc(torch.from_numpy(q.astype(np.float64)).to(dev),
                          torch.from_numpy(st.astype(np.float64)[s.types]).to(dev),
                          torch.from_numpy(et.astype(np.float64)[s.types]).to(dev),
                          torch.from_numpy(s.types).to(dev), kq=kq)
        return p, prm

    out = {"peak_tflops": peak, "basis": "FP32 lane ops per pair x pairs / kernel time"}
    rows = []
    pg, vg, eg = grav(262144)
    acc = torch.empty_like(pg)
    gtile, _ = nb.get_config(nb.LAW_GRAV, 262144)
    if nb.tile_info(nb.LAW_GRAV, gtile)["symmetric"]:
        # ops per ordered pair: half the symmetric kernel's ops per unordered pair
        rows.append(("gravity forces (Newton-symmetric)", 262144,
                     SYM_OPS_PER_UNORDERED_PAIR / 2 * (262144 - 1) / 262144,
                     kernel_ms(lambda: nb.forces(pg, eps=eg, out=acc), 0)))
    # the fastest one-sided tile (256 threads x 2 targets, 8 j-slices)
    rows.append(("gravity forces (one-sided)", 262144, 12,
                 kernel_ms(lambda: nb.forces(pg, eps=eg, out=acc, tile=12, jsplit=8), 0)))
    jt, _ = nb.get_config(nb.TABLE_JERK, 262144)
    if nb.tile_info(nb.TABLE_JERK, jt)["symmetric"]:
        rows.append(("acceleration + jerk (Newton-symmetric)", 262144,
                     SYM_GAJ_OPS_PER_UNORDERED_PAIR / 2 * (262144 - 1) / 262144,
                     kernel_ms(lambda: nb.forces_jerk(pg, vg, eps=eg), 0)))
    # the fastest one-sided jerk tile (packed, 128 threads x 2 targets, 32 j-slices)
    rows.append(("acceleration + jerk (one-sided)", 262144, 26,
                 kernel_ms(lambda: nb.forces_jerk(pg, vg, eps=eg, tile=6, jsplit=32), 0)))
    lp, lprm = ljc(65536, K / 80.0)
    lacc = torch.empty_like(lp)
    lp2, lprm2 = ljc(65536, K / 4.0)
    for name, law, prm_, one, sym, one_tile in (
            ("LJC forces", nb.LAW_LJC, lprm, 23, SYM_LJC_OPS_PER_UNORDERED_PAIR, (6, 32)),
            ("LJC(linear) forces", nb.LAW_LJC_LINEAR, lprm2, 24,
             SYM_LJCLIN_OPS_PER_UNORDERED_PAIR, (3, 32))):
        p_ = lp if law == nb.LAW_LJC else lp2
        lt, _ = nb.get_config(law, 65536)
        if nb.tile_info(law, lt)["symmetric"]:
            rows.append((f"{name} (Newton-symmetric)", 65536, sym / 2 * (65536 - 1) / 65536,
                         kernel_ms(lambda: nb.forces(p_, prm_, law=law, out=lacc), 0)))
        # the fastest one-sided tile at this size
        rows.append((f"{name} (one-sided)", 65536, one,
                     kernel_ms(lambda: nb.forces(p_, prm_, law=law, out=lacc, tile=one_tile[0],
                                                 jsplit=one_tile[1]), 0)))
    pv, _, ev = grav(65536, seed=4)
    lam = torch.randn_like(pv)
    gx, gm = torch.empty_like(pv), torch.empty(65536, device=dev)
    vtile, _ = nb.get_config(nb.TABLE_VJP_GRAV, 65536)
    if nb.tile_info(nb.TABLE_VJP_GRAV, vtile)["symmetric"]:
        rows.append(("gravity VJP (Newton-symmetric)", 65536,
                     SYM_VJP_OPS_PER_UNORDERED_PAIR / 2 * (65536 - 1) / 65536,
                     kernel_ms(lambda: nb.adjoint(pv, lam, eps=ev, grad_x=gx, grad_m=gm), 1)))
    # the fastest one-sided VJP tile at this size (256 threads x 1 target, unrolled x4)
    rows.append(("gravity VJP (one-sided)", 65536, 29,
                 kernel_ms(lambda: nb.adjoint(pv, lam, eps=ev, grad_x=gx, grad_m=gm, tile=8,
                                              jsplit=16), 1)))
    gt = torch.zeros(8, dtype=torch.float64, device=dev)
    for name, law, table, p_, prm_, one, sym, one_tile in (
            ("LJC VJP", nb.LAW_LJC, nb.TABLE_VJP_LJC, lp, lprm, 48,
             SYM_LJC_VJP_OPS_PER_UNORDERED_PAIR, (6, 16)),
            ("LJC(linear) VJP", nb.LAW_LJC_LINEAR, nb.TABLE_VJP_LJC_LINEAR, lp2, lprm2, 49,
             SYM_LJCLIN_VJP_OPS_PER_UNORDERED_PAIR, (0, 16))):
        vt, _ = nb.get_config(table, 65536)
        if nb.tile_info(table, vt)["symmetric"]:
            rows.append((f"{name} (Newton-symmetric)", 65536, sym / 2 * (65536 - 1) / 65536,
                         kernel_ms(lambda: nb.adjoint(p_, lam, prm_, law=law, grad_x=gx,
                                                      grad_m=gm, grad_types=gt), 1)))
        # the fastest one-sided tile at this size
        rows.append((f"{name} (one-sided)", 65536, one,
                     kernel_ms(lambda: nb.adjoint(p_, lam, prm_, law=law, grad_x=gx, grad_m=gm,
                                                  grad_types=gt, tile=one_tile[0],
                                                  jsplit=one_tile[1]), 1)))
    for name, n, ops, ms in rows:
        pairs = float(n) * n
        t = ops * pairs / (ms * 1e-3) / 1e12
        out[name] = {"n": n, "ops_per_pair": ops, "kernel_ms": ms,
                     "gpairs_per_s": pairs / (ms * 1e-3) / 1e9, "achieved_tflops": t,
                     "frac": t / peak}
    # the batched persistent kernel over the 512-system ensemble: one-sided tiles do
    # 12 ops per gravity pair and 23 per LJC pair; the Newton-symmetric tiles 16 and
    # 26 per unordered pair
    ens = workloads.ensemble(nsys=512, seed=3)
    bpos, bvel, bprm, table = _ensemble_arrays(nb, torch, dev, ens)
    bacc = torch.zeros_like(bpos)
    pg2 = sum(float(x.n) ** 2 for x in ens.systems if isinstance(x, workloads.GravInput))
    pl2 = sum(float(x.n) ** 2 for x in ens.systems if not isinstance(x, workloads.GravInput))
    pgu = sum(x.n * (x.n - 1) / 2 for x in ens.systems if isinstance(x, workloads.GravInput))
    plu = sum(x.n * (x.n - 1) / 2 for x in ens.systems if not isinstance(x, workloads.GravInput))
    btile, _ = nb.get_config(nb.TABLE_BATCHED, 0)
    forms = [("batched ensemble (one-sided)", 9)]
    if nb.tile_info(nb.TABLE_BATCHED, btile)["symmetric"]:
        forms.insert(0, ("batched ensemble (Newton-symmetric)", btile))
    for name, tl in forms:
        plan = nb.BatchPlan(table, tile=tl)
        ms = kernel_ms(lambda: plan.run(bpos, bvel, bacc, bprm, nsteps=0, graph=False), 0)
        plan.close()
        if nb.tile_info(nb.TABLE_BATCHED, tl)["symmetric"]:
            ops = SYM_OPS_PER_UNORDERED_PAIR * pgu + SYM_LJC_OPS_PER_UNORDERED_PAIR * plu
        else:
            ops = 12 * pg2 + 23 * pl2
        t = ops / (ms * 1e-3) / 1e12
        out[name] = {"systems": 512, "tile": tl, "pairs": pg2 + pl2, "kernel_ms": ms,
                     "gpairs_per_s": (pg2 + pl2) / (ms * 1e-3) / 1e9,
                     "achieved_tflops": t, "frac": t / peak}
    return out


def oracle_family_rates():
    """The FP64 oracle's rate for each force form, timed on this host's cores on one
    evaluation of a small case (gravity forms: Plummer N = 16384; LJC forms: the
    8192-atom sphere), for comparison with the GPU rates beside them."""
    import oracle
    import workloads
    g = workloads.plummer(16384, seed=4, eps=workloads.plummer_softening(16384))
    x, v, m = g.f32_as_f64()
    e = float(np.float32(g.eps))
    s = workloads.ljc_sphere(8192, seed=2)
    lx, _, lm, q, st, et = s.f32_as_f64()
    lam_g = np.random.default_rng(0).standard_normal((16384, 3))
    lam_l = np.random.default_rng(1).standard_normal((8192, 3))
    cases = {
        "grav": (16384, lambda: oracle.grav_accel(x, m, eps=e)),
        "jerk": (16384, lambda: oracle.grav_jerk(x, v, m, eps=e)),
        "grav_vjp": (16384, lambda: oracle.grav_vjp(x, m, lam_g, eps=e)),
        "ljc": (8192, lambda: oracle.ljc_force(lx, q, st[s.types], et[s.types])),
        "ljc_linear": (8192, lambda: oracle.ljc_force(lx, q, st[s.types], et[s.types],
                                                      kq=oracle.COULOMB_K / 4.0, linear=True)),
        "ljc_vjp": (8192, lambda: oracle.ljc_vjp(lx, lm, q, s.types, st, et, lam_l)),
    }
    out = {"cores": oracle.set_threads(None)}
    for name, (n, fn) in cases.items():
        t0 = time.perf_counter()
        fn()
        out[name] = float(n) * n / (time.perf_counter() - t0) / 1e9
    return out


def _device_ms(torch, fn, reps=5):
    fn()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def _back_to_back_ms(torch, fn, calls=20, reps=5):
    """Device milliseconds per call with `calls` eager calls issued back to back
    (no synchronization between them: the host's launch work for one call overlaps
    the GPU's work for the previous ones, as in a simulation loop)."""
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(calls):
            fn()
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b) / calls)
    return float(np.median(ts))


def _graph_ms(torch, fn, calls=10, reps=5):
    """Device milliseconds per call with the calls replayed from a CUDA graph (no
    host launch overhead between them): warm up on the capture stream, capture
    `calls` calls, replay."""
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        for _ in range(3):
            fn()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        for _ in range(calls):
            fn()
    g.replay()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        g.replay()
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b) / calls)
    return float(np.median(ts))


def secondary_kernel_extras(nb, torch, dev, pos, eps):
    """Throughput of the other force forms on the same GPU (device time per call,
    and for the 8192-atom cases also per call issued back to back and per call
    replayed from a CUDA graph, which hide or remove the host launch overhead that
    dominates a synchronous call this small):
    LJ + Coulomb (constant and linear dielectric) on the 8192-atom sphere;
    acceleration + jerk, a Hermite step, an active subset of 1024 targets and the
    fixed-point mode on the N = 262144 Plummer sphere."""
    import workloads
    out = {}
    s = workloads.ljc_sphere(8192, seed=2)
    x, v, m, q, st, et = s.f32()
    lpos = torch.from_numpy(np.concatenate([x, m[:, None]], 1)).to(dev).contiguous()
    prm = nb.pack_ljc(torch.from_numpy(q.astype(np.float64)).to(dev),
                      torch.from_numpy(st.astype(np.float64)[s.types]).to(dev),
                      torch.from_numpy(et.astype(np.float64)[s.types]).to(dev),
                      torch.from_numpy(s.types).to(dev), kq=332.0637 / 80.0)
    lacc = torch.empty_like(lpos)
    ms = _device_ms(torch, lambda: nb.forces(lpos, prm))
    out["ljc_8192_gpairs_per_s"] = 8192.0 ** 2 / ms / 1e6
    ms = _back_to_back_ms(torch, lambda: nb.forces(lpos, prm, out=lacc))
    out["ljc_8192_back_to_back_gpairs_per_s"] = 8192.0 ** 2 / ms / 1e6
    ms = _graph_ms(torch, lambda: nb.forces(lpos, prm, out=lacc))
    out["ljc_8192_graph_gpairs_per_s"] = 8192.0 ** 2 / ms / 1e6
    n = pos.shape[0]
    vel = torch.zeros_like(pos)
    ms = _device_ms(torch, lambda: nb.forces_jerk(pos, vel, eps=eps), reps=3)
    out["jerk_262144_gpairs_per_s"] = float(n) ** 2 / ms / 1e6
    idx = torch.from_numpy(np.random.default_rng(1).choice(n, 1024, replace=False)
                           .astype(np.int32)).to(dev)
    ms = _device_ms(torch, lambda: nb.forces_subset(pos, idx, eps=eps))
    out["subset_1024_of_262144_gpairs_per_s"] = 1024.0 * n / ms / 1e6
    prm_lin = nb.pack_ljc(torch.from_numpy(q.astype(np.float64)).to(dev),
                          torch.from_numpy(st.astype(np.float64)[s.types]).to(dev),
                          torch.from_numpy(et.astype(np.float64)[s.types]).to(dev),
                          torch.from_numpy(s.types).to(dev), kq=332.0637 / 4.0)
    ms = _device_ms(torch, lambda: nb.forces(lpos, prm_lin, law=nb.LAW_LJC_LINEAR))
    out["ljc_linear_8192_gpairs_per_s"] = 8192.0 ** 2 / ms / 1e6
    ms = _back_to_back_ms(torch, lambda: nb.forces(lpos, prm_lin, law=nb.LAW_LJC_LINEAR,
                                                    out=lacc))
    out["ljc_linear_8192_back_to_back_gpairs_per_s"] = 8192.0 ** 2 / ms / 1e6
    ms = _graph_ms(torch, lambda: nb.forces(lpos, prm_lin, law=nb.LAW_LJC_LINEAR, out=lacc))
    out["ljc_linear_8192_graph_gpairs_per_s"] = 8192.0 ** 2 / ms / 1e6
    # 20 leapfrog steps in one call (one force and one finalize launch per step
    # after the first), from a copy of the sphere at rest
    lp, lv = lpos.clone(), torch.zeros_like(lpos)
    ms = _device_ms(torch, lambda: nb.step(lp, lv, lacc, prm, dt=1e-5, nsteps=20))
    out["ljc_8192_step20_gpairs_per_s"] = 20 * 8192.0 ** 2 / ms / 1e6
    lam = torch.randn_like(lpos)
    lgx, lgm = torch.empty_like(lpos), torch.empty(lpos.shape[0], device=dev)
    lgt = torch.zeros(8, dtype=torch.float64, device=dev)
    vjp = lambda: nb.adjoint(lpos, lam, prm, grad_x=lgx, grad_m=lgm, grad_types=lgt)  # noqa: E731
    ms = _device_ms(torch, vjp)
    out["ljc_vjp_8192_gpairs_per_s"] = 8192.0 ** 2 / ms / 1e6
    ms = _back_to_back_ms(torch, vjp)
    out["ljc_vjp_8192_back_to_back_gpairs_per_s"] = 8192.0 ** 2 / ms / 1e6
    ms = _graph_ms(torch, vjp)
    out["ljc_vjp_8192_graph_gpairs_per_s"] = 8192.0 ** 2 / ms / 1e6
    hp, hv = pos.clone(), vel.clone()
    ha, hj = torch.empty_like(pos), torch.empty_like(pos)
    nb.hermite_step(hp, hv, ha, hj, dt=DT, nsteps=0, eps=eps)
    ms = _device_ms(torch, lambda: nb.hermite_step(hp, hv, ha, hj, dt=DT, nsteps=1, eps=eps,
                                                    acc_valid=True), reps=3)
    out["hermite_step_262144_gpairs_per_s"] = float(n) ** 2 / ms / 1e6
    return out


def size_sweep_extras(nb, torch, dev, sizes=(16384, 65536, 262144, 1048576)):
    """One force evaluation (tuned tile, device time) on seeded Plummer spheres of each
    size with softening 0.04 N^(-1/3); at the smallest size also 20 leapfrog steps in
    one call; at the largest size, the error of 256 sampled targets against the FP64
    oracle."""
    import oracle
    import workloads
    rate, err = {}, {}
    for n in sizes:
        g = workloads.plummer(n, seed=1, eps=workloads.plummer_softening(n))
        e32 = float(np.float32(g.eps))
        x, _, m = g.f32()
        p = torch.from_numpy(np.concatenate([x, m[:, None]], 1)).to(dev).contiguous()
        ms = _device_ms(torch, lambda: nb.forces(p, eps=e32), reps=3)
        rate[str(n)] = float(n) ** 2 / ms / 1e6
        if n == sizes[0]:  # 20 leapfrog steps in one call at the smallest size
            pv, v0, a0 = p.clone(), torch.zeros_like(p), torch.empty_like(p)
            ms = _device_ms(torch, lambda: nb.step(pv, v0, a0, dt=1e-5, nsteps=20, eps=e32))
            steps20 = {"n": n, "gpairs_per_s": 20 * float(n) ** 2 / ms / 1e6}
        if n == sizes[-1]:
            a = nb.forces(p, eps=e32).cpu().numpy()
            idx = np.sort(np.random.default_rng(7).choice(n, 256, replace=False))
            ref = oracle.grav_accel(x.astype(np.float64), m.astype(np.float64), eps=e32, idx=idx)
            e = np.linalg.norm(a[idx, :3] - ref, axis=1) / np.linalg.norm(ref, axis=1)
            err = {"n": n, "rms": float(np.sqrt(np.mean(e * e))), "max": float(e.max()),
                   "sample": "256 seeded targets vs FP64 oracle"}
        del p
    return {"forces_gpairs_per_s_by_n": rate, "force_err_largest_n": err,
            "step20_smallest_n": steps20}


def _ensemble_arrays(nb, torch, dev, ens):
    """Concatenate an ensemble into shared float4 arrays and a system table."""
    import workloads
    total = sum(s.n for s in ens.systems)
    pos = np.zeros((total, 4), np.float32)
    vel = np.zeros((total, 4), np.float32)
    q, sg, ep = np.zeros(total), np.full(total, 3.0), np.full(total, 0.1)
    ty = np.zeros(total, np.int32)
    table, off = [], 0
    for s in ens.systems:
        if isinstance(s, workloads.GravInput):
            x, v, m = s.f32()
            table.append(dict(offset=off, n=s.n, law=nb.LAW_GRAV, G=1.0,
                              eps=float(np.float32(s.eps)), dt=1e-3))
        else:
            x, v, m, qq, st, et = s.f32()
            q[off:off + s.n] = qq
            sg[off:off + s.n] = st.astype(np.float64)[s.types]
            ep[off:off + s.n] = et.astype(np.float64)[s.types]
            ty[off:off + s.n] = s.types
            table.append(dict(offset=off, n=s.n, law=nb.LAW_LJC, dt=1e-4))
        pos[off:off + s.n, :3], pos[off:off + s.n, 3], vel[off:off + s.n, :3] = x, m, v
        off += s.n
    prm = nb.pack_ljc(torch.from_numpy(q).to(dev), torch.from_numpy(sg).to(dev),
                      torch.from_numpy(ep).to(dev), torch.from_numpy(ty).to(dev),
                      kq=332.0637 / 80.0)
    return (torch.from_numpy(pos).to(dev).contiguous(), torch.from_numpy(vel).to(dev).contiguous(),
            prm, table)


def _time(torch, fn, reps=3):
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        best = min(best, time.perf_counter() - t0)
    return best


def batched_extras(nb, torch, dev, nsys=512, steps=50):
    """512 systems, N log-uniform in [64, 4096], half gravity / half LJ + Coulomb,
    50 leapfrog steps: one persistent launch per step under a CUDA graph, against
    one nbody_step call per system, issued eagerly and replayed from a CUDA graph."""
    import workloads
    ens = workloads.ensemble(nsys=nsys, seed=3)
    pos, vel, prm, table = _ensemble_arrays(nb, torch, dev, ens)
    acc = torch.zeros_like(pos)
    plan = nb.BatchPlan(table)
    p0, v0 = pos.clone(), vel.clone()

    def batched():
        pos.copy_(p0)
        vel.copy_(v0)
        plan.run(pos, vel, acc, prm, nsteps=steps, graph=True)

    t_b = _time(torch, batched)
    pairs = float(sum(s.n * s.n for s in ens.systems)) * (steps + 1)
    views = [(pos[t["offset"]:t["offset"] + t["n"]], vel[t["offset"]:t["offset"] + t["n"]],
              acc[t["offset"]:t["offset"] + t["n"]], prm[t["offset"]:t["offset"] + t["n"]], t)
             for t in table]

    def per_system():
        pos.copy_(p0)
        vel.copy_(v0)
        for p, v, a, q, t in views:
            if t["law"] == nb.LAW_GRAV:
                nb.step(p, v, a, dt=t["dt"], nsteps=steps, eps=t["eps"])
            else:
                nb.step(p, v, a, q, dt=t["dt"], nsteps=steps)

    t_s = _time(torch, per_system, reps=1)
    # the same per-system calls replayed from one CUDA graph (no host launch cost;
    # the workspace of the capturing stream is sized by an uncaptured run first)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        per_system()
    torch.cuda.synchronize()
    g_ps = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_ps, stream=side):
        per_system()
    t_sg = _time(torch, g_ps.replay)
    del g_ps
    # accuracy beside the rate: forces of every 32nd system against the FP64 oracle
    import oracle
    pos.copy_(p0)
    plan.run(pos, vel, acc, prm, nsteps=0, graph=False)
    a = acc.cpu().numpy()
    worst_rms = worst_max = 0.0
    for k in range(0, nsys, 32):
        s, t = ens.systems[k], table[k]
        if isinstance(s, workloads.GravInput):
            xs, _, ms = s.f32_as_f64()
            ref = oracle.grav_accel(xs, ms, eps=t["eps"])
        else:
            xs, _, ms, q, st, et = s.f32_as_f64()
            ref = oracle.LJCSystem(ms, q, s.types, st, et, 332.0637 / 80.0).accel(xs)
        got = a[t["offset"]:t["offset"] + t["n"], :3]
        e = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
        worst_rms = max(worst_rms, float(np.sqrt(np.mean(e * e))))
        worst_max = max(worst_max, float(e.max()))
    return {"batched_systems": nsys, "batched_steps": steps,
            "batched_force_err_rms_worst": worst_rms, "batched_force_err_max_worst": worst_max,
            "batched_force_err_sample": f"systems 0, 32, ..., {nsys - 32} vs FP64 oracle",
            "batched_system_steps_per_s": nsys * steps / t_b,
            "batched_gpairs_per_s": pairs / t_b / 1e9,
            "per_system_launch_system_steps_per_s": nsys * steps / t_s,
            "per_system_graph_system_steps_per_s": nsys * steps / t_sg,
            "batched_speedup_vs_per_system": t_s / t_b,
            "batched_speedup_vs_per_system_graph": t_sg / t_b}


def adjoint_extras(nb, torch, dev, n=16384, steps=200, k=20):
    """Plummer N = 16384, 200 steps at dt = 1e-4, checkpoints every 20 steps:
    backward (recompute + reverse sweep) time over forward time."""
    import workloads
    from paper_0706_3060_gb300.autograd import leapfrog
    g = workloads.plummer(n, seed=4, eps=workloads.plummer_softening(n))
    x, v, m = g.f32()
    tgt = torch.from_numpy(workloads.perturbed_target(x.astype(np.float64), seed=4)
                           .astype(np.float32)).to(dev)
    eps = float(np.float32(g.eps))
    def timed(kk):
        best_f = best_b = float("inf")
        for _ in range(3):
            x0 = torch.from_numpy(x).to(dev).requires_grad_(True)
            v0 = torch.from_numpy(v).to(dev).requires_grad_(True)
            m0 = torch.from_numpy(m).to(dev).requires_grad_(True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            xT, _ = leapfrog(x0, v0, m0, dt=1e-4, nsteps=steps, k=kk, eps=eps)
            loss = ((xT - tgt) ** 2).sum() / n
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            loss.backward()
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            best_f, best_b = min(best_f, t1 - t0), min(best_b, t2 - t1)
        return best_f, best_b

    best_f, best_b = timed(k)
    all_f, all_b = timed(steps)  # one chunk: every position kept, nothing recomputed
    out = {"adjoint_n": n, "adjoint_steps": steps, "adjoint_checkpoint_every": k,
           "adjoint_forward_s": best_f, "adjoint_backward_s": best_b,
           "adjoint_forward_ratio": best_b / best_f,
           "adjoint_forward_ratio_all_positions_kept": all_b / all_f,
           "adjoint_positions_kept_bytes": (steps + 1) * n * 16}
    out.update(adjoint_accuracy(torch, dev))
    return out


def adjoint_accuracy(torch, dev, n=16384, steps=200, k=20, dt=1e-4):
    """The gradients of the timed adjoint configuration itself against the FP64
    oracle's answer stored in tests/golden/adjoint_plummer16384.json (written by
    make_adjoint_golden.py from oracle/ only): per-particle error of dL/dx0,
    dL/dv0, dL/dm on its 256 seeded particles (denominator floored at 10% of the
    RMS gradient), and the directional derivatives against central differences
    (h = 1e-4) of the oracle loss."""
    import json
    import workloads
    from paper_0706_3060_gb300.autograd import leapfrog
    path = os.path.join(ROOT, "tests", "golden", "adjoint_plummer16384.json")
    golden = json.load(open(path))
    assert (golden["n"], golden["steps"], golden["k"]) == (n, steps, k)
    g = workloads.plummer(n, seed=4, eps=workloads.plummer_softening(n))
    x, v, m = g.f32()
    target = workloads.perturbed_target(x.astype(np.float64), seed=4).astype(np.float32)
    x0 = torch.from_numpy(x).to(dev).requires_grad_(True)
    v0 = torch.from_numpy(v).to(dev).requires_grad_(True)
    m0 = torch.from_numpy(m).to(dev).requires_grad_(True)
    xT, _ = leapfrog(x0, v0, m0, dt=dt, nsteps=steps, k=k, eps=float(np.float32(g.eps)))
    loss = ((xT - torch.from_numpy(target).to(dev)) ** 2).sum() / n
    loss.backward()
    got = {"x0": x0.grad.double().cpu().numpy(), "v0": v0.grad.double().cpu().numpy(),
           "m": m0.grad.double().cpu().numpy()}
    idx = np.asarray(golden["index"])
    out = {"adjoint_grad_err_case": f"Plummer N = {n}, {steps} steps, k = {k}: 256 seeded "
                                    "particles vs the stored FP64 oracle gradient "
                                    "(per particle, floor 10% of RMS); directional "
                                    "derivatives vs oracle central differences (h = 1e-4)",
           "adjoint_loss_rel_err": abs(float(loss.detach()) - golden["loss"]) / golden["loss"]}
    for key in ("x0", "v0", "m"):
        ref = np.reshape(np.asarray(golden[key]), (len(idx), -1))
        num = np.linalg.norm(np.reshape(got[key][idx], (len(idx), -1)) - ref, axis=1)
        e = num / np.maximum(np.linalg.norm(ref, axis=1), 0.1 * golden["rms"][key])
        out[f"adjoint_grad_err_{key}_rms"] = float(np.sqrt(np.mean(e * e)))
        out[f"adjoint_grad_err_{key}_max"] = float(e.max())
    dirs = workloads.random_directions((n, 7), len(golden["fd"]), seed=golden["dir_seed"])
    worst = 0.0
    for d, fd in zip(dirs, golden["fd"]):
        an = float(np.sum(got["x0"] * d[:, :3]) + np.sum(got["v0"] * d[:, 3:6])
                   + np.sum(got["m"] * d[:, 6] * 1e-2))
        worst = max(worst, abs(an - fd["fd"]) / abs(fd["fd"]))
    out["adjoint_fd_rel_err_max"] = worst
    return out

if __name__ == "__main__":
    main()
