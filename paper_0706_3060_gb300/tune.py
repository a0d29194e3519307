"""Autotuner for the all-pairs force kernels.

For each law and problem size it times every compiled tile configuration
(threads x targets-per-thread x j-lanes) with several j-splits through the
C ABI, keeps the fastest, installs it with nbody_set_tuned for that size bucket
(floor(log2 N)), and stores the table in a JSON cache keyed by the GPU name and
SM count. ``load_cache()`` re-installs a stored table on the same kind of GPU.

    python -m paper_0706_3060_gb300.tune --law grav --n 1024 16384 262144
"""
from __future__ import annotations

import argparse
import json
import math
import os

import numpy as np

from . import api
from ._lib import (LAW_GRAV, LAW_LJC, LAW_LJC_LINEAR, TABLE_BATCHED, TABLE_GRAV_FIXED,
                   TABLE_JERK, TABLE_VJP_GRAV, TABLE_VJP_LJC, TABLE_VJP_LJC_LINEAR)

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")


def _gpu_key(torch):
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}/{p.multi_processor_count}"


def _inputs(torch, law, n, seed=0):
    rng = np.random.default_rng(seed)
    dev = torch.device("cuda", torch.cuda.current_device())
    if law == LAW_GRAV:
        x = rng.standard_normal((n, 3)).astype(np.float32)
        pos = np.concatenate([x, np.full((n, 1), 1.0 / n, np.float32)], 1)
        return torch.from_numpy(pos).to(dev).contiguous(), None
    # atoms on a jittered cubic lattice (spacing 3.6 A, as in the 45 A / 8192 sphere)
    side = int(math.ceil(n ** (1.0 / 3.0)))
    g = np.stack(np.meshgrid(*[np.arange(side)] * 3, indexing="ij"), -1).reshape(-1, 3)[:n]
    x = (g * 3.6 + rng.uniform(-0.5, 0.5, (n, 3))).astype(np.float32)
    pos = np.concatenate([x, np.full((n, 1), 12.0, np.float32)], 1)
    pos_t = torch.from_numpy(pos).to(dev).contiguous()
    q = torch.from_numpy(rng.uniform(-0.8, 0.8, n)).to(dev)
    s = torch.from_numpy(rng.uniform(2.5, 3.8, n)).to(dev)
    e = torch.from_numpy(rng.uniform(0.05, 0.2, n)).to(dev)
    t = torch.from_numpy(rng.integers(0, 4, n).astype(np.int32)).to(dev)
    return pos_t, api.pack_ljc(q, s, e, t)


def time_config(torch, law, pos, prm, tile, jsplit, reps=5):
    """Median device milliseconds of one force evaluation."""
    acc = torch.empty_like(pos)
    kw = dict(law=law, eps=0.01, tile=tile, jsplit=jsplit, out=acc)
    api.forces(pos, prm, **kw)
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        api.forces(pos, prm, **kw)
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def _vjp_timer(torch, table):
    """Timing function of one VJP (tables 5, 6) or acceleration + jerk (table 7)
    evaluation, with the same signature as time_config."""
    def run(torch_, law, pos, prm, tile, jsplit, reps=5):
        n = pos.shape[0]
        lam = torch.randn((n, 4), device=pos.device)
        if table == TABLE_JERK:
            fn = lambda: api.forces_jerk(pos, lam, eps=0.01, tile=tile, jsplit=jsplit)  # noqa: E731
        else:
            gx = torch.zeros_like(pos)
            gm = torch.zeros(n, device=pos.device)
            vlaw = {TABLE_VJP_GRAV: LAW_GRAV, TABLE_VJP_LJC: LAW_LJC,
                    TABLE_VJP_LJC_LINEAR: LAW_LJC_LINEAR}[table]
            fn = lambda: api.adjoint(pos, lam, prm, law=vlaw, eps=0.01, grad_x=gx,  # noqa: E731
                                     grad_m=gm, tile=tile, jsplit=jsplit)
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
    return run


def tune(law: int, sizes, jsplits=(0, 1, 2, 4, 8, 16, 32), reps=5, verbose=True,
         native=True, tiles=None):
    """Time every tile x j-split of tile table `law` (0-2 force laws, 4 fixed point,
    5-7 the VJP and jerk tables) at each size and install the fastest per size
    bucket. native=True runs the search inside the library (nbody_tune, the same
    j-splits); native=False times each configuration from Python and prints it,
    optionally only the tiles listed in `tiles` (for sizes where timing every
    configuration would take hours)."""
    import torch
    if native:
        table = {}
        in_law = (LAW_LJC if law in (LAW_LJC, LAW_LJC_LINEAR, TABLE_VJP_LJC, TABLE_VJP_LJC_LINEAR)
                  else LAW_GRAV)
        for n in sizes:
            pos, prm = _inputs(torch, in_law, n)
            got = api.tune_table(law, pos, prm, eps=0.01, reps=reps)
            table[str(int(math.floor(math.log2(n))))] = {
                "n": n, "tile": got["tile"], "jsplit": got["jsplit"], "ms": got["ms"],
                "gpairs_per_s": n * n / got["ms"] / 1e6}
            if verbose:
                print(f"table={law} n={n}: tile={got['tile']} jsplit={got['jsplit']} "
                      f"{got['ms']:.4f} ms", flush=True)
        return table
    if law == TABLE_GRAV_FIXED:
        raise ValueError("the fixed-point table is tuned by the library (native=True)")
    timer = time_config
    in_law = law
    if law in (TABLE_VJP_GRAV, TABLE_VJP_LJC, TABLE_VJP_LJC_LINEAR, TABLE_JERK):
        timer = _vjp_timer(torch, law)
        in_law = LAW_LJC if law in (TABLE_VJP_LJC, TABLE_VJP_LJC_LINEAR) else LAW_GRAV
    table = {}
    for n in sizes:
        pos, prm = _inputs(torch, in_law, n)
        results = []
        for tile in (range(api.tile_count(law)) if tiles is None else tiles):
            info = api.tile_info(law, tile)
            tile_i = info["threads"] // info["j_lanes"] * info["i_per_thread"]
            for js in jsplits:
                if js > 0 and js * info["j_tile"] > n:
                    continue
                if js == 0 and tile_i > 4 * n:
                    continue
                ms = timer(torch, law, pos, prm, tile, js, reps)
                results.append((ms, tile, js))
                if verbose:
                    print(f"law={law} n={n} tile={tile} jsplit={js}: {ms:.4f} ms "
                          f"({n * n / ms / 1e6:.1f} G pairs/s)", flush=True)
        ms, tile, js = min(results)
        api.set_tuned(law, n, tile, js)
        table[str(int(math.floor(math.log2(n))))] = {"n": n, "tile": tile, "jsplit": js, "ms": ms,
                                                     "gpairs_per_s": n * n / ms / 1e6}
    return table


def tune_batched(reps=3, verbose=True, nsys=512, seed=3):
    """Pick the mixed-law work-list tile for the batched ensemble (512 systems, N
    log-uniform in [64, 4096]); stored as tile table 3 (batched), bucket 0."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    rng = np.random.default_rng(seed)
    sizes = np.clip(np.rint(np.exp(rng.uniform(math.log(64), math.log(4096), nsys))), 64, 4096)
    sizes = sizes.astype(int)
    total = int(sizes.sum())
    pos = np.zeros((total, 4), np.float32)
    table, off = [], 0
    for k, n in enumerate(sizes):
        if k % 2 == 0:
            pos[off:off + n, :3] = rng.standard_normal((n, 3))
            pos[off:off + n, 3] = 1.0 / n
            table.append(dict(offset=off, n=int(n), law=LAW_GRAV, eps=0.01, dt=1e-3))
        else:
            side = int(math.ceil(n ** (1.0 / 3.0)))
            g = np.stack(np.meshgrid(*[np.arange(side)] * 3, indexing="ij"), -1).reshape(-1, 3)
            pos[off:off + n, :3] = g[:n] * 3.6 + rng.uniform(-0.5, 0.5, (n, 3))
            pos[off:off + n, 3] = 12.0
            table.append(dict(offset=off, n=int(n), law=LAW_LJC, dt=1e-4))
        off += n
    p = torch.from_numpy(pos).to(dev).contiguous()
    prm = api.pack_ljc(torch.from_numpy(rng.uniform(-0.8, 0.8, total)).to(dev),
                       torch.from_numpy(rng.uniform(2.5, 3.8, total)).to(dev),
                       torch.from_numpy(rng.uniform(0.05, 0.2, total)).to(dev),
                       torch.zeros(total, dtype=torch.int32, device=dev))
    vel = torch.zeros_like(p)
    acc = torch.zeros_like(p)
    results = []
    for tile in range(api.tile_count(TABLE_BATCHED)):
        plan = api.BatchPlan(table, tile=tile)
        plan.run(p, vel, acc, prm, nsteps=0, graph=False)
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            plan.run(p, vel, acc, prm, nsteps=0, graph=False)
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        ms = float(np.median(ts))
        results.append((ms, tile))
        plan.close()
        if verbose:
            print(f"batched tile={tile}: {ms:.4f} ms "
                  f"({float(np.sum(sizes.astype(float) ** 2)) / ms / 1e6:.1f} G pairs/s)",
                  flush=True)
    ms, tile = min(results)
    api.set_tuned(TABLE_BATCHED, 1, tile, 0)
    return {"0": {"n": 0, "tile": tile, "jsplit": 0, "ms": ms}}


def save_cache(law: int, table: dict, path: str = CACHE):
    import torch
    data = json.load(open(path)) if os.path.exists(path) else {}
    key = _gpu_key(torch)
    # merge: buckets not re-tuned now keep their stored entries
    data.setdefault(key, {}).setdefault(str(law), {}).update(table)
    with open(path, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)


def load_cache(path: str = CACHE) -> int:
    """Install stored (tile, jsplit) entries for this GPU; returns how many."""
    import torch
    if not os.path.exists(path) or not torch.cuda.is_available():
        return 0
    data = json.load(open(path)).get(_gpu_key(torch), {})
    count = 0
    for law, table in data.items():
        for bucket, ent in table.items():
            api.set_tuned(int(law), 2 ** int(bucket), int(ent["tile"]), int(ent["jsplit"]))
            count += 1
    return count


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--law", choices=["grav", "ljc", "ljclin", "fixed", "batched", "vjp",
                                      "vjpljc", "vjpljclin", "jerk"], default="grav")
    ap.add_argument("--n", type=int, nargs="+", default=[1024, 4096, 16384, 65536, 262144])
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--save", action="store_true")
    ap.add_argument("--python", action="store_true",
                    help="time each configuration from Python and print it (default: the "
                         "library's nbody_tune)")
    ap.add_argument("--tiles", type=int, nargs="+", default=None,
                    help="with --python: only these tiles")
    ap.add_argument("--jsplits", type=int, nargs="+", default=[0, 1, 2, 4, 8, 16, 32],
                    help="with --python: the j-splits to time")
    a = ap.parse_args()
    if a.law == "batched":
        table = tune_batched(reps=a.reps)
        print(json.dumps(table))
        if a.save:
            save_cache(TABLE_BATCHED, table)
        return
    law = {"grav": LAW_GRAV, "ljc": LAW_LJC, "ljclin": LAW_LJC_LINEAR, "fixed": TABLE_GRAV_FIXED,
           "vjp": TABLE_VJP_GRAV, "vjpljc": TABLE_VJP_LJC, "vjpljclin": TABLE_VJP_LJC_LINEAR,
           "jerk": TABLE_JERK}[a.law]
    if (a.tiles is not None or a.jsplits != [0, 1, 2, 4, 8, 16, 32]) and not a.python:
        ap.error("--tiles and --jsplits need --python")
    table = tune(law, a.n, jsplits=tuple(a.jsplits), reps=a.reps, native=not a.python,
                 tiles=a.tiles)
    print(json.dumps(table))
    if a.save:
        save_cache(law, table)


if __name__ == "__main__":
    main()
