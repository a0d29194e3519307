"""Write ``adjoint_plummer16384.json``: the FP64 oracle's answer for the adjoint
workload, so that the GPU gradient at full size can be checked (and reported by
the benchmark) without re-running a minutes-long oracle sweep each time.

Workload: Plummer sphere N = 16384 (seed 4), softening eps = 0.04 N^(-1/3),
200 kick-drift-kick steps at dt = 1e-4, loss L = (1/N) sum_i |x_i(T) - x*_i|^2
with x* = x(0) + 0.01 xi, xi ~ N(0, I) (seed 4). The loss and its gradient are
derived from Eq. 1 (the paper has no adjoint). Inputs are the FP32-rounded values
the GPU consumes; the target is rounded to FP32 as well.

Stored (all from ``oracle/`` only):
  * the loss;
  * dL/dx0, dL/dv0, dL/dm of 256 seeded particles, from the oracle's reverse
    leapfrog (every state stored, two VJPs per step);
  * the RMS magnitude of each full gradient (the floor of the per-particle
    metric);
  * directional central differences of the oracle loss with h = 1e-4 along
    4 seeded directions in (x0, v0, m) (the mass component scaled by 1e-2),
    with the oracle gradient's own directional derivative beside each.

Run from the repository root:  python tests/golden/make_adjoint_golden.py
(about 15 minutes on 8 cores).
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads  # noqa: E402

N, T, DT, K = 16384, 200, 1e-4, 20
H = 1e-4
SAMPLE_SEED, N_SAMPLE = 7, 256
DIR_SEED, N_DIR = 5, 4
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "adjoint_plummer16384.json")


def inputs():
    g = workloads.plummer(N, seed=4, eps=workloads.plummer_softening(N))
    x, v, m = g.f32_as_f64()
    target = workloads.perturbed_target(x, seed=4).astype(np.float32).astype(np.float64)
    return g, x, v, m, target, float(np.float32(g.eps))


def directions():
    """Seeded directions (N, 7): dx, dv and dm (the last column times 1e-2)."""
    d = workloads.random_directions((N, 7), N_DIR, seed=DIR_SEED)
    return [np.concatenate([di[:, :6], di[:, 6:7] * 1e-2], axis=1) for di in d]


def sample_index():
    return np.sort(np.random.default_rng(SAMPLE_SEED).choice(N, size=N_SAMPLE, replace=False))


def main():
    t0 = time.time()
    g, x, v, m, target, eps = inputs()
    sysm = oracle.GravSystem(m, eps=eps)
    xs, _ = oracle.leapfrog(sysm, x, v, DT, T, store=True)
    loss = oracle.target_loss(xs[-1], target)
    ref = oracle.adjoint_leapfrog(sysm, x, v, DT, T, oracle.target_loss_grad(xs[-1], target),
                                  xs=xs)
    print(f"oracle adjoint done in {time.time() - t0:.0f} s", flush=True)

    def loss_at(x0, v0, m0):
        xT, _ = oracle.leapfrog(oracle.GravSystem(m0, eps=eps), x0, v0, DT, T)
        return oracle.target_loss(xT, target)

    fd = []
    for k, d in enumerate(directions()):
        dx, dv, dm = d[:, :3], d[:, 3:6], d[:, 6]
        lp = loss_at(x + H * dx, v + H * dv, m + H * dm)
        lm = loss_at(x - H * dx, v - H * dv, m - H * dm)
        an = float(np.sum(ref["x0"] * dx) + np.sum(ref["v0"] * dv) + np.sum(ref["m"] * dm))
        fd.append({"fd": (lp - lm) / (2 * H), "oracle_directional": an})
        print(f"direction {k}: fd {fd[-1]['fd']:.12e} oracle {an:.12e} "
              f"({time.time() - t0:.0f} s)", flush=True)
    idx = sample_index()
    out = {
        "what": "FP64 oracle gradient of the adjoint workload (Plummer N=16384, eps=0.04 N^-1/3, "
                "200 KDK steps, dt=1e-4, loss (1/N) sum |x_T - x*|^2); written by "
                "make_adjoint_golden.py from oracle/ only",
        "n": N, "steps": T, "dt": DT, "k": K, "eps": eps, "h": H,
        "sample_seed": SAMPLE_SEED, "dir_seed": DIR_SEED,
        "loss": loss,
        "rms": {key: float(np.sqrt(np.mean(np.sum(np.reshape(ref[key], (N, -1)) ** 2, axis=1))))
                for key in ("x0", "v0", "m")},
        "index": idx.tolist(),
        "x0": ref["x0"][idx].tolist(),
        "v0": ref["v0"][idx].tolist(),
        "m": ref["m"][idx].tolist(),
        "fd": fd,
    }
    with open(OUT, "w") as f:
        json.dump(out, f, indent=0)
    print(f"wrote {OUT} in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
