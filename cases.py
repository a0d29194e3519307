"""Run one named workload a few times through the C ABI (for profilers such as
``ncu -k regex:<kernel>``): each case builds its seeded inputs, runs ``--warmup``
untimed calls and ``--iters`` more, then synchronizes.

    python cases.py grav262144 --warmup 1 --iters 2
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np


def _grav(nb, torch, dev, n, seed=1):
    import workloads
    g = workloads.plummer(n, seed=seed, eps=workloads.plummer_softening(n))
    x, v, m = g.f32()
    pos = torch.from_numpy(np.concatenate([x, m[:, None]], 1)).to(dev).contiguous()
    vel = torch.from_numpy(np.concatenate([v, np.zeros((n, 1), np.float32)], 1)).to(dev)
    return pos, vel.contiguous(), float(np.float32(g.eps))


def _ljc(nb, torch, dev, n, seed=2):
    import workloads
    s = workloads.ljc_sphere(n, seed=seed)
    x, v, m, q, st, et = s.f32()
    pos = torch.from_numpy(np.concatenate([x, m[:, None]], 1)).to(dev).contiguous()
    prm = nb.pack_ljc(torch.from_numpy(q.astype(np.float64)).to(dev),
                      torch.from_numpy(st.astype(np.float64)[s.types]).to(dev),
                      torch.from_numpy(et.astype(np.float64)[s.types]).to(dev),
                      torch.from_numpy(s.types).to(dev), kq=332.0637 / 80.0)
    return pos, prm


def _ensemble(nb, torch, dev, nsys=512, seed=3):
    """The 512-system ensemble (N log-uniform in [64, 4096], even systems gravity,
    odd LJ + Coulomb) packed back to back, with its system table."""
    import workloads
    ens = workloads.ensemble(nsys=nsys, seed=seed)
    total = sum(s.n for s in ens.systems)
    pos = np.zeros((total, 4), np.float32)
    q, sg, ep = np.zeros(total), np.full(total, 3.0), np.full(total, 0.1)
    ty = np.zeros(total, np.int32)
    table, off = [], 0
    for s in ens.systems:
        if isinstance(s, workloads.GravInput):
            x, _, m = s.f32()
            table.append(dict(offset=off, n=s.n, law=nb.LAW_GRAV, eps=float(np.float32(s.eps)),
                              dt=1e-3))
        else:
            x, _, m, qq, st, et = s.f32()
            q[off:off + s.n] = qq
            sg[off:off + s.n] = st.astype(np.float64)[s.types]
            ep[off:off + s.n] = et.astype(np.float64)[s.types]
            ty[off:off + s.n] = s.types
            table.append(dict(offset=off, n=s.n, law=nb.LAW_LJC, dt=1e-4))
        pos[off:off + s.n, :3], pos[off:off + s.n, 3] = x, m
        off += s.n
    prm = nb.pack_ljc(torch.from_numpy(q).to(dev), torch.from_numpy(sg).to(dev),
                      torch.from_numpy(ep).to(dev), torch.from_numpy(ty).to(dev),
                      kq=332.0637 / 80.0)
    return torch.from_numpy(pos).to(dev).contiguous(), prm, table


def build_case(name, nb, torch, dev, tile=-1, jsplit=0):
    """Return a zero-argument callable running one call of the named workload
    (force and VJP cases with the given tile and j-split; -1 / 0: tuned)."""
    if name in ("grav65536", "grav262144"):
        pos, _, eps = _grav(nb, torch, dev, int(name[4:]))
        acc = torch.empty_like(pos)
        return lambda: nb.forces(pos, eps=eps, out=acc, tile=tile, jsplit=jsplit)
    if name in ("ljc8192", "ljc65536"):
        pos, prm = _ljc(nb, torch, dev, int(name[3:]))
        acc = torch.empty_like(pos)
        return lambda: nb.forces(pos, prm, out=acc, tile=tile, jsplit=jsplit)
    if name == "ljcvjp8192":
        pos, prm = _ljc(nb, torch, dev, 8192)
        lam = torch.randn_like(pos)
        gx = torch.empty_like(pos)
        gm = torch.empty(pos.shape[0], device=dev)
        gt = torch.zeros(8, dtype=torch.float64, device=dev)
        return lambda: nb.adjoint(pos, lam, prm, grad_x=gx, grad_m=gm, grad_types=gt)
    if name == "vjp16384":
        pos, _, eps = _grav(nb, torch, dev, 16384, seed=4)
        lam = torch.randn_like(pos)
        gx = torch.empty_like(pos)
        gm = torch.empty(pos.shape[0], device=dev)
        return lambda: nb.adjoint(pos, lam, eps=eps, grad_x=gx, grad_m=gm, tile=tile,
                                  jsplit=jsplit)
    if name == "adjoint16384":  # forward + backward of the adjoint workload (200 steps, k = 20)
        import numpy as np
        import workloads
        from paper_0706_3060_gb300.autograd import leapfrog
        n = 16384
        g = workloads.plummer(n, seed=4, eps=workloads.plummer_softening(n))
        x, v, m = g.f32()
        tgt = torch.from_numpy(workloads.perturbed_target(x.astype(np.float64), seed=4)
                               .astype(np.float32)).to(dev)
        eps = float(np.float32(g.eps))

        def run():
            x0 = torch.from_numpy(x).to(dev).requires_grad_(True)
            v0 = torch.from_numpy(v).to(dev).requires_grad_(True)
            m0 = torch.from_numpy(m).to(dev).requires_grad_(True)
            xT, _ = leapfrog(x0, v0, m0, dt=1e-4, nsteps=200, k=20, eps=eps)
            (((xT - tgt) ** 2).sum() / n).backward()
        return run
    if name in ("jerk65536", "jerk262144"):
        pos, vel, eps = _grav(nb, torch, dev, int(name[4:]))
        return lambda: nb.forces_jerk(pos, vel, eps=eps)
    if name == "batched512":
        pos, prm, table = _ensemble(nb, torch, dev)
        vel = torch.zeros_like(pos)
        acc = torch.zeros_like(pos)
        plan = nb.BatchPlan(table)
        return lambda: plan.run(pos, vel, acc, prm, nsteps=0, graph=False)
    raise ValueError(f"unknown case {name}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["grav65536", "grav262144", "ljc8192", "ljcvjp8192", "ljc65536", "vjp16384",
                                     "jerk65536", "jerk262144", "batched512", "adjoint16384"])
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--iters", type=int, default=2)
    ap.add_argument("--tile", type=int, default=-1)
    ap.add_argument("--jsplit", type=int, default=0)
    a = ap.parse_args()
    root = os.path.dirname(os.path.abspath(__file__))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch

    import paper_0706_3060_gb300 as nb
    dev = torch.device("cuda", 0)
    fn = build_case(a.case, nb, torch, dev, a.tile, a.jsplit)
    for _ in range(a.warmup + a.iters):
        fn()
    torch.cuda.synchronize()
    nb.sync_check()
    print(f"{a.case}: ok")


if __name__ == "__main__":
    main()
