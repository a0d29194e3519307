"""Reverse-mode leapfrog as a torch.autograd.Function with checkpointing.

Forward: ``nsteps`` KDK steps through nbody_step with the compensated two-float
state, storing (x, v, low parts) every ``k`` steps, and the positions of the
newest chunk. Backward: for each chunk, newest first, run the reverse sweep
nbody_adjoint_leapfrog (force VJP kernels + fused adjoint updates) over the
chunk's positions; those are recomputed from the checkpoint (positions,
velocities, two-float low parts and the acceleration carried in) with
nbody_step's trace on a second stream while the sweep of the next-newer chunk
runs, so the two fill each other's partial waves (the newest chunk's positions
are stored): k - 1 force evaluations per chunk of k steps.
With merged half-kicks the sweep is

    lam_x += dt/2 J(x_T)^T lam_v                      (only if dL/dv_T != 0)
    for n = T-1 .. 0:  lam_v += dt lam_x;  lam_x += w_n J(x_n)^T lam_v
                       (w_n = dt, w_0 = dt/2)

and returns dL/dx_0 = lam_x, dL/dv_0 = lam_v, dL/dm and, for LJC, dL/dsigma_t
and dL/deps_t. All arithmetic runs in the library's kernels.
"""
from __future__ import annotations

import torch

from . import api
from ._lib import LAW_GRAV, LAW_LJC, LAW_LJC_LINEAR

_LJC_LAWS = (LAW_LJC, LAW_LJC_LINEAR)

_SIDE: dict = {}  # device index -> the stream that recomputes chunk positions


def _side_stream(dev):
    idx = dev.index if dev.index is not None else torch.cuda.current_device()
    if idx not in _SIDE:
        _SIDE[idx] = torch.cuda.Stream(device=dev)
    return _SIDE[idx]


class _Cfg:
    def __init__(self, law, dt, nsteps, k, G, eps, q=None, types=None, kq=None, ntypes=4):
        self.law, self.dt, self.nsteps, self.k = law, float(dt), int(nsteps), int(k)
        self.G, self.eps = float(G), float(eps)
        self.q, self.types, self.kq, self.ntypes = q, types, kq, ntypes


def _prm(cfg, sig_t, eps_t):
    if cfg.law not in _LJC_LAWS:
        return None
    t = cfg.types.long()
    return api.pack_ljc(cfg.q, sig_t.double()[t], eps_t.double()[t], cfg.types, kq=cfg.kq)


class NBodyLeapfrog(torch.autograd.Function):
    """(x0, v0, m, sig_t, eps_t) -> (x_T, v_T) through ``nsteps`` leapfrog steps."""

    @staticmethod
    def forward(ctx, x0, v0, m, sig_t, eps_t, cfg):
        dev = x0.device
        n = x0.shape[0]
        pos = torch.empty((n, 4), dtype=torch.float32, device=dev)
        pos[:, :3] = x0.detach()
        pos[:, 3] = m.detach()
        vel = torch.zeros((n, 4), dtype=torch.float32, device=dev)
        vel[:, :3] = v0.detach()
        acc = torch.empty_like(pos)
        lo = torch.zeros((2 * n, 4), dtype=torch.float32, device=dev)  # two-float state
        prm = _prm(cfg, sig_t, eps_t)
        ckpts = []
        done = 0
        last_trace = None
        while done < cfg.nsteps:
            steps = min(cfg.k, cfg.nsteps - done)
            # the checkpoint keeps a(x) at its positions too (carried in from the
            # previous chunk), so that its recompute starts without an evaluation
            ckpts.append((pos.clone(), vel.clone(), lo.clone(),
                          acc.clone() if done > 0 else None))
            # The newest chunk is the first one the backward pass needs: keep its
            # positions now instead of recomputing them from the checkpoint.
            if done + steps == cfg.nsteps:
                last_trace = torch.empty(((steps + 1) * n, 4), dtype=torch.float32, device=dev)
            api.step(pos, vel, acc, prm, dt=cfg.dt, nsteps=steps, law=cfg.law, G=cfg.G,
                     eps=cfg.eps, acc_valid=done > 0, state_lo=lo, trace=last_trace)
            done += steps
        ctx.cfg = cfg
        ctx.ckpts = ckpts
        ctx.last_trace = last_trace
        ctx.prm = prm
        ctx.save_for_backward(pos)
        return pos[:, :3].clone(), vel[:, :3].clone()

    @staticmethod
    def backward(ctx, gx, gv):
        cfg = ctx.cfg
        (pos_T,) = ctx.saved_tensors
        n = pos_T.shape[0]
        dev = pos_T.device
        lam_x = torch.zeros((n, 4), dtype=torch.float32, device=dev)
        lam_v = torch.zeros((n, 4), dtype=torch.float32, device=dev)
        if gx is not None:
            lam_x[:, :3] = gx
        if gv is not None:
            lam_v[:, :3] = gv
        grad_m = torch.zeros(n, dtype=torch.float32, device=dev)
        grad_t = torch.zeros(2 * cfg.ntypes, dtype=torch.float64, device=dev)
        gt = grad_t if cfg.law in _LJC_LAWS else None
        if gv is not None and bool(torch.any(gv != 0)):
            api.adjoint(pos_T, lam_v, ctx.prm, law=cfg.law, G=cfg.G, eps=cfg.eps,
                        alpha=0.5 * cfg.dt, grad_x=lam_x, grad_m=grad_m, grad_types=gt,
                        ntypes=cfg.ntypes, accumulate=True)
        nck = len(ctx.ckpts)
        starts = [cfg.k * c for c in range(nck)]
        main = torch.cuda.current_stream(dev)
        side = _side_stream(dev)
        side.wait_stream(main)  # checkpoints and prm were written on the main stream
        side_acc = []

        def recompute(c):
            """Enqueue chunk c's positions on the side stream; (trace, done event).
            The sweep reads x_0 .. x_{steps-1} of the chunk: steps - 1 leapfrog
            steps from the checkpoint (with its stored a(x_0) where the forward pass
            carried one in) give exactly those, with the forward's own kernels and
            bits, and no force evaluation whose result the sweep does not use."""
            p0, v0, l0, a0 = ctx.ckpts[c]
            steps = min(cfg.k, cfg.nsteps - starts[c])
            with torch.cuda.stream(side):
                pos, vel, lo = p0.clone(), v0.clone(), l0.clone()
                if not side_acc:
                    side_acc.append(torch.empty_like(pos))
                if a0 is not None:
                    side_acc[0].copy_(a0)
                trace = torch.empty((steps * n, 4), dtype=torch.float32, device=dev)
                api.step(pos, vel, side_acc[0], ctx.prm, dt=cfg.dt, nsteps=steps - 1,
                         law=cfg.law, G=cfg.G, eps=cfg.eps, acc_valid=a0 is not None,
                         trace=trace, state_lo=lo, stream=side)
            done = torch.cuda.Event()
            done.record(side)
            return trace, done

        pending = None
        if nck and ctx.last_trace is None:
            pending = recompute(nck - 1)
        for c in range(nck - 1, -1, -1):
            steps = min(cfg.k, cfg.nsteps - starts[c])
            if pending is None:  # the newest chunk, stored by the forward pass
                trace = ctx.last_trace
            else:
                trace, done = pending
                main.wait_event(done)
                trace.record_stream(main)
            pending = recompute(c - 1) if c > 0 else None
            api.adjoint_leapfrog(trace, lam_x, lam_v, ctx.prm, k=steps, dt=cfg.dt,
                                 first=starts[c] == 0, law=cfg.law, G=cfg.G, eps=cfg.eps,
                                 grad_m=grad_m, grad_types=gt, ntypes=cfg.ntypes, stream=main)
        g_sig = g_eps = None
        if cfg.law in _LJC_LAWS:
            g_sig = grad_t[:cfg.ntypes].to(torch.float32)
            g_eps = grad_t[cfg.ntypes:].to(torch.float32)
        return lam_x[:, :3].clone(), lam_v[:, :3].clone(), grad_m, g_sig, g_eps, None


def leapfrog(x0, v0, m, *, dt, nsteps, k=20, G=1.0, eps=0.0, law=LAW_GRAV, q=None,
             types=None, sig_t=None, eps_t=None, kq=None):
    """Differentiable leapfrog: returns (x_T, v_T); gradients flow to x0, v0, m
    and (LJC) sig_t, eps_t. Gravity by default; pass law=LAW_LJC (or
    LAW_LJC_LINEAR, the linear dielectric) with per-atom charges q (float64),
    int32 types and per-type sig_t, eps_t for LJ + Coulomb; kq defaults to
    k_e / 80 (constant) or k_e / 4 (linear, dielectric 4 r)."""
    if law in _LJC_LAWS:
        if kq is None:
            kq = api.COULOMB_K / (80.0 if law == LAW_LJC else 4.0)
        ntypes = int(sig_t.shape[0])
        cfg = _Cfg(law, dt, nsteps, k, G, eps, q=q, types=types, kq=kq, ntypes=ntypes)
    else:
        cfg = _Cfg(law, dt, nsteps, k, G, eps)
        sig_t = eps_t = torch.zeros(0, device=x0.device)
    return NBodyLeapfrog.apply(x0, v0, m, sig_t, eps_t, cfg)
