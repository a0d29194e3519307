"""GPU parity: the batched persistent kernel (many uneven systems, mixed laws,
one launch per force evaluation, CUDA-graph replay) against the FP64 oracle,
system by system; graph and eager runs agree bitwise; system order does not
change any system's result."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from gpu_util import assert_forces_close, dev, lib, traj_errors

pytestmark = pytest.mark.gpu

DT_GRAV = 1e-3
DT_LJC = 1e-4


def _pack_ensemble(ens, order=None, gap=3):
    """Concatenate the systems (with `gap` unused slots between them) into
    shared float4 arrays; returns tensors and the system table."""
    nb = lib()
    order = list(range(len(ens.systems))) if order is None else order
    offs, off = {}, 0
    for k in order:
        offs[k] = off
        off += ens.systems[k].n + gap
    total = off
    pos = np.zeros((total, 4), np.float32)
    pos[:, 3] = 1.0
    vel = np.zeros((total, 4), np.float32)
    q = np.zeros(total)
    sg = np.full(total, 3.0)
    ep = np.full(total, 0.1)
    ty = np.zeros(total, np.int32)
    table = []
    for k, s in enumerate(ens.systems):
        o = offs[k]
        if isinstance(s, workloads.GravInput):
            x, v, m = s.f32()
            table.append(dict(offset=o, n=s.n, law=nb.LAW_GRAV, G=1.0, eps=float(np.float32(s.eps)),
                              dt=DT_GRAV))
        else:
            x, v, m, qq, st, et = s.f32()
            q[o:o + s.n] = qq.astype(np.float64)
            sg[o:o + s.n] = st.astype(np.float64)[s.types]
            ep[o:o + s.n] = et.astype(np.float64)[s.types]
            ty[o:o + s.n] = s.types
            table.append(dict(offset=o, n=s.n, law=nb.LAW_LJC, dt=DT_LJC))
        pos[o:o + s.n, :3] = x
        pos[o:o + s.n, 3] = m
        vel[o:o + s.n, :3] = v
    d = dev()
    prm = nb.pack_ljc(torch.from_numpy(q).to(d), torch.from_numpy(sg).to(d),
                      torch.from_numpy(ep).to(d), torch.from_numpy(ty).to(d),
                      kq=332.0637 / 80.0)
    return (torch.from_numpy(pos).to(d).contiguous(), torch.from_numpy(vel).to(d).contiguous(),
            prm, table)


def _oracle_system(s):
    if isinstance(s, workloads.GravInput):
        x, v, m = s.f32_as_f64()
        return oracle.GravSystem(m, eps=float(np.float32(s.eps))), x, v
    x, v, m, q, st, et = s.f32_as_f64()
    return oracle.LJCSystem(m, q, s.types, st, et, 332.0637 / 80.0), x, v


@pytest.fixture(scope="module")
def small_ensemble():
    return workloads.ensemble(nsys=24, seed=31, nmin=40, nmax=700)


def test_batched_forces_match_oracle(small_ensemble):
    nb = lib()
    pos, vel, prm, table = _pack_ensemble(small_ensemble)
    acc = torch.zeros_like(pos)
    plan = nb.BatchPlan(table)
    plan.run(pos, vel, acc, prm, nsteps=0, graph=False)
    a = acc.cpu().numpy()
    for k, s in enumerate(small_ensemble.systems):
        sysm, x, _ = _oracle_system(s)
        o = table[k]["offset"]
        assert_forces_close(a[o:o + s.n, :3], sysm.accel(x), what=f"system {k} n={s.n}")


def test_batched_steps_graph_eager_and_order(small_ensemble):
    nb = lib()
    p1, v1, q1, t1 = _pack_ensemble(small_ensemble)
    a1 = torch.zeros_like(p1)
    plan = nb.BatchPlan(t1)
    plan.run(p1, v1, a1, q1, nsteps=5, graph=True)
    torch.cuda.synchronize()
    p2, v2, q2, _ = _pack_ensemble(small_ensemble)
    a2 = torch.zeros_like(p2)
    plan.run(p2, v2, a2, q2, nsteps=5, graph=False)
    assert torch.equal(p1, p2) and torch.equal(v1, v2)
    # replaying the cached graph continues the trajectory: 5 + 5 == 10 eager
    plan.run(p1, v1, a1, q1, nsteps=5, graph=True, acc_valid=True)
    plan.run(p2, v2, a2, q2, nsteps=5, graph=False, acc_valid=True)
    assert torch.equal(p1, p2) and torch.equal(v1, v2)
    # reversed system order: each system's result is unchanged bit for bit
    order = list(range(len(small_ensemble.systems)))[::-1]
    p3, v3, q3, t3 = _pack_ensemble(small_ensemble, order=order, gap=5)
    a3 = torch.zeros_like(p3)
    plan3 = nb.BatchPlan(t3)
    plan3.run(p3, v3, a3, q3, nsteps=10, graph=False)
    for k, s in enumerate(small_ensemble.systems):
        o1, o3 = t1[k]["offset"], t3[k]["offset"]
        assert torch.equal(p1[o1:o1 + s.n], p3[o3:o3 + s.n]), k
    # trajectories against the oracle
    pn = p1.cpu().numpy()
    vn = v1.cpu().numpy()
    for k, s in enumerate(small_ensemble.systems):
        sysm, x, v = _oracle_system(s)
        dt = DT_GRAV if isinstance(s, workloads.GravInput) else DT_LJC
        xr, vr = oracle.leapfrog(sysm, x, v, dt, 10)
        o = t1[k]["offset"]
        ex = traj_errors(pn[o:o + s.n, :3], xr)
        assert ex[0] <= 1e-6 and ex[1] <= 1e-5, (k, ex)


def test_full_ensemble_sampled():
    """512 systems, N log-uniform in [64, 4096], half gravity, half LJ + Coulomb:
    one persistent launch; every 16th system checked against the oracle."""
    nb = lib()
    ens = workloads.ensemble(nsys=512, seed=3)
    pos, vel, prm, table = _pack_ensemble(ens, gap=0)
    acc = torch.zeros_like(pos)
    plan = nb.BatchPlan(table)
    plan.run(pos, vel, acc, prm, nsteps=0, graph=True)
    a = acc.cpu().numpy()
    for k in range(0, 512, 16):
        s = ens.systems[k]
        sysm, x, _ = _oracle_system(s)
        o = table[k]["offset"]
        assert_forces_close(a[o:o + s.n, :3], sysm.accel(x), what=f"system {k} n={s.n}")
    nb.sync_check()


def test_one_shot_and_bad_tables():
    nb = lib()
    ens = workloads.ensemble(nsys=4, seed=5, nmin=50, nmax=90)
    pos, vel, prm, table = _pack_ensemble(ens)
    acc = torch.zeros_like(pos)
    nb.forces_batched(table, pos, vel, acc, prm, nsteps=0)
    for k, s in enumerate(ens.systems):
        sysm, x, _ = _oracle_system(s)
        o = table[k]["offset"]
        assert_forces_close(acc[o:o + s.n, :3].cpu().numpy(), sysm.accel(x))
    bad = [dict(offset=0, n=10, law=0, dt=1e-3), dict(offset=5, n=10, law=0, dt=1e-3)]
    with pytest.raises(nb.NBodyError):
        nb.BatchPlan(bad)   # overlapping systems
    with pytest.raises(nb.NBodyError):
        nb.BatchPlan([dict(offset=0, n=0, law=0, dt=1e-3)])


@pytest.mark.parametrize("tile", range(14))
def test_batched_every_tile(small_ensemble, tile):
    """Every compiled batched tile (scalar and packed f32x2, with odd-sized systems
    padded inside their pair buffers) against the oracle, then 3 steps."""
    nb = lib()
    pos, vel, prm, table = _pack_ensemble(small_ensemble)
    acc = torch.zeros_like(pos)
    plan = nb.BatchPlan(table, tile=tile)
    plan.run(pos, vel, acc, prm, nsteps=0, graph=False)
    a = acc.cpu().numpy()
    for k, s in enumerate(small_ensemble.systems):
        sysm, x, _ = _oracle_system(s)
        o = table[k]["offset"]
        assert_forces_close(a[o:o + s.n, :3], sysm.accel(x), what=f"tile {tile} system {k}")
    p2, v2, q2, _ = _pack_ensemble(small_ensemble)
    plan.run(p2, v2, acc, q2, nsteps=3, graph=True)
    pn = p2.cpu().numpy()
    for k, s in enumerate(small_ensemble.systems[:6]):
        sysm, x, v = _oracle_system(s)
        dt = DT_GRAV if isinstance(s, workloads.GravInput) else DT_LJC
        xr, _ = oracle.leapfrog(sysm, x, v, dt, 3)
        o = table[k]["offset"]
        ex = traj_errors(pn[o:o + s.n, :3], xr)
        assert ex[0] <= 1e-6, (tile, k, ex)


def test_batched_tiny_and_large_systems():
    """Systems of 1, 2, 3 and 5 particles (the single one feels no force) beside
    one of 20000 split into many j-slices, gravity and LJC, every tile."""
    nb = lib()
    rng = np.random.default_rng(44)
    sizes = [1, 2, 3, 5, 20000, 3, 1]
    gs = [workloads.plummer(n, seed=100 + k, eps=0.02) if n > 1 else None
          for k, n in enumerate(sizes)]
    total = sum(sizes)
    pos = np.zeros((total, 4), np.float32)
    table, off = [], 0
    for k, n in enumerate(sizes):
        if n == 1:
            pos[off] = [rng.standard_normal(), rng.standard_normal(), 0.5, 1.0]
        else:
            x, _, m = gs[k].f32()
            pos[off:off + n, :3], pos[off:off + n, 3] = x, m
        table.append(dict(offset=off, n=n, law=nb.LAW_GRAV, eps=float(np.float32(0.02)),
                          dt=1e-3))
        off += n
    d = dev()
    p = torch.from_numpy(pos).to(d)
    for tile in range(nb.tile_count(nb.TABLE_BATCHED)):
        acc = torch.full_like(p, float("nan"))
        plan = nb.BatchPlan(table, tile=tile)
        plan.run(p, torch.zeros_like(p), acc, None, nsteps=0, graph=False)
        a = acc.cpu().numpy()
        for k, t in enumerate(table):
            o, n = t["offset"], t["n"]
            if n == 1:
                assert np.all(a[o, :3] == 0.0), (tile, k)
                continue
            x, _, m = gs[k].f32_as_f64()
            if n > 5000:
                idx = np.sort(rng.choice(n, 512, replace=False))
                ref = oracle.grav_accel(x, m, eps=float(np.float32(0.02)), idx=idx)
                assert_forces_close(a[o + idx, :3], ref, what=f"tile {tile} n={n}")
            else:
                ref = oracle.grav_accel(x, m, eps=float(np.float32(0.02)))
                assert_forces_close(a[o:o + n, :3], ref, what=f"tile {tile} n={n}")
        plan.close()


def test_batched_linear_dielectric_systems():
    """Gravity, LJC(constant) and LJC(linear) systems in one plan (each LJC
    system packed with its own kq), on every batched tile, against the oracle;
    then 3 graph-replayed steps of a linear-dielectric system."""
    nb = lib()
    K = 332.0637
    laws = [nb.LAW_GRAV, nb.LAW_LJC, nb.LAW_LJC_LINEAR, nb.LAW_LJC_LINEAR, nb.LAW_LJC]
    sizes = [300, 257, 410, 129, 600]
    d = dev()
    total = sum(sizes)
    pos = np.zeros((total, 4), np.float32)
    vel = np.zeros((total, 4), np.float32)
    prm = torch.zeros((total, 4), dtype=torch.float32, device=d)
    table, refs, off = [], [], 0
    for k, (law, n) in enumerate(zip(laws, sizes)):
        if law == nb.LAW_GRAV:
            g = workloads.plummer(n, seed=200 + k, eps=0.02)
            x, v, m = g.f32()
            eps = float(np.float32(0.02))
            table.append(dict(offset=off, n=n, law=law, eps=eps, dt=1e-3))
            xd, vd, md = g.f32_as_f64()
            refs.append((oracle.GravSystem(md, eps=eps), xd, vd))
        else:
            s = workloads.ljc_sphere(n, seed=200 + k)
            x, v, m, q, st, et = s.f32()
            kq = K / 80.0 if law == nb.LAW_LJC else K / 4.0
            prm[off:off + n] = nb.pack_ljc(torch.from_numpy(q.astype(np.float64)).to(d),
                                           torch.from_numpy(st.astype(np.float64)[s.types]).to(d),
                                           torch.from_numpy(et.astype(np.float64)[s.types]).to(d),
                                           torch.from_numpy(s.types).to(d), kq=kq)
            table.append(dict(offset=off, n=n, law=law, dt=1e-4))
            xd, vd, md, qd, std, etd = s.f32_as_f64()
            refs.append((oracle.LJCSystem(md, qd, s.types, std, etd, kq,
                                          linear=law == nb.LAW_LJC_LINEAR), xd, vd))
        pos[off:off + n, :3], pos[off:off + n, 3], vel[off:off + n, :3] = x, m, v
        off += n
    p0 = torch.from_numpy(pos).to(d)
    v0 = torch.from_numpy(vel).to(d)
    for tile in range(nb.tile_count(nb.TABLE_BATCHED)):
        acc = torch.zeros_like(p0)
        plan = nb.BatchPlan(table, tile=tile)
        plan.run(p0, v0, acc, prm, nsteps=0, graph=False)
        a = acc.cpu().numpy()
        for k, (sysm, x, _) in enumerate(refs):
            o, n = table[k]["offset"], table[k]["n"]
            assert_forces_close(a[o:o + n, :3], sysm.accel(x), what=f"tile {tile} system {k}")
        plan.close()
    p1, v1 = p0.clone(), v0.clone()
    acc = torch.zeros_like(p1)
    plan = nb.BatchPlan(table)
    plan.run(p1, v1, acc, prm, nsteps=3, graph=True)
    sysm, x, v = refs[2]
    xr, _ = oracle.leapfrog(sysm, x, v, 1e-4, 3)
    o, n = table[2]["offset"], table[2]["n"]
    ex = traj_errors(p1[o:o + n, :3].cpu().numpy(), xr)
    assert ex[0] <= 1e-6, ex


def test_batched_50_steps_against_conditioning_floor(small_ensemble):
    """The batched workload's 50 steps (graph-replayed) for a 24-system ensemble:
    each system's trajectory against the oracle, within 10x the oracle's own
    conditioning floor (its run from positions perturbed by 1e-7 relative)."""
    nb = lib()
    pos, vel, prm, table = _pack_ensemble(small_ensemble)
    acc = torch.zeros_like(pos)
    plan = nb.BatchPlan(table)
    plan.run(pos, vel, acc, prm, nsteps=50, graph=True)
    pn = pos.cpu().numpy()
    rng = np.random.default_rng(6)
    for k, s in enumerate(small_ensemble.systems):
        sysm, x, v = _oracle_system(s)
        dt = DT_GRAV if isinstance(s, workloads.GravInput) else DT_LJC
        xr, _ = oracle.leapfrog(sysm, x, v, dt, 50)
        xp, _ = oracle.leapfrog(sysm, x * (1.0 + 1e-7 * rng.standard_normal(x.shape)), v, dt, 50)
        floor = traj_errors(xp, xr)
        o = table[k]["offset"]
        got = traj_errors(pn[o:o + s.n, :3], xr)
        assert got[0] <= 10.0 * floor[0] + 1e-7, (k, got, floor)
