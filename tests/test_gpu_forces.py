"""GPU parity: nbody_forces (gravity, Eq. 1; LJC, Table 1) against the FP64 oracle.

Tolerance: relative per-particle L2 error, RMS <= 1e-5 and max <= 1e-4, at
sizes spanning several tiles with ragged tails, every compiled tile shape, the
edge cases (N = 1, 2, 3, eps = 0 with the self-pair mask) and, at the
benchmark's N = 262144, a seeded sample of targets checked one by one.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads
from gpu_util import (assert_forces_close, dev, grav_tensors, lib, ljc_tensors,
                      oracle_ljc_system, rel_errors)

pytestmark = pytest.mark.gpu


def _grav_ref(g, idx=None, potential=False):
    x, _, m = g.f32_as_f64()
    return oracle.grav_accel(x, m, G=g.G, eps=float(np.float32(g.eps)), idx=idx,
                             potential=potential)


@pytest.mark.parametrize("n", [1, 2, 3, 31, 33, 127, 1000, 1024, 4099, 8192])
def test_grav_default_config(n):
    nb = lib()
    g = workloads.plummer(n, seed=100 + n, eps=0.01)
    pos, _ = grav_tensors(g)
    acc = nb.forces(pos, eps=float(np.float32(g.eps)))
    torch.cuda.synchronize()
    ref = _grav_ref(g)
    if n == 1:
        assert torch.all(acc[:, :3] == 0)
        return
    assert_forces_close(acc[:, :3].cpu().numpy(), ref, what=f"n={n}")


@pytest.mark.parametrize("tile", range(27))
@pytest.mark.parametrize("jsplit", [1, 3])
def test_grav_every_tile(tile, jsplit):
    nb = lib()
    n = 3001
    g = workloads.plummer(n, seed=7, eps=0.02)
    pos, _ = grav_tensors(g)
    acc = nb.forces(pos, eps=float(np.float32(g.eps)), tile=tile, jsplit=jsplit, pot=True)
    ref, phi = _grav_ref(g, potential=True)
    a = acc.cpu().numpy()
    assert_forces_close(a[:, :3], ref, what=f"tile={tile} jsplit={jsplit}")
    e = np.abs(a[:, 3] - phi) / np.abs(phi)
    assert np.sqrt(np.mean(e * e)) <= 1e-5 and e.max() <= 1e-4


def test_grav_unsoftened_two_and_three_body():
    nb = lib()
    # eps = 0: the self pair would be 0/0 without the index mask.
    x = np.array([[0.0, 0.0, 0.0, 5.0], [3.0, 4.0, 0.0, 2.0], [-1.0, 0.5, 2.0, 1.0]],
                 dtype=np.float32)
    for n in (2, 3):
        pos = torch.from_numpy(x[:n]).to(dev()).contiguous()
        acc = nb.forces(pos, G=1.5, eps=0.0, pot=True).cpu().numpy()
        ref, phi = oracle.grav_accel(x[:n, :3].astype(np.float64), x[:n, 3].astype(np.float64),
                                     G=1.5, eps=0.0, potential=True)
        assert np.all(np.isfinite(acc))
        np.testing.assert_allclose(acc[:, :3], ref, rtol=2e-6, atol=1e-7)
        np.testing.assert_allclose(acc[:, 3], phi, rtol=2e-6)


def test_grav_precise_and_uncompensated_modes():
    nb = lib()
    g = workloads.plummer(5000, seed=3, eps=0.01)
    pos, _ = grav_tensors(g)
    ref = _grav_ref(g)
    eps = float(np.float32(g.eps))
    for kw in ({"precise": True}, {"compensated": False}, {"precise": True, "compensated": False}):
        acc = nb.forces(pos, eps=eps, **kw).cpu().numpy()
        assert_forces_close(acc[:, :3], ref, what=str(kw))


def test_grav_acc_lo_is_residual():
    nb = lib()
    g = workloads.plummer(2048, seed=4, eps=0.01)
    pos, _ = grav_tensors(g)
    acc, lo = nb.forces(pos, eps=float(np.float32(g.eps)), want_lo=True)
    ref = _grav_ref(g)
    hi = acc[:, :3].double().cpu().numpy()
    both = hi + lo[:, :3].double().cpu().numpy()
    e_hi = rel_errors(hi, ref)
    e_both = rel_errors(both, ref)
    assert np.mean(e_both) <= np.mean(e_hi) * 1.01
    assert np.all(np.abs(lo[:, :3].cpu().numpy()) <= np.abs(acc[:, :3].cpu().numpy()) * 1e-6 + 1e-30)


def test_grav_deterministic_and_host_path():
    nb = lib()
    g = workloads.plummer(20000, seed=5, eps=0.01)
    pos, _ = grav_tensors(g)
    eps = float(np.float32(g.eps))
    a1 = nb.forces(pos, eps=eps)
    a2 = nb.forces(pos, eps=eps)
    assert torch.equal(a1, a2)
    a3 = nb.forces(pos.cpu(), eps=eps)   # host pointers: staged through the device
    assert torch.equal(a1.cpu(), a3)


def test_grav_full_size_sampled():
    """N = 262144 Plummer (eps = 0.04 N^-1/3) in the benchmark's launch configuration;
    4096 seeded targets checked against the oracle one by one."""
    nb = lib()
    n = 262144
    g = workloads.plummer(n, seed=1, eps=workloads.plummer_softening(n))
    pos, _ = grav_tensors(g)
    acc = nb.forces(pos, eps=float(np.float32(g.eps))).cpu().numpy()
    idx = np.sort(np.random.default_rng(0).choice(n, 4096, replace=False))
    ref = _grav_ref(g, idx=idx)
    assert_forces_close(acc[idx, :3], ref, what="N=262144 sample")


def test_full_size_secondary_forms_sampled():
    """The bench's other forms at N = 262144 in their launch configurations, on
    sampled targets against the oracle one by one: acceleration + jerk, the
    1024-target subset, fixed-point and Newton-refined sums."""
    nb = lib()
    n = 262144
    g = workloads.plummer(n, seed=1, eps=workloads.plummer_softening(n))
    eps = float(np.float32(g.eps))
    pos, vel = grav_tensors(g)
    x, v, m = g.f32_as_f64()
    idx = np.sort(np.random.default_rng(3).choice(n, 512, replace=False))
    acc, jerk = nb.forces_jerk(pos, vel, eps=eps)
    ra, rj = oracle.grav_jerk(x, v, m, eps=eps, idx=idx)
    assert_forces_close(acc[idx, :3].cpu().numpy(), ra, what="jerk path acc")
    assert_forces_close(jerk[idx, :3].cpu().numpy(), rj, what="jerk")
    ref = _grav_ref(g, idx=idx)
    for kw in ({"fixed": True}, {"precise": True}, {"compensated": False}):
        a = nb.forces(pos, eps=eps, **kw).cpu().numpy()
        assert_forces_close(a[idx, :3], ref, what=str(kw))
    sub = np.random.default_rng(1).choice(n, 1024, replace=False).astype(np.int32)
    a = nb.forces_subset(pos, torch.from_numpy(sub).to(dev()), eps=eps).cpu().numpy()
    assert_forces_close(a[:, :3], _grav_ref(g, idx=sub.astype(np.int64)), what="subset")


@pytest.mark.slow
def test_grav_million_sampled():
    nb = lib()
    n = 1048576
    g = workloads.plummer(n, seed=1, eps=workloads.plummer_softening(n))
    pos, _ = grav_tensors(g)
    acc = nb.forces(pos, eps=float(np.float32(g.eps))).cpu().numpy()
    idx = np.sort(np.random.default_rng(1).choice(n, 1024, replace=False))
    ref = _grav_ref(g, idx=idx)
    assert_forces_close(acc[idx, :3], ref, what="N=1048576 sample")


@pytest.mark.parametrize("n", [2, 33, 517, 2048, 8192])
def test_ljc_forces(n):
    nb = lib()
    s = workloads.ljc_sphere(n, seed=2 if n == 8192 else 40 + n)
    pos, _, prm = ljc_tensors(s)
    acc = nb.forces(pos, prm, pot=True).cpu().numpy()
    sysm, x, _ = oracle_ljc_system(s)
    ref, phi = sysm.accel(x, potential=True)
    assert_forces_close(acc[:, :3], ref, what=f"LJC n={n}")
    e = np.abs(acc[:, 3] - phi) / np.maximum(np.abs(phi), 1e-3 * np.abs(phi).max())
    assert np.sqrt(np.mean(e * e)) <= 1e-5 and e.max() <= 1e-4


LJC_TILES = 21  # rows of the LJC force table (checked below against the library)


LJCLIN_TILES = 11  # rows of the LJC(linear) force table


def test_ljc_tile_count():
    assert lib().tile_count(lib().LAW_LJC) == LJC_TILES
    assert lib().tile_count(lib().LAW_LJC_LINEAR) == LJCLIN_TILES


@pytest.mark.parametrize("tile", range(LJC_TILES))
def test_ljc_every_tile(tile):
    nb = lib()
    s = workloads.ljc_sphere(1500, seed=9)
    pos, _, prm = ljc_tensors(s)
    acc = nb.forces(pos, prm, tile=tile, jsplit=2).cpu().numpy()
    sysm, x, _ = oracle_ljc_system(s)
    assert_forces_close(acc[:, :3], sysm.accel(x), what=f"LJC tile={tile}")


def test_ljc_pair_minimum():
    """Two atoms at r = 2^(1/6) sigma with no charge feel no force (closed form)."""
    nb = lib()
    sig, eps = 3.0, 0.1
    r = 2.0 ** (1.0 / 6.0) * sig
    pos = torch.tensor([[0, 0, 0, 12.0], [r, 0, 0, 12.0]], dtype=torch.float32, device=dev())
    prm = nb.pack_ljc(torch.zeros(2, dtype=torch.float64, device=dev()),
                      torch.full((2,), sig, dtype=torch.float64, device=dev()),
                      torch.full((2,), eps, dtype=torch.float64, device=dev()),
                      torch.zeros(2, dtype=torch.int32, device=dev()))
    acc = nb.forces(pos, prm, pot=True).cpu().numpy()
    assert np.all(np.abs(acc[:, :3]) < 1e-5 * 24 * eps / sig / 12.0)
    np.testing.assert_allclose(acc[:, 3], [-eps, -eps], rtol=1e-5)


def test_invalid_arguments_are_rejected():
    nb = lib()
    pos = torch.zeros((8, 4), device=dev())
    with pytest.raises(nb.NBodyError) as ei:
        nb.forces(pos, law=nb.LAW_LJC)            # LJC without prm
    assert ei.value.status == 1
    bad = torch.zeros(8 * 4 + 1, device=dev())[1:].view(8, 4)   # 4-byte offset
    with pytest.raises(nb.NBodyError) as ei:
        nb.forces(bad)
    assert ei.value.status == 2
    with pytest.raises(nb.NBodyError):
        nb.forces(pos, tile=99)
    acc = nb.forces(torch.zeros((0, 4), device=dev()))   # n == 0 is a no-op
    assert acc.shape == (0, 4)


@pytest.mark.parametrize("n,na", [(1000, 1), (4099, 37), (20000, 900), (262144, 1000)])
def test_grav_subset_matches_oracle(n, na):
    """Block time steps (Sec. 3.4): forces on an active subset against all particles."""
    nb = lib()
    g = workloads.plummer(n, seed=200 + na, eps=0.01 if n < 100000 else
                          workloads.plummer_softening(n))
    pos, _ = grav_tensors(g)
    idx = np.random.default_rng(na).choice(n, na, replace=False).astype(np.int32)
    acc = nb.forces_subset(pos, torch.from_numpy(idx).to(dev()), eps=float(np.float32(g.eps)),
                           pot=True).cpu().numpy()
    ref, phi = _grav_ref(g, idx=idx, potential=True)
    assert_forces_close(acc[:, :3], ref, what=f"subset n={n} na={na}")
    e = np.abs(acc[:, 3] - phi) / np.abs(phi)
    assert e.max() <= 1e-4


def test_subset_equals_full_rows_and_unsoftened():
    nb = lib()
    g = workloads.plummer(3001, seed=8, eps=0.01)
    pos, _ = grav_tensors(g)
    full = nb.forces(pos, eps=0.0)
    idx = torch.tensor([3000, 0, 17, 17, 1500], dtype=torch.int32, device=dev())
    sub = nb.forces_subset(pos, idx, eps=0.0)   # eps = 0: the self mask is essential
    assert torch.all(torch.isfinite(sub))
    e = rel_errors(sub[:, :3].cpu().numpy(), full[idx.long()][:, :3].cpu().numpy())
    assert e.max() <= 2e-6


def test_ljc_subset():
    nb = lib()
    s = workloads.ljc_sphere(3000, seed=44)
    pos, _, prm = ljc_tensors(s)
    idx = np.arange(5, 3000, 7).astype(np.int32)
    acc = nb.forces_subset(pos, torch.from_numpy(idx).to(dev()), prm).cpu().numpy()
    sysm, x, _ = oracle_ljc_system(s)
    assert_forces_close(acc[:, :3], sysm.accel(x)[idx], what="LJC subset")


@pytest.mark.parametrize("n", [2, 33, 1000, 9001])
def test_grav_acceleration_and_jerk(n):
    """Table 1 "Gravity (accel & jerk)" against the FP64 oracle."""
    nb = lib()
    g = workloads.plummer(n, seed=300 + n, eps=0.01)
    pos, vel = grav_tensors(g)
    acc, jerk = nb.forces_jerk(pos, vel, eps=float(np.float32(g.eps)))
    x, v, m = g.f32_as_f64()
    ra, rj = oracle.grav_jerk(x, v, m, eps=float(np.float32(g.eps)))
    assert_forces_close(acc[:, :3].cpu().numpy(), ra, what=f"GAJ acc n={n}")
    assert_forces_close(jerk[:, :3].cpu().numpy(), rj, what=f"GAJ jerk n={n}")


@pytest.mark.parametrize("tile", range(12))
def test_jerk_every_tile(tile):
    """Every acceleration + jerk tile (scalar and packed f32x2) at an odd size
    spanning several j-tiles (the packed source buffer ends in a pad particle)."""
    nb = lib()
    n = 1300
    g = workloads.plummer(n, seed=301, eps=0.01)
    pos, vel = grav_tensors(g)
    acc, jerk = nb.forces_jerk(pos, vel, eps=float(np.float32(g.eps)), tile=tile)
    x, v, m = g.f32_as_f64()
    ra, rj = oracle.grav_jerk(x, v, m, eps=float(np.float32(g.eps)))
    assert_forces_close(acc[:, :3].cpu().numpy(), ra, what=f"GAJ acc tile {tile}")
    assert_forces_close(jerk[:, :3].cpu().numpy(), rj, what=f"GAJ jerk tile {tile}")


def test_jerk_unsoftened_pair():
    nb = lib()
    pos = torch.tensor([[0, 0, 0, 5.0], [3, 4, 0, 2.0]], dtype=torch.float32, device=dev())
    vel = torch.tensor([[0, 0, 0, 0], [1, 0, 0, 0]], dtype=torch.float32, device=dev())
    acc, jerk = nb.forces_jerk(pos, vel, eps=0.0)
    np.testing.assert_allclose(jerk[0, :3].cpu().numpy(), [-0.00128, -0.02304, 0.0], rtol=2e-6,
                               atol=1e-9)


def _ljclin_tensors(s, D=4.0):
    nb = lib()
    x, v, m, q, st, et = s.f32()
    d = dev()
    pos = torch.from_numpy(np.concatenate([x, m[:, None]], 1).astype(np.float32)).to(d)
    prm = nb.pack_ljc(torch.from_numpy(q.astype(np.float64)).to(d),
                      torch.from_numpy(st.astype(np.float64)[s.types]).to(d),
                      torch.from_numpy(et.astype(np.float64)[s.types]).to(d),
                      torch.from_numpy(s.types).to(d), kq=332.0637 / D)
    sysm = oracle.LJCSystem(m.astype(np.float64), q.astype(np.float64), s.types,
                            st.astype(np.float64), et.astype(np.float64), 332.0637 / D,
                            linear=True)
    return pos.contiguous(), prm, sysm, x.astype(np.float64)


@pytest.mark.parametrize("tile", range(LJCLIN_TILES))
@pytest.mark.parametrize("n", [257, 3000, 8192])
def test_ljc_linear_dielectric(tile, n):
    """Table 1 LJC(linear): dielectric D r with D = 4 (reading C3)."""
    nb = lib()
    s = workloads.ljc_sphere(n, seed=500 + n)
    pos, prm, sysm, x = _ljclin_tensors(s)
    acc = nb.forces(pos, prm, law=nb.LAW_LJC_LINEAR, pot=True, tile=tile, jsplit=2).cpu().numpy()
    ref, phi = sysm.accel(x, potential=True)
    assert_forces_close(acc[:, :3], ref, what=f"LJC(linear) tile={tile} n={n}")
    e = np.abs(acc[:, 3] - phi) / np.maximum(np.abs(phi), 1e-3 * np.abs(phi).max())
    assert np.sqrt(np.mean(e * e)) <= 1e-5 and e.max() <= 1e-4


def test_ljc_linear_steps_and_subset():
    nb = lib()
    s = workloads.ljc_sphere(1500, seed=77)
    pos, prm, sysm, x = _ljclin_tensors(s)
    idx = np.arange(0, 1500, 11).astype(np.int32)
    sub = nb.forces_subset(pos, torch.from_numpy(idx).to(dev()), prm, law=nb.LAW_LJC_LINEAR)
    assert_forces_close(sub[:, :3].cpu().numpy(), sysm.accel(x)[idx], what="LJC(linear) subset")
    vel = torch.zeros_like(pos)
    acc = torch.empty_like(pos)
    nb.step(pos, vel, acc, prm, law=nb.LAW_LJC_LINEAR, dt=1e-4, nsteps=4)
    xs, _ = oracle.leapfrog(sysm, x, np.zeros_like(x), 1e-4, 4)
    err = np.linalg.norm(pos[:, :3].cpu().numpy() - xs, axis=1) / np.sqrt(np.mean(np.sum(xs**2, 1)))
    assert np.sqrt(np.mean(err ** 2)) <= 1e-6


def test_fixed_point_accuracy_and_split_independence():
    """64-bit fixed-point accumulation (Sec. 3.2, GRAPE-6): oracle accuracy, and the
    same bits for every j-split because integer sums are associative."""
    nb = lib()
    g = workloads.plummer(20001, seed=91, eps=0.01)
    pos, _ = grav_tensors(g)
    eps = float(np.float32(g.eps))
    ref, phi = _grav_ref(g, potential=True)
    outs = []
    for js in (1, 2, 3, 5, 8):
        a = nb.forces(pos, eps=eps, fixed=True, tile=0, jsplit=js, pot=True)
        outs.append(a)
        assert_forces_close(a[:, :3].cpu().numpy(), ref, what=f"fixed jsplit={js}")
    for a in outs[1:]:
        assert torch.equal(a, outs[0])
    e = np.abs(outs[0][:, 3].cpu().numpy() - phi) / np.abs(phi)
    assert e.max() <= 1e-4
    for tile in range(nb.tile_count(nb.TABLE_GRAV_FIXED)):
        a = nb.forces(pos, eps=eps, fixed=True, tile=tile)
        assert_forces_close(a[:, :3].cpu().numpy(), ref, what=f"fixed tile={tile}")


def test_fixed_point_steps_split_independent_and_rejections():
    nb = lib()
    g = workloads.plummer(4097, seed=92, eps=0.01)
    eps = float(np.float32(g.eps))
    runs = []
    for js in (1, 4):
        pos, vel = grav_tensors(g)
        acc = torch.empty_like(pos)
        nb.step(pos, vel, acc, dt=1e-3, nsteps=5, eps=eps, fixed=True, tile=0, jsplit=js)
        runs.append((pos, vel))
    assert torch.equal(runs[0][0], runs[1][0]) and torch.equal(runs[0][1], runs[1][1])
    pos, _ = grav_tensors(g)
    with pytest.raises(nb.NBodyError):
        nb.forces(pos, eps=0.0, fixed=True)     # no bound without softening
    s = workloads.ljc_sphere(64, seed=1)
    lpos, _, prm = ljc_tensors(s)
    with pytest.raises(nb.NBodyError):
        nb.forces(lpos, prm, fixed=True)


def test_force_call_captures_into_cuda_graph():
    """A warmed-up nbody_forces call can be captured in a CUDA graph and replayed
    (launch-bound small systems), giving the same bits as the direct call."""
    nb = lib()
    g = workloads.plummer(4096, seed=3, eps=0.01)
    pos, _ = grav_tensors(g)
    eps = float(np.float32(g.eps))
    acc = torch.empty_like(pos)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        nb.forces(pos, eps=eps, out=acc)      # sizes the workspace outside capture
    s.synchronize()
    ref = acc.clone()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        nb.forces(pos, eps=eps, out=acc)
    acc.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(acc, ref)


def test_edge_cases_coincident_massless_and_far():
    """Coincident distinct particles with eps > 0 stay finite (d = 0 gives no force);
    massless tracers feel the others but pull on nobody; coordinates far from the
    origin (1e4) keep the relative accuracy of the differences."""
    nb = lib()
    g = workloads.plummer(1000, seed=55, eps=0.05)
    x, v, m = g.f32()
    x = x.copy()
    m = m.copy()
    x[1] = x[0]                      # two distinct particles at one point
    m[10:20] = 0.0                   # massless tracers
    pos = torch.from_numpy(np.concatenate([x, m[:, None]], 1)).to(dev()).contiguous()
    acc = nb.forces(pos, eps=0.05, pot=True).cpu().numpy()
    assert np.all(np.isfinite(acc))
    ref, phi = oracle.grav_accel(x.astype(np.float64), m.astype(np.float64), eps=0.05,
                                 potential=True)
    assert_forces_close(acc[:, :3], ref, what="coincident + massless")
    # tracers do not act on anybody: removing them changes no other acceleration
    keep = np.r_[0:10, 20:1000]
    pos2 = pos[torch.from_numpy(keep).to(dev())].contiguous()
    acc2 = nb.forces(pos2, eps=0.05).cpu().numpy()
    e = rel_errors(acc2[:, :3], acc[keep, :3])
    assert e.max() <= 1e-5
    # shift far from the origin: positions of size 1e4 (FP32 ulp ~1e-3)
    xf = (x.astype(np.float64) + 1e4).astype(np.float32)
    posf = torch.from_numpy(np.concatenate([xf, m[:, None]], 1)).to(dev()).contiguous()
    accf = nb.forces(posf, eps=0.05).cpu().numpy()
    reff = oracle.grav_accel(xf.astype(np.float64), m.astype(np.float64), eps=0.05)
    assert_forces_close(accf[:, :3], reff, what="far from origin")


def test_workspace_size_covers_the_partials():
    """nbody_workspace_size: at least the two partial-sum arrays of the chosen
    j-split plus the packed source copy, and growing with the j-split."""
    nb = lib()
    n = 4096
    tile = 13  # packed, 256 targets per item, j-tile 512
    w2 = nb.workspace_size(n, eps=0.01, tile=tile, jsplit=2)
    w8 = nb.workspace_size(n, eps=0.01, tile=tile, jsplit=8)
    assert w2 >= 2 * 2 * n * 16 + (n // 2) * 32
    assert w8 - w2 == 2 * 6 * n * 16
    assert nb.workspace_size(n, eps=0.01, report_rows=10) > nb.workspace_size(n, eps=0.01)


@pytest.mark.slow
def test_subset_largest_size():
    """N = 2^24 Plummer particles (16.8 M sources, 268 MB of positions): forces on 512
    sampled targets through the subset path, against the oracle one by one."""
    nb = lib()
    n = 1 << 24
    g = workloads.plummer(n, seed=9, eps=workloads.plummer_softening(n))
    pos, _ = grav_tensors(g)
    idx = np.sort(np.random.default_rng(2).choice(n, 512, replace=False)).astype(np.int32)
    eps = float(np.float32(g.eps))
    a = nb.forces_subset(pos, torch.from_numpy(idx).to(dev()), eps=eps).cpu().numpy()
    assert_forces_close(a[:, :3], _grav_ref(g, idx=idx.astype(np.int64)), what="N=2^24 subset")
