"""The library's own autotuner (nbody_tune): for each tile table it searches
the compiled tiles x j-splits on the caller's inputs, installs the winner for
the size bucket, and the winner then reproduces the oracle."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from gpu_util import assert_forces_close, grav_tensors, lib, ljc_tensors, oracle_ljc_system

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("table", [0, 4, 5, 7])
def test_tune_gravity_tables(table):
    nb = lib()
    n = 3000
    g = workloads.plummer(n, seed=90, eps=0.01)
    pos, vel = grav_tensors(g)
    eps = float(np.float32(g.eps))
    before = nb.get_config(table, n)
    got = nb.tune_table(table, pos, eps=eps, reps=2)
    try:
        assert 0 <= got["tile"] < nb.tile_count(table) and got["ms"] > 0.0
        assert nb.get_config(table, n) == (got["tile"], got["jsplit"])
        x, v, m = g.f32_as_f64()
        if table in (0, 4):
            acc = nb.forces(pos, eps=eps, fixed=table == 4)
            assert_forces_close(acc[:, :3].cpu().numpy(), oracle.grav_accel(x, m, eps=eps))
        elif table == 7:
            acc, jerk = nb.forces_jerk(pos, vel, eps=eps)
            ra, rj = oracle.grav_jerk(x, v, m, eps=eps)
            assert_forces_close(jerk[:, :3].cpu().numpy(), rj)
        else:
            lam = torch.from_numpy(v.astype(np.float32))
            lam = torch.cat([lam, torch.zeros(n, 1)], 1).to(pos.device).contiguous()
            gx, gm, _ = nb.adjoint(pos, lam, eps=eps)
            rg, rm = oracle.grav_vjp(x, m, v, eps=eps)
            err = np.linalg.norm(gx[:, :3].cpu().numpy() - rg) / np.linalg.norm(rg)
            assert err <= 2e-5
    finally:
        nb.set_tuned(table, n, *before)


def test_tune_ljc_table():
    nb = lib()
    s = workloads.ljc_sphere(1500, seed=91)
    pos, _, prm = ljc_tensors(s)
    before = nb.get_config(nb.LAW_LJC, 1500)
    got = nb.tune_table(nb.LAW_LJC, pos, prm, reps=2)
    try:
        acc = nb.forces(pos, prm)
        sysm, x, _ = oracle_ljc_system(s)
        assert_forces_close(acc[:, :3].cpu().numpy(), sysm.accel(x), what=f"tuned {got}")
    finally:
        nb.set_tuned(nb.LAW_LJC, 1500, *before)
