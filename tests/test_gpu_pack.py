"""Packing (caller FP64 SoA -> the float4 streams the kernels read; Sec. 2 keeps
the coordinates as GPU streams and the Appendix listing reads (position, mass)
as one float4): bitwise against NumPy's round-to-nearest FP64 -> FP32
conversion, and used end to end in a force evaluation against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from gpu_util import assert_forces_close, dev, lib

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [1, 2, 255, 256, 257, 100003])
def test_pack_grav_is_fp32_rounding(n):
    nb = lib()
    rng = np.random.default_rng(n)
    # values spread over many binades, with halfway-looking tails
    x = rng.standard_normal((n, 3)) * 10.0 ** rng.uniform(-6, 6, (n, 1))
    m = rng.uniform(0.0, 1.0, n) * 10.0 ** rng.uniform(-8, 2, n)
    got = nb.pack_grav(torch.from_numpy(x).to(dev()), torch.from_numpy(m).to(dev()))
    torch.cuda.synchronize()
    want = np.concatenate([x, m[:, None]], axis=1).astype(np.float32)
    assert np.array_equal(got.cpu().numpy().view(np.uint32), want.view(np.uint32))


def test_pack_grav_end_to_end_forces():
    """The small gravity workload packed on the GPU from its FP64 draw, then one
    force evaluation against the oracle on the same FP32-rounded inputs."""
    nb = lib()
    g = workloads.plummer(1024, seed=0, eps=0.01)
    pos = nb.pack_grav(torch.from_numpy(g.x).to(dev()), torch.from_numpy(g.m).to(dev()))
    x32, _, m32 = g.f32()
    assert np.array_equal(pos.cpu().numpy(), np.concatenate([x32, m32[:, None]], 1))
    eps = float(np.float32(g.eps))
    acc = nb.forces(pos, eps=eps)
    x, _, m = g.f32_as_f64()
    assert_forces_close(acc[:, :3].double().cpu().numpy(), oracle.grav_accel(x, m, eps=eps),
                        what="packed input")


def test_pack_ljc_matches_its_definition():
    """prm = (q sqrt(kq), sigma / 2, sqrt(24 eps), type), each computed in FP64 and
    rounded once (IEEE square root on both sides), bit for bit."""
    nb = lib()
    s = workloads.ljc_sphere(3001, seed=9)
    _, _, _, q, st, et = s.f32()
    qd, sd, ed = q.astype(np.float64), st.astype(np.float64)[s.types], et.astype(np.float64)[s.types]
    kq = 332.0637 / 80.0
    prm = nb.pack_ljc(torch.from_numpy(qd).to(dev()), torch.from_numpy(sd).to(dev()),
                      torch.from_numpy(ed).to(dev()), torch.from_numpy(s.types).to(dev()), kq=kq)
    want = np.stack([qd * np.sqrt(kq), 0.5 * sd, np.sqrt(24.0 * ed),
                     s.types.astype(np.float64)], axis=1).astype(np.float32)
    assert np.array_equal(prm.cpu().numpy().view(np.uint32), want.view(np.uint32))
