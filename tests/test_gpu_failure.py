"""Failure detection on the GPU without a fault: a kernel's bounded mbarrier wait
runs out (nothing ever completes the barrier), the kernel returns, the host
reads NBODY_ETIMEOUT from nbody_check, and the context keeps working."""
import ctypes

import numpy as np
import pytest
import torch

import workloads
from gpu_util import grav_tensors, lib

pytestmark = pytest.mark.gpu


def test_expired_wait_is_reported_and_context_survives():
    nb = lib()
    from paper_0706_3060_gb300 import _lib
    L = _lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.nbody_check(stream) == 0
    assert L.nbody_selftest_timeout(2_000_000, stream) == 0   # ~1 ms at 2 GHz
    assert L.nbody_check(stream) == 5                          # NBODY_ETIMEOUT
    assert b"bounded device wait" in L.nbody_last_error()
    assert L.nbody_check(stream) == 0                          # reported once, then cleared
    # the context is intact: a force evaluation still runs and checks clean
    g = workloads.plummer(2048, seed=1, eps=0.01)
    pos, _ = grav_tensors(g)
    acc = nb.forces(pos, eps=float(np.float32(g.eps)))
    assert torch.all(torch.isfinite(acc))
    assert L.nbody_check(stream) == 0
    assert L.nbody_selftest_timeout(0, stream) == 1            # bad limit rejected
