"""CPU-only checks of the C ABI: the library builds, loads, exports every symbol
include/nbody.h declares, and rejects bad arguments before touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_0706_3060_gb300 import _lib, build
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    return _lib.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "nbody.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nbody_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    from paper_0706_3060_gb300 import _lib
    names = _declared()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(_lib.EXPORTS) == names


def test_version_and_tiles(lib):
    import paper_0706_3060_gb300 as nb
    assert nb.version() >= 10000
    for law in range(9):
        c = nb.tile_count(law)
        assert c >= 4
        for t in range(c):
            info = nb.tile_info(law, t)
            assert info["threads"] % 32 == 0 and 32 % info["j_lanes"] == 0
            assert info["j_tile"] % info["j_lanes"] == 0
            if info["packed"]:   # packed tiles walk source pairs
                assert info["j_tile"] % 2 == 0
            if info["symmetric"]:  # force laws and the gravity VJP; blocks of threads x targets
                assert law in (nb.LAW_GRAV, nb.LAW_LJC, nb.LAW_LJC_LINEAR, nb.TABLE_BATCHED,
                               nb.TABLE_GRAV_FIXED, nb.TABLE_VJP_GRAV, nb.TABLE_VJP_LJC,
                               nb.TABLE_JERK, nb.TABLE_VJP_LJC_LINEAR)
                assert info["packed"]
                assert info["j_tile"] == info["threads"] * info["i_per_thread"]
    with pytest.raises(nb.NBodyError):
        nb.tile_info(0, 99)


def test_tuned_table_roundtrip(lib):
    import paper_0706_3060_gb300 as nb
    # entries a GPU session may have installed from the stored table come back at the end
    keep = [(t, n, nb.get_config(t, n)) for t, n in
            ((nb.LAW_GRAV, 5000), (nb.TABLE_VJP_GRAV, 16384), (nb.TABLE_JERK, 1000))]
    try:
        nb.set_tuned(nb.LAW_GRAV, 5000, 3, 2)
        assert nb.get_config(nb.LAW_GRAV, 5000) == (3, 2)
        nb.set_tuned(nb.LAW_GRAV, 5000, -1, 0)
        assert nb.get_config(nb.LAW_GRAV, 5000)[1] == 0
        # VJP tables: defaults (row 0 from 8192 up, row 1 below), then a tuned entry
        nb.set_tuned(nb.TABLE_VJP_GRAV, 16384, -1, 0)
        nb.set_tuned(nb.TABLE_JERK, 1000, -1, 0)
        assert nb.get_config(nb.TABLE_VJP_GRAV, 16384)[0] == 0
        assert nb.get_config(nb.TABLE_JERK, 1000)[0] == 1
        nb.set_tuned(nb.TABLE_VJP_GRAV, 16384, 2, 4)
        assert nb.get_config(nb.TABLE_VJP_GRAV, 16384) == (2, 4)
    finally:
        for t, n, (tile, js) in keep:
            nb.set_tuned(t, n, tile, js)
    with pytest.raises(nb.NBodyError):
        nb.tile_count(9)


def test_bad_arguments_rejected_without_gpu(lib):
    from paper_0706_3060_gb300._lib import NBodyParams
    p = NBodyParams(0, 0, 1.0, 0.0, -1, 0)
    # NULL params
    assert lib.nbody_forces(None, None, None, None, 8, None, None) == 1
    # negative n
    assert lib.nbody_forces(None, None, None, None, -1, ctypes.byref(p), None) == 1
    # unknown law
    q = NBodyParams(7, 0, 1.0, 0.0, -1, 0)
    assert lib.nbody_forces(ctypes.c_void_p(16), None, ctypes.c_void_p(16), None, 8,
                            ctypes.byref(q), None) == 1
    # misaligned pointer
    assert lib.nbody_forces(ctypes.c_void_p(8), None, ctypes.c_void_p(16), None, 8,
                            ctypes.byref(p), None) == 2
    assert b"aligned" in lib.nbody_last_error()
    # LJC without prm
    q = NBodyParams(1, 0, 1.0, 0.0, -1, 0)
    assert lib.nbody_forces(ctypes.c_void_p(16), None, ctypes.c_void_p(16), None, 8,
                            ctypes.byref(q), None) == 1
    # n == 0 is a no-op even without a device
    assert lib.nbody_forces(None, None, None, None, 0, ctypes.byref(p), None) == 0
    # negative steps
    assert lib.nbody_step(ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16), None, 8,
                          ctypes.c_float(1e-3), -1, 0, None, None, None, ctypes.byref(p),
                          None) == 1


def test_fixed_point_needs_softened_gravity_without_gpu(lib):
    """NBODY_FIXED_POINT for the VJP and acceleration + jerk: its scale needs a
    bound, so eps2 == 0 (and, for the VJP, an LJC law) is refused before any
    device work."""
    from paper_0706_3060_gb300._lib import FIXED_POINT, NBodyParams
    ptr = ctypes.c_void_p(16)
    p = NBodyParams(0, FIXED_POINT, 1.0, 0.0, -1, 0)
    st = lib.nbody_adjoint(ptr, None, ptr, ptr, None, None, 4, ctypes.c_float(1.0), 8,
                           ctypes.byref(p), None)
    assert st == 1 and b"eps2 > 0" in lib.nbody_last_error()
    q = NBodyParams(1, FIXED_POINT, 1.0, 0.01, -1, 0)
    st = lib.nbody_adjoint(ptr, ptr, ptr, ptr, None, None, 4, ctypes.c_float(1.0), 8,
                           ctypes.byref(q), None)
    assert st == 1 and b"gravity" in lib.nbody_last_error()
    st = lib.nbody_forces_jerk(ptr, ptr, ptr, ptr, 8, ctypes.byref(p), None)
    assert st == 1 and b"eps2 > 0" in lib.nbody_last_error()


def test_no_device_is_reported(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_0706_3060_gb300._lib import NBodyParams
    p = NBodyParams(0, 0, 1.0, 0.0, -1, 0)
    st = lib.nbody_forces(ctypes.c_void_p(16), None, ctypes.c_void_p(32), None, 8,
                          ctypes.byref(p), None)
    assert st == 6  # NBODY_EUNSUPPORTED


def test_tune_rejects_bad_arguments_without_gpu(lib):
    t, j, ms = ctypes.c_int32(-7), ctypes.c_int32(-7), ctypes.c_float(0.0)
    args = (ctypes.byref(t), ctypes.byref(j), ctypes.byref(ms), None)
    # the batched table is tuned over a system table, not here
    assert lib.nbody_tune(3, ctypes.c_void_p(16), None, 1024, 1e-4, 3, *args) == 6
    assert lib.nbody_tune(9, ctypes.c_void_p(16), None, 1024, 1e-4, 3, *args) == 6
    assert lib.nbody_tune(8, ctypes.c_void_p(16), None, 1024, 1e-4, 3, *args) == 1  # prm
    assert lib.nbody_tune(0, ctypes.c_void_p(16), None, 0, 1e-4, 3, *args) == 1
    assert lib.nbody_tune(0, ctypes.c_void_p(16), None, 1024, 1e-4, 0, *args) == 1
    assert lib.nbody_tune(0, None, None, 1024, 1e-4, 3, *args) == 1
    assert lib.nbody_tune(1, ctypes.c_void_p(16), None, 1024, 0.0, 3, *args) == 1  # LJC: prm
    assert lib.nbody_tune(4, ctypes.c_void_p(16), None, 1024, 0.0, 3, *args) == 1  # eps2 > 0
    assert t.value == -7 and j.value == -7  # nothing written on error


def test_state_file_round_trip(tmp_path):
    import torch

    from paper_0706_3060_gb300.checkpoint import load_state, save_state
    rng = np.random.default_rng(0)
    pos = torch.from_numpy(rng.standard_normal((7, 4)).astype(np.float32))
    vel = torch.from_numpy(rng.standard_normal((7, 4)).astype(np.float32))
    acc = torch.from_numpy(rng.standard_normal((7, 4)).astype(np.float32))
    lo = torch.from_numpy(rng.standard_normal((14, 4)).astype(np.float32))
    f = tmp_path / "run.npz"
    save_state(f, pos, vel, acc, step=42, params={"dt": 1e-3, "eps": 0.01}, state_lo=lo)
    st = load_state(f, device=torch.device("cpu"))
    assert st["step"] == 42 and st["params"] == {"dt": 1e-3, "eps": 0.01}
    for k, t in (("pos_m", pos), ("vel", vel), ("acc", acc), ("state_lo", lo)):
        assert torch.equal(st[k], t)


def test_workspace_size_rejects_bad_arguments_without_gpu(lib):
    from paper_0706_3060_gb300._lib import NBodyParams
    p = NBodyParams(0, 0, 1.0, 1e-4, -1, 0)
    b = ctypes.c_size_t(7)
    assert lib.nbody_workspace_size(ctypes.byref(p), 100, 0, None) == 1
    assert lib.nbody_workspace_size(None, 100, 0, ctypes.byref(b)) == 1
    assert lib.nbody_workspace_size(ctypes.byref(p), -1, 0, ctypes.byref(b)) == 1
    assert lib.nbody_workspace_size(ctypes.byref(p), 100, -1, ctypes.byref(b)) == 1
    assert lib.nbody_workspace_size(ctypes.byref(p), 0, 0, ctypes.byref(b)) == 0 and b.value == 0
