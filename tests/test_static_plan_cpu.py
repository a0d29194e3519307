"""Host-only check (no GPU) that nbody_forces_static never plans past its static
scratch: compiles tests/static_plan_host.cpp against the built library and runs
it over laws, sizes (including 131072 .. 524288, where the tuned symmetric tile
falls back to a one-sided tile whose automatic j-split would not fit), tiles,
j-splits and SM counts."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_static_plan_stays_inside_scratch(tmp_path):
    from paper_0706_3060_gb300 import _lib, build
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    pkg = os.path.dirname(_lib.LIB_PATH)
    exe = str(tmp_path / "static_plan_host")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(pkg, "csrc"),
                    os.path.join(ROOT, "tests", "static_plan_host.cpp"), "-o", exe,
                    "-L", pkg, "-lnbody", "-Wl,-rpath," + pkg], check=True)
    res = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stdout[-4000:] + res.stderr[-2000:]
    assert "failures 0" in res.stdout
    acc = int(res.stdout.split("accepted")[1].split()[0])
    assert acc > 1000
