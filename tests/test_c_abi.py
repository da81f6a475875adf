"""The C ABI from plain C: tests/c/abi_check.c includes only
include/hpgmxp.h and links libhpgmxp.so (gcc, no Python, no CUDA headers).
On the CPU it is compiled and its argument-validation checks run; on a GPU
it solves a 16^3 system with host buffers."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2507_11512_gb300")


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    import __graft_entry__
    __graft_entry__.build()
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    out = str(tmp_path_factory.mktemp("cabi") / "abi_check")
    cmd = [cc, "-std=c99", "-O1", "-Wall", "-Werror", os.path.join(ROOT, "tests", "c", "abi_check.c"),
           "-I" + os.path.join(ROOT, "include"), "-L" + PKG, "-lhpgmxp",
           "-Wl,-rpath," + PKG, "-o", out]
    p = subprocess.run(cmd, capture_output=True, text=True)
    assert p.returncode == 0, p.stderr
    return out


def test_c_caller_host_checks(exe):
    p = subprocess.run([exe, "host"], capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stdout + p.stderr
    assert "host checks ok" in p.stdout


@pytest.mark.gpu
def test_c_caller_solves_with_host_buffers(exe):
    p = subprocess.run([exe, "solve"], capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stdout + p.stderr
    assert "converged 1" in p.stdout
