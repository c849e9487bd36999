"""The C ABI from a plain C99 program (no Python, no device): the header compiles as C99 and as
C++17, the library links by name, and the host-only calls behave as the header states."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1508_07621_gb300")
LIB = os.path.join(PKG, "libfloquet.so")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        import __graft_entry__
        __graft_entry__.build()
    return LIB


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_plain_c_client(lib, tmp_path):
    exe = tmp_path / "abi_host_smoke"
    src = os.path.join(ROOT, "tests", "c", "abi_host_smoke.c")
    r = subprocess.run(["gcc", "-std=c99", "-D_DEFAULT_SOURCE", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        src, "-o", str(exe), "-L", PKG, "-lfloquet", "-lm", f"-Wl,-rpath,{PKG}"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_header_compiles_as_cpp(tmp_path):
    src = tmp_path / "inc.cpp"
    src.write_text('#include "floquet.h"\nint main() { fq_problem p{}; return p.n; }\n')
    r = subprocess.run(["g++", "-std=c++17", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-c", str(src),
                        "-o", str(tmp_path / "inc.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
