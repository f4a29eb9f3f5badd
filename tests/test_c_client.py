"""The C ABI from a plain C program (tests/c_client.c), without Python in the loop:
FPS, grid and filtration of a regular tetrahedron against its closed forms."""
import os
import shutil
import subprocess
import tempfile

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_client_regular_tetrahedron():
    from paper_2509_22432_b300 import _lib
    lib = _lib.get()._name
    cc = shutil.which("gcc") or shutil.which("cc")
    cuda = "/usr/local/cuda"
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "c_client")
        r = subprocess.run([cc, "-std=c99", "-O2", os.path.join(ROOT, "tests", "c_client.c"), "-I",
                            os.path.join(ROOT, "include"), "-I", f"{cuda}/include", lib, f"-L{cuda}/lib64",
                            "-lcudart", "-lm", f"-Wl,-rpath,{os.path.dirname(lib)}", f"-Wl,-rpath,{cuda}/lib64",
                            "-o", exe], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
        assert r.returncode == 0, r.stdout + r.stderr
        assert "ok" in r.stdout
