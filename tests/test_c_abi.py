"""The C ABI from a plain C program (tests/c_abi/host_only.c): compiled with gcc against
include/delimit.h, linked to the built library and run without a GPU (host-only
handles, table queries, error codes)."""
import os
import shutil
import subprocess

import pytest

from paper_1808_01517_gb300 import _lib as L

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_c_program_uses_the_abi(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    L.get()  # builds the library if needed
    from paper_1808_01517_gb300 import build
    lib = build.LIB
    exe = str(tmp_path / "host_only")
    subprocess.run([gcc, "-std=c99", "-O1", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(HERE, "c_abi", "host_only.c"), "-o", exe, lib, "-lm",
                    "-Wl,-rpath," + os.path.dirname(lib)], check=True)
    env = dict(os.environ)
    cuda_lib = "/usr/local/cuda/lib64"
    env["LD_LIBRARY_PATH"] = ":".join(p for p in (cuda_lib, env.get("LD_LIBRARY_PATH", "")) if p)
    r = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "c abi ok" in r.stdout
