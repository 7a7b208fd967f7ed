"""The C ABI from a plain C program (tests/c_abi/host_only.c): compiled with gcc against
include/delimit.h, linked to the built library and run without a GPU (host-only
handles, table queries, error codes); and the host FP64 table code under the address and
undefined-behaviour sanitizers."""
import os
import shutil
import subprocess
import sys

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


def test_host_tables_under_address_and_undefined_sanitizers(tmp_path):
    """csrc/host_tables.cpp (the FP64 basis, pseudo-inverse, kernel geometry, collapse and
    neighbour tables) built with -fsanitize=address,undefined beside a driver
    (tests/c_abi/host_tables_sanitized.cpp) that runs every table builder over orders
    0-8, both lambdas, every window, both LSC forms and the refused inputs."""
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    flags = ["-std=c++17", "-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
             "-fno-omit-frame-pointer"]
    probe = tmp_path / "probe.cpp"
    probe.write_text("int main() { return 0; }\n")
    if subprocess.run([gxx, *flags, str(probe), "-o", str(tmp_path / "probe")], capture_output=True).returncode:
        pytest.skip("sanitizer runtimes not available")
    exe = str(tmp_path / "host_tables_sanitized")
    csrc = os.path.join(ROOT, "paper_1808_01517_gb300", "csrc")
    subprocess.run([gxx, *flags, "-Wall", "-Werror", "-I", csrc, os.path.join(HERE, "c_abi", "host_tables_sanitized.cpp"),
                    os.path.join(csrc, "host_tables.cpp"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "host tables ok" in r.stdout


def test_library_host_code_under_sanitizers(tmp_path):
    """The whole library built with its host code under the address and undefined-behaviour
    sanitizers (build(sanitize=True)): the plain C program and the host tests of the
    binding (tests/test_lib_host.py) run against it with the sanitizer runtimes preloaded.
    Any out-of-bounds access, use after free, leak (C program) or undefined behaviour in
    the host side fails the run."""
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    asan, ubsan = (subprocess.run([gcc, f"-print-file-name={n}"], capture_output=True, text=True).stdout.strip()
                   for n in ("libasan.so", "libubsan.so"))
    if not (os.path.isabs(asan) and os.path.exists(asan) and os.path.isabs(ubsan) and os.path.exists(ubsan)):
        pytest.skip("sanitizer runtimes not available")
    from paper_1808_01517_gb300 import build
    lib = build.build(sanitize=True)
    env = dict(os.environ)
    env["LD_LIBRARY_PATH"] = ":".join(p for p in ("/usr/local/cuda/lib64", env.get("LD_LIBRARY_PATH", "")) if p)
    exe = str(tmp_path / "host_only_sanitized")
    subprocess.run([gcc, "-std=c99", "-O1", "-g", "-fsanitize=address,undefined", "-fno-omit-frame-pointer", "-Wall",
                    "-Werror", "-I", os.path.join(ROOT, "include"), os.path.join(HERE, "c_abi", "host_only.c"),
                    "-o", exe, lib, "-lm", "-Wl,-rpath," + os.path.dirname(lib)], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, env=dict(env, ASAN_OPTIONS="detect_leaks=1"),
                       timeout=120)
    assert r.returncode == 0 and "c abi ok" in r.stdout, r.stdout + r.stderr
    # the interpreter's own allocations are not the library's: no leak check under python
    py_env = dict(env, LD_PRELOAD=f"{asan} {ubsan}", ASAN_OPTIONS="detect_leaks=0:protect_shadow_gap=0",
                  DELIMIT_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "not gpu",
                        os.path.join(HERE, "test_lib_host.py")], capture_output=True, text=True, env=py_env,
                       cwd=ROOT, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
