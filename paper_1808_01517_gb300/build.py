"""Builds the in-tree CUDA library ``_build/libdelimit.so`` for sm_103a with nvcc.

Translation units are compiled in parallel and linked with the CUDA runtime;
a unit is rebuilt only when its source or a header changed.  Used by
``__graft_entry__.build()`` and, on first import, by the Python binding.
"""
from __future__ import annotations

import glob
import hashlib
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libdelimit.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdelimit")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
                  + glob.glob(os.path.join(ROOT, "include", "*.h")))


def _digest(paths, extra=""):
    h = hashlib.sha256(extra.encode())
    for p in paths:
        with open(p, "rb") as f:
            h.update(p.encode() + b"\0" + f.read())
    return h.hexdigest()


# host code of the sanitized build: address and undefined-behaviour sanitizers (the
# device code is compiled as in the regular build)
SANITIZE_OUT = os.path.join(OUT, "sanitize")
SANITIZE_LIB = os.path.join(SANITIZE_OUT, "libdelimit.so")
SANITIZE_FLAGS = ["-Xcompiler=-fsanitize=address", "-Xcompiler=-fsanitize=undefined",
                  "-Xcompiler=-fno-omit-frame-pointer", "-Xcompiler=-fno-sanitize-recover=all"]


def build(verbose: bool = False, jobs: int = 8, sanitize: bool = False) -> str:
    """Compile every unit (if stale) and link libdelimit.so; returns the library path.

    sanitize: a separate build under ``_build/sanitize`` whose host code runs under the
    address and undefined-behaviour sanitizers (load it with the sanitizer runtimes
    preloaded), for checking the host side of the library on a machine without a GPU."""
    out_dir, lib_path = (SANITIZE_OUT, SANITIZE_LIB) if sanitize else (OUT, LIB)
    os.makedirs(out_dir, exist_ok=True)
    nvcc = _nvcc()
    hdr = _digest(_headers())
    host_opt = ["-Xcompiler", "-O1", "-g"] + SANITIZE_FLAGS if sanitize else ["-Xcompiler", "-O3"]
    flags = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC"] + host_opt + [
             "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")] + ARCH
    objs, jobs_list = [], []
    for src in _sources():
        obj = os.path.join(out_dir, os.path.basename(src) + ".o")
        stamp = obj + ".sha"
        key = _digest([src], hdr + " ".join(flags))
        objs.append(obj)
        if os.path.exists(obj) and os.path.exists(stamp) and open(stamp).read() == key:
            continue
        cmd = [nvcc, "-c", src, "-o", obj] + flags
        if src.endswith(".cpp"):
            cmd = [nvcc, "-x", "cu", "-c", src, "-o", obj] + flags
        jobs_list.append((cmd, stamp, key))

    def run(item):
        cmd, stamp, key = item
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        with open(stamp, "w") as f:
            f.write(key)
        return r.stdout + r.stderr

    with ThreadPoolExecutor(max_workers=jobs) as ex:
        for out in ex.map(run, jobs_list):
            if verbose and out.strip():
                print(out)
    relink = bool(jobs_list) or not os.path.exists(lib_path)
    if relink:
        tmp = lib_path + ".tmp"
        cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-lcudart"] + (SANITIZE_FLAGS if sanitize else [])
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(verbose=True))
