"""Builds libsimplex.so in-tree for sm_103a (nvcc + g++, translation units in parallel).

    python -m paper_2208_11617_gb300.build          # build if sources changed
    python -m paper_2208_11617_gb300.build --force  # rebuild everything
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libsimplex.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _nvcc() -> str:
    p = shutil.which("nvcc") or os.path.join(CUDA_HOME, "bin", "nvcc")
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsimplex")
    return p


def _sources():
    cu = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    cpp = sorted(f for f in os.listdir(CSRC) if f.endswith(".cpp"))
    hdr = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hdr.append(os.path.join(INCLUDE, "simplex.h"))
    return cu, cpp, hdr


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every CUDA/C++ translation unit and link libsimplex.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    cu, cpp, hdr = _sources()
    nvcc = _nvcc()
    inc = [f"-I{CSRC}", f"-I{INCLUDE}", f"-I{os.path.join(CUDA_HOME, 'include')}"]
    jobs = []
    objs = []
    for f in cu:
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, f + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + hdr):
            cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-Xptxas", "-warn-spills", *inc, "-c", src, "-o", obj]
            jobs.append((f, cmd))
    for f in cpp:
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, f + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + hdr):
            cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-Wno-unknown-pragmas", *inc, "-c", src, "-o", obj]
            jobs.append((f, cmd))
    procs = [(f, cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True))
             for f, cmd in jobs]
    errors = []
    for f, cmd, pr in procs:
        out, _ = pr.communicate()
        if pr.returncode != 0:
            errors.append(f"--- {f}\n{' '.join(cmd)}\n{out}")
        elif verbose and out.strip():
            print(f"--- {f}\n{out}")
    if errors:
        raise RuntimeError("libsimplex build failed:\n" + "\n".join(errors))
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
               f"-L{os.path.join(CUDA_HOME, 'lib64')}"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("libsimplex link failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
