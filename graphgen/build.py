"""Builds the generator libraries in-tree (host C + its CUDA twin)."""
from __future__ import annotations

import os
import shutil
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
GENCODE = "-gencode=arch=compute_103a,code=sm_103a"


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)


def build_host():
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_HERE, "gg_host.c")
    out = os.path.join(_BUILD, "libgg_host.so")
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", src, "-o", out]
    try:
        _run(base[:1] + ["-fopenmp"] + base[1:])
    except RuntimeError:
        _run(base)  # same results without threads
    return out


def build_dev(nvcc=None):
    os.makedirs(_BUILD, exist_ok=True)
    nvcc = nvcc or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    src = os.path.join(_HERE, "gg_dev.cu")
    out = os.path.join(_BUILD, "libgg_dev.so")
    _run([nvcc, GENCODE, "-O3", "-lineinfo", "-shared", "-Xcompiler", "-fPIC", src, "-o", out])
    return out


def build():
    return build_host(), build_dev()


if __name__ == "__main__":
    print(build())
