"""Compiles the host hybrid BFS (plain gcc with OpenMP, no GPU code)."""
from __future__ import annotations

import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(_HERE, "_build", "libhostbfs.so")


def build():
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    src = os.path.join(_HERE, "hostbfs.c")
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(src):
        return LIB
    cmd = ["gcc", "-O3", "-std=gnu11", "-fopenmp", "-shared", "-fPIC", src, "-o", LIB]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("hostbfs build failed:\n" + r.stdout + r.stderr)
    return LIB


if __name__ == "__main__":
    print(build())
