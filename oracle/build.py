"""Compiles the C oracle (plain gcc, no GPU code). Test infrastructure only."""
from __future__ import annotations

import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))


def build():
    out_dir = os.path.join(_HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    out = os.path.join(out_dir, "liboracle.so")
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", os.path.join(_HERE, "oracle.c"),
           "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("oracle build failed:\n" + r.stdout + r.stderr)
    return out


if __name__ == "__main__":
    print(build())
