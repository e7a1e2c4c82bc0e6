"""Build the C++ oracle (oracle/cpp/*.cpp) into oracle/liboracle_cpp.so with g++.

Test infrastructure: the library never loads it.  Plain -O2, no target-specific flags,
so the same sources build on x86-64 and on the Arm hosts.  Rebuilds only when a source
is newer than the library.
"""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cpp")
LIB = os.path.join(HERE, "liboracle_cpp.so")


def build(force: bool = False) -> str:
    srcs = sorted(os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith(".cpp"))
    deps = srcs + [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".hpp", ".h"))]
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(p) for p in deps):
        return LIB
    cxx = os.environ.get("CXX") or shutil.which("g++") or "g++"
    cmd = [cxx, "-std=c++17", "-O2", "-fPIC", "-shared", *srcs, "-o", LIB + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"oracle build failed:\n{r.stdout}\n{r.stderr}")
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
