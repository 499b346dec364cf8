"""Build the FP64 CPU oracle (test infrastructure only) into oracle/liboracle.so.

Plain gcc, no CUDA.  `-ffp-contract=off` keeps results identical on x86_64
and aarch64 hosts (gcc contracts a*b+c into FMA by default on aarch64).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["philox.c", "voigt.c", "scatter.c", "grid.c", "transport.c"]
HEADERS = ["oracle.h", "grid.h"]
LIB = os.path.join(HERE, "liboracle.so")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    for f in SOURCES + HEADERS + ["build.py"]:
        if os.path.getmtime(os.path.join(HERE, f)) > t:
            return True
    return False


def build(force: bool = False) -> str:
    if force or _stale():
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
               "-ffp-contract=off", "-fno-fast-math", "-Wall", "-Wno-unused-function",
               "-o", tmp] + [os.path.join(HERE, s) for s in SOURCES] + ["-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
