"""Compiles the CPU oracle (plain C) into oracle/libmpv_oracle.so.

The oracle is test infrastructure: only the test suite, the smoke check and the
benchmark's CPU-baseline leg load it.  Built with -ffp-contract=off and no
machine-specific flags so that it gives the same results on x86-64 and AArch64.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mpv_oracle.c")
LIB = os.path.join(HERE, "libmpv_oracle.so")


def build(force: bool = False) -> str:
    hdr = os.path.join(HERE, "mpv_oracle.h")
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC), os.path.getmtime(hdr))):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-Wall", "-Wextra", "-o", tmp, SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
