"""Build the CPU oracle (test infrastructure only) as a shared library.

Flags: -O2 for speed, -ffp-contract=off so that no multiply-add is fused and
every FP64 expression rounds exactly as written (the acceptance table and the
weight recursion are compared bit for bit).
"""
import os
import platform
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "muca_oracle.c")
LIB = os.path.join(HERE, "libmuca_oracle.so")


def build(force: bool = False) -> str:
    hdr = os.path.join(HERE, "muca_oracle.h")
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC), os.path.getmtime(hdr))):
        return LIB
    libs = ["-lm", "-lpthread"]
    if platform.machine() in ("x86_64", "AMD64", "i686"):
        libs.append("-lquadmath")
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
           "-Wall", "-Wextra", "-o", LIB + ".tmp", SRC] + libs
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
