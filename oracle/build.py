"""Build the CPU oracle (plain C, FP64) into oracle/liborc.so.

Test infrastructure only: the oracle checks the CUDA library and is never
linked or imported by it.  Compiled with -ffp-contract=off so that no fused
multiply-add changes the rounding of the stated formulas on either x86-64
or aarch64 hosts.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["rng.c", "collide.c", "transport.c", "init_moments.c"]
LIB = os.path.join(HERE, "liborc.so")


def build_oracle(force: bool = False) -> str:
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    deps = srcs + [os.path.join(HERE, "trmc_oracle.h")]
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in deps):
            return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-Wno-unused-function", "-pthread",
           "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force="--force" in sys.argv))
