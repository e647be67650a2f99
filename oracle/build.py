"""Build the FP64 CPU oracle (``oracle/liboracle.so``) with gcc.

Test infrastructure only.  ``-ffp-contract=off`` keeps the floating-point
results identical between the x86 build host and the Arm GPU host (no fused
multiply-add contraction on either).
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")
SRC = [os.path.join(HERE, "ora.c")]


def build(force: bool = False) -> str:
    newest = max(os.path.getmtime(p) for p in SRC + [os.path.join(HERE, "ora.h")])
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-shared",
           "-fPIC", *SRC, "-o", tmp, "-lm"]
    # OpenMP shares the independent cell loops over the host's cores; a
    # toolchain without it builds the same oracle single-threaded
    if subprocess.call(cmd[:1] + ["-fopenmp"] + cmd[1:], stdout=subprocess.DEVNULL,
                       stderr=subprocess.DEVNULL) != 0:
        subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
