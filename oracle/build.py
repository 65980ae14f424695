"""Builds the CPU oracle (TEST INFRASTRUCTURE ONLY) into oracle/liboracle.so.

-ffp-contract=off keeps every binary32 decision expression free of fused
multiply-adds, so coverage and fragment order follow the stated formulas exactly.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")
SRC = [os.path.join(HERE, "ms_oracle.c"), os.path.join(HERE, "ms_oracle_splat.c")]


def build(force: bool = False) -> str:
    deps = SRC + [os.path.join(HERE, "ms_oracle.h")]
    if not force and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(s) for s in deps):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-pthread", *SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
