"""Compile the oracle (``oracle.c``) into ``liboracle.so`` with gcc.

Test infrastructure: the library is used by the tests, the package smoke
check and the benchmark's CPU-baseline leg only.  ``-ffp-contract=off`` keeps
every multiply and add a separately rounded IEEE double operation on every
host architecture (no fused multiply-add), so results are the same on x86-64
and aarch64.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-pthread", "-shared", SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
