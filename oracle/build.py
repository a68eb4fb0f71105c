"""Compile the FP64 CPU oracle (test infrastructure) into oracle/liboracle.so.

Plain gcc, no architecture-specific flags, FP contraction off so that the oracle gives the
same bits on x86-64 and aarch64 hosts.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")
SRC = os.path.join(HERE, "tt_oracle.c")


def build(force=False):
    hdr = os.path.join(HERE, "tt_oracle.h")
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC), os.path.getmtime(hdr))):
        return LIB
    tmp = LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c99", "-Wall", "-fPIC",
                           "-shared", "-o", tmp, SRC, "-lm"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
