"""Compile the CPU oracle (test infrastructure) into oracle/libcos_oracle.so."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cos_oracle.c")
DEPS = [SRC, os.path.join(HERE, "oracle_impl.h"), os.path.join(HERE, "oracle_bip.h"),
        os.path.join(HERE, "oracle_det.h")]
LIB = os.path.join(HERE, "libcos_oracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(d) for d in DEPS):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, SRC, "-lquadmath", "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
