"""Compile the FP64 CPU oracle (plain C + OpenMP) into ``oracle/liboracle.so``.

Test infrastructure: the oracle is the independent checker of the CUDA
library.  Building it is not using it; only the tests, the smoke check and
the CPU-baseline leg of the benchmark load it.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["orc.c", "orc_imex.c"]
LIB = os.path.join(HERE, "liboracle.so")


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = SOURCES + ["orc_core.h"]
    return any(os.path.getmtime(os.path.join(HERE, s)) > t for s in deps if os.path.exists(os.path.join(HERE, s)))


def build(force=False):
    """Build liboracle.so if it is missing or older than its sources."""
    if not force and not _stale():
        return LIB
    srcs = [os.path.join(HERE, s) for s in SOURCES if os.path.exists(os.path.join(HERE, s))]
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu99", "-fopenmp", "-fPIC", "-shared", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
