"""Compile the C oracle into oracle/_orc.so (gcc, -O2, OpenMP).

Test infrastructure: the oracle is only loaded by the tests, the smoke check
and the CPU-baseline leg of the benchmark.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["lsys.c", "collide.c", "lbm.c"]
TARGET = os.path.join(HERE, "_orc.so")


def build(force: bool = False) -> str:
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    deps = srcs + [os.path.join(HERE, "orc.h")]
    if not force and os.path.exists(TARGET):
        t = os.path.getmtime(TARGET)
        if all(os.path.getmtime(d) <= t for d in deps):
            return TARGET
    tmp = TARGET + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-Wall", "-Wno-unused-function",
           "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, TARGET)
    return TARGET


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
