"""Build the FP64 CPU oracle (plain C) into oracle/_liborc.so.

Test infrastructure only: the test-suite, the smoke check and the benchmark's CPU-baseline leg load
it; the CUDA library never does. Compiled with -ffp-contract=off so that x86 and Arm hosts round the
same way (no fused multiply-add contraction).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["orc_basis.c", "orc_physics.c", "orc_dg.c", "orc_exact.c"]
LIB = os.path.join(HERE, "_liborc.so")


def build(force: bool = False) -> str:
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    deps = srcs + [os.path.join(HERE, "dg_oracle.h")]
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in deps):
            return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fPIC", "-shared",
           "-fopenmp", "-o", tmp] + srcs + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
