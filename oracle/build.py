"""Build step of the FP64 CPU oracle (test infrastructure only).

Compiles ``ssm_oracle.c`` into ``libssm_oracle.so`` beside it with the host C
compiler.  Plain IEEE double: no fast-math, no fused multiply-add contraction, no
machine-specific flags, so the same source gives the same results on x86-64 and
aarch64 hosts.  OpenMP parallelises the loops over target particles only.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ssm_oracle.c")
LIB = os.path.join(HERE, "libssm_oracle.so")


def build_oracle(force: bool = False) -> str:
    """Compile the oracle if the shared library is missing or older than its source."""
    deps = [SRC, os.path.join(HERE, "ssm_oracle.h")]
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(p) for p in deps)):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force="--force" in sys.argv))
