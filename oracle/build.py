"""Build the CPU oracle shared library (plain C, gcc).

TEST INFRASTRUCTURE ONLY: the oracle is loaded by tests, the smoke check and
the bench's CPU-baseline leg; the CUDA product path never touches it.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sw_oracle.c")
LIB = os.path.join(HERE, "liboracle_sw.so")


def build(force: bool = False) -> str:
    """Compile sw_oracle.c into liboracle_sw.so next to it; return the path."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC),
                                             os.path.getmtime(os.path.join(HERE, "sw_oracle.h")))):
        return LIB
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-Wall", "-Wextra",
           "-fno-fast-math", "-o", LIB + ".tmp", SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
