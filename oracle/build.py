"""Build the CPU oracle shared library (plain C, gcc).

TEST INFRASTRUCTURE ONLY: the oracle is loaded by tests, the smoke check and
the bench's CPU-baseline leg; the CUDA product path never touches it.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, f) for f in ("sw_oracle.c", "xy_oracle.c", "wolff_oracle.c")]
HDRS = [os.path.join(HERE, f) for f in ("sw_oracle.h", "xy_oracle.h", "wolff_oracle.h")]
LIB = os.path.join(HERE, "liboracle_sw.so")


def build(force: bool = False) -> str:
    """Compile the oracle's C files into liboracle_sw.so next to them; return
    the path."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(f) for f in SRCS + HDRS)):
        return LIB
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-Wall", "-Wextra",
           "-fno-fast-math", "-o", LIB + ".tmp"] + SRCS + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
